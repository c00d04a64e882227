// C ABI of the solver (include/lbm.h): domain lifecycle, state
// initialisation, stepping, the steady-state loop, observables and
// read-back.  Compiled with -fmad=false: the FP64 initial state and read-back
// follow the definitions operation for operation.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>

#include "lbm.h"

#include "kernel_body.cuh"
#include "lbm_internal.cuh"

namespace lbm {
bool build_mask(const lbm_geometry_desc& g, uint8_t* out, lbm_geometry_info* info,
                std::string& err);
void mark_near_boundary(uint8_t* m, int nx, int ny);

StepPlan step_plan(int precision, int mode, Shape shape) {
    return precision == 0 ? step_plan_f64(mode, shape) : step_plan_lp(precision, mode, shape);
}

// The entries a plan's kernel runs.  The list holds the ntiles tiles, then
// the same tiles with the nchunks edge-cell chunks spread evenly among them:
// a plain step that takes the chunks runs the second part, the other kernels
// the first.  Its grid: one block per entry, or at most cap blocks (cap > 0)
// looping over them.
static void plan_entries(const StepPlan& pl, const int4* all, int nchunks, int ntiles, int cap, const int4** t,
                         int* n, int* grid) {
    *t = pl.edges ? all + ntiles : all;
    *n = pl.edges ? nchunks + ntiles : ntiles;
    *grid = std::max(1, cap > 0 ? std::min(cap, *n) : *n);
    if (pl.max_grid > 0) *grid = std::min(*grid, pl.max_grid);
}

cudaError_t launch_step(int precision, const InstDesc* insts, const int4* all, int nchunks, int ntiles,
                        int flip, int mode, Shape shape, int cap, cudaStream_t s) {
    const StepPlan pl = step_plan(precision, mode, shape);
    const int4* tiles = nullptr;
    int n = 0, grid = 0;
    plan_entries(pl, all, nchunks, ntiles, cap, &tiles, &n, &grid);
    if (n <= 0) return cudaSuccess;
    void* args[] = {&insts, &tiles, &n, &flip, &mode, &shape};
    return cudaLaunchKernel(pl.func, dim3(grid), pl.block, args, pl.smem, s);
}

StepPlan flow_plan(int precision, Shape shape, bool keep) {
    return precision == 0 ? flow_plan_f64(shape, keep) : flow_plan_lp(precision, shape, keep);
}

// grid must not exceed the co-resident capacity (the cooperative launch checks it)
cudaError_t launch_flow(int precision, const InstDesc* insts, const FlowArgs& fa, Shape shape,
                        bool keep, int grid, cudaStream_t s) {
    if (fa.ntiles <= 0 || fa.nsteps <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(fa.flags + 1, 0, (size_t)(fa.ntiles + 1) * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const StepPlan pl = flow_plan(precision, shape, keep);
    FlowArgs a = fa;
    void* args[] = {&insts, &a, &shape};
    return cudaLaunchCooperativeKernel(pl.func, dim3(grid), pl.block, args, pl.smem, s);
}
}  // namespace lbm

using namespace lbm;

// ---------------------------------------------------------------------------
// errors
static thread_local std::string g_err;

static lbm_status fail(lbm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

extern "C" const char* lbm_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// memory layout of one domain inside the caller's buffer
static constexpr size_t ALIGN = 256;
static size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }
static constexpr int MIN_TILE_AREA = 128;

static size_t store_size(int prec) {
    switch (prec) {
    case LBM_F64: return 8;
    case LBM_F32: return 4;
    case LBM_F16DEV: case LBM_BF16DEV: return 2;
    default: return 0;
    }
}
static size_t real_size(int prec) { return prec == LBM_F64 ? 8 : 4; }

struct Layout {
    int64_t npad, max_tiles, max_entries;
    size_t desc, obs, mask, tiles, nbr, flags, items, qcol, qtab, partials, usnap, pops, tmap, fold, edges, etypes,
        eoff, total;
    int64_t max_curved;
};

static int64_t max_tiles_for(int nx, int ny) {
    int64_t best = 0;
    for (int tw = 32; tw <= 256; tw *= 2) {
        const int th = (MIN_TILE_AREA + tw - 1) / tw;
        const int64_t n = (int64_t)((nx + tw - 1) / tw) * ((ny + th - 1) / th);
        best = std::max(best, n);
    }
    return best;
}

static bool make_layout(int nx, int ny, int prec, Layout& L) {
    const size_t ss = store_size(prec);
    if (!ss || nx <= 0 || ny <= 0) return false;
    const int64_t N = (int64_t)nx * ny;
    L.npad = (N + 127) / 128 * 128;
    if (13 * L.npad > (int64_t)INT32_MAX) return false;  // kernels index planes in 32 bits
    L.max_tiles = max_tiles_for(nx, ny);
    size_t off = 0;
    L.desc = off; off = align_up(off + sizeof(InstDesc));
    L.obs = off; off = align_up(off + NOBS * sizeof(double));
    L.mask = off; off = align_up(off + (size_t)L.npad);
    // tile list: the tiles, then the tiles with the edge-cell chunks (at most
    // one per 32 cells) spread among them
    L.max_entries = 2 * L.max_tiles + L.npad / 32 + 1;
    L.tiles = off; off = align_up(off + (size_t)L.max_entries * sizeof(int4));
    L.nbr = off; off = align_up(off + (size_t)L.max_tiles * 8 * sizeof(int));
    L.flags = off; off = align_up(off + (size_t)(L.max_tiles + 2) * sizeof(int));
    L.items = off; off = align_up(off + (size_t)SWEEP_MAX * L.max_tiles * sizeof(int4));
    // curved cornea cells: a few per column of the arc
    L.max_curved = 4 * ((int64_t)nx + ny) + 64;
    L.qcol = off; off = align_up(off + (size_t)(nx + 1) * sizeof(int32_t));
    L.qtab = off; off = align_up(off + (size_t)L.max_curved * sizeof(CurvedCell));
    L.partials = off; off = align_up(off + (size_t)L.max_tiles * NPART * sizeof(double));
    L.usnap = off; off = align_up(off + 2 * (size_t)L.npad * real_size(prec));
    L.pops = off; off = align_up(off + 13 * (size_t)L.npad * ss);
    L.tmap = off; off = align_up(off + sizeof(CUtensorMap));
    L.fold = off; off = align_up(off + ((size_t)FOLD_MAX * NPART + 1) * sizeof(double));
    // edge cells: at most one entry per cell, and per-tile offsets
    L.edges = off; off = align_up(off + (size_t)L.npad * sizeof(int32_t));
    L.etypes = off; off = align_up(off + (size_t)L.npad * sizeof(uint32_t));
    L.eoff = off; off = align_up(off + (size_t)(L.max_tiles + 1) * sizeof(int32_t));
    L.total = off;
    return true;
}

// ---------------------------------------------------------------------------
struct lbm_domain {
    int nx = 0, ny = 0, prec = 0;
    int64_t N = 0;
    Layout L{};
    lbm_geometry_info info{};
    std::vector<uint8_t> hmask;  // cell types with near-boundary bits
    cudaStream_t stream = nullptr;
    int num_sms = 1;
    int device = 0;              // CUDA device current at creation (the buffer's)
    char* base = nullptr;
    InstDesc h{};                // host copy of the device descriptor
    InstDesc* d_desc = nullptr;
    double* d_obs = nullptr;
    int4* d_tiles = nullptr;
    int* d_nbr = nullptr;             // 8 neighbour tiles per tile (-1: none)
    int* d_flags = nullptr;           // dataflow status, abort and progress words
    int4* d_items = nullptr;          // work items of one dataflow sweep
    int per_sweep = 0;                // items of one sweep
    int sweep_k = 1;                  // steps per sweep in effect
    bool periodic_x = false, periodic_y = false;
    bool coop = false;                // device supports cooperative launches
    int flow_grid = 0;                // co-resident blocks of the dataflow kernel
    int stall_tile = -1;              // test hook (lbm_debug_stall_tile)
    // steady-state loop: two pinned read-back slots of (observables, status)
    // and their completion events, so that one interval can run while the
    // host checks the previous one
    double* pin = nullptr;
    cudaEvent_t pin_ev[2] = {nullptr, nullptr};
    int ntiles = 0;
    int64_t tiled_cells = 0;
    int64_t n_edges = 0;              // edge cells (plain FP32-arithmetic steps)
    int nchunks = 0;                  // edge-cell chunks in d_tiles' second part
    int split = 0;                    // plain steps take the edge-cell chunks (Shape::split)
    int64_t active_cells = 0;         // fluid and porous cells
    int64_t slow_cells = 0;           // active cells of row segments that need the per-cell update
    std::vector<int4> hchunks;        // host copy of them (instance 0)
    lbm_launch launch{128, 1, 2, 0, LBM_STEP_PER_LAUNCH, 1, 0};
    lbm_params params{};
    bool have_params = false;
    int64_t step = 0;
    double u_seep = 0.0;              // lumped TM: current seepage speed
    double last_iop = 0.0;            // IOP of the last steady-state check
    // Pressure reference of the stored flow populations: the library stores
    // f_i - kappa_i p_ref (kappa_0 = -4 sigma, lambda on the axes, gamma on the
    // diagonals, Eq. 7) and runs the kernels with the outlet pressure
    // p_out - p_ref.  Guo's incompressible model is invariant under this
    // shift (every equilibrium, moment and boundary rule keeps its form with
    // p - p_ref in place of p), so it changes only the size of the stored
    // values: the steady-state loops move p_ref to the chamber pressure, and
    // the rounding of FP32 and 16-bit populations then scales with the
    // velocity and the pressure variation instead of the IOP.  Always 0 for
    // FP64 (bit parity with a plain evaluation).
    double p_ref = 0.0;
    double pin_pref[2] = {0.0, 0.0};  // p_ref of the interval in each pinned slot
    int checks_since_recenter = -1;   // steady-state checks since the last move of p_ref (-1: never)
    cudaGraphExec_t graph = nullptr;  // GRAPH_STEPS plain steps from an even step
    std::vector<int4> htiles;         // host copy of the tile list
    std::vector<int> hnbr;            // host copy of the neighbour lists
    int64_t n_curved = 0;             // cells with a curved-cornea link
    lbm_batch* batch = nullptr;       // batch this domain belongs to, if any
    cudaStream_t own_stream = nullptr;
    lbm_observables last_obs{};       // observables of the last steady-state check
    bool have_last_obs = false;
};

// plain steps captured per CUDA graph (even, so a replay returns to the same parity)
static constexpr int GRAPH_STEPS = 32;

// prec: the storage precision (it sets the cells each thread updates, hence
// the threads of a block: at most 256)
static bool launch_ok(const lbm_launch& l, int prec) {
    const bool tw_ok = l.tile_w == 32 || l.tile_w == 64 || l.tile_w == 128 || l.tile_w == 256;
    const bool rows_ok = cells_per_thread(prec, l.tile_w) >= 4 ? l.block_rows <= 256 / 32
                                                                : l.tile_w * l.block_rows <= 256;
    return tw_ok && l.block_rows >= 1 && l.rows_per_thread >= 1 && l.rows_per_thread <= 64 && rows_ok &&
           (int64_t)l.tile_w * l.block_rows * l.rows_per_thread >= MIN_TILE_AREA &&
           l.blocks_per_sm >= 0 && l.blocks_per_sm <= 32 &&
           (l.stepping == LBM_STEP_FLOW || l.stepping == LBM_STEP_PER_LAUNCH) &&
           l.sweep_steps >= 0 && l.sweep_steps <= SWEEP_MAX &&
           (l.sweep_lag == 0 || (l.sweep_lag >= 2 && l.sweep_lag <= 4096));
}

// wavefront lag between consecutive steps of a sweep, in bands (tile rows)
static constexpr int DEFAULT_SWEEP_LAG = 8;

static Shape shape_of(const lbm_launch& l, int split) {
    return Shape{l.tile_w, l.block_rows, l.rows_per_thread, split};
}

// FP32 grids take edge-cell chunks (Shape::split) when more than this share
// of their active cells lie in row segments that would otherwise run the
// per-cell update (the chunks' own per-cell work and the masked rows cost a
// few per cent of the interior rows' speed; 16-bit storages always take them)
constexpr double SPLIT_SHARE = 0.08;

// cap on the blocks of a step launch (0: one block per entry)
static int grid_cap(const lbm_domain* d) {
    return d->launch.blocks_per_sm > 0 ? d->launch.blocks_per_sm * d->num_sms : 0;
}

// Launch order of a domain's per-step kernels.  On a large tile list (many
// waves of blocks per step) tiles with boundary cells (slower: the general
// per-cell update) go first and pure tiles after, each in list order, so the
// last blocks of a step run fast tiles and the step's tail shortens.  Each
// entry carries its own tile index, so the order changes nothing else.  On
// small grids and merged batch lists the raster order measured faster, so
// they keep it.
static constexpr size_t BOUNDARY_FIRST_MIN_TILES = 4096;

static std::vector<int4> boundary_tiles_first(const std::vector<int4>& tiles) {
    if (tiles.size() < BOUNDARY_FIRST_MIN_TILES) return tiles;
    std::vector<int4> order;
    order.reserve(tiles.size());
    for (const int4& t : tiles)
        if (!(t.y & TILE_PURE)) order.push_back(t);
    for (const int4& t : tiles)
        if (t.y & TILE_PURE) order.push_back(t);
    return order;
}

// tile list: every tw x th tile holding at least one active cell
// Appends tiles with chunks spread evenly among them (chunk j before tile
// j * ntiles / nchunks).
static void append_interleaved(std::vector<int4>& out, const std::vector<int4>& tiles,
                               const std::vector<int4>& chunks) {
    size_t j = 0;
    for (size_t i = 0; i < tiles.size(); ++i) {
        while (j < chunks.size() && j * tiles.size() <= i * chunks.size()) out.push_back(chunks[j++]);
        out.push_back(tiles[i]);
    }
    while (j < chunks.size()) out.push_back(chunks[j++]);
}

static lbm_status build_tiles(lbm_domain* d) {
    const int tw = d->launch.tile_w, th = d->launch.block_rows * d->launch.rows_per_thread;
    const int ntx = (d->nx + tw - 1) / tw, nty = (d->ny + th - 1) / th;
    std::vector<int4> tiles;
    std::vector<int> at((size_t)ntx * nty, -1);  // tile index of a tile-grid cell, -1 if none
    int64_t cells = 0;
    for (int y0 = 0; y0 < d->ny; y0 += th) {
        for (int x0 = 0; x0 < d->nx; x0 += tw) {
            bool any = false;
            for (int y = y0; y < std::min(d->ny, y0 + th) && !any; ++y)
                for (int x = x0; x < std::min(d->nx, x0 + tw) && !any; ++x)
                    any = (d->hmask[(int64_t)y * d->nx + x] & TYPE_BITS) <= POROUS;
            if (any) {
                // pure: wholly inside the grid, fluid only, no cell linked to a boundary
                bool pure = x0 + tw <= d->nx && y0 + th <= d->ny;
                for (int y = y0; y < std::min(d->ny, y0 + th) && pure; ++y)
                    for (int x = x0; x < std::min(d->nx, x0 + tw) && pure; ++x)
                        pure = d->hmask[(int64_t)y * d->nx + x] == FLUID;
                at[(size_t)(y0 / th) * ntx + x0 / tw] = (int)tiles.size();
                tiles.push_back(make_int4(0, (int)tiles.size() | (pure ? TILE_PURE : 0), x0, y0));
                cells += (int64_t)std::min(tw, d->nx - x0) * std::min(th, d->ny - y0);
            }
        }
    }
    if ((int64_t)tiles.size() > d->L.max_tiles) return fail(LBM_EINVAL, "tile list overflow");
    // Edge cells (FP32-arithmetic kernels whose rows take the pair or vector
    // path: warps of 32 threads on a row, an even grid width).  A row is taken
    // in 64-cell segments from the tile's origin; the pair (x, x + 1), x even,
    // of a segment that lies wholly in the grid is interior when both cells
    // are fluid or porous and not next to a boundary (the kernels' mask test).
    // Every other active cell is an edge cell, which a plain step updates in
    // an edge-cell chunk: one cell per thread of a block.
    std::vector<int32_t> edges, eoff(tiles.size() + 1, 0);
    const int cpt = cells_per_thread(d->prec, tw);
    const bool pair_rows = d->prec != LBM_F64 && (tw / cpt) % 32 == 0 && d->nx % 2 == 0;
    int64_t active = 0, slow = 0;
    for (size_t k = 0; k < tiles.size(); ++k) {
        eoff[k] = (int32_t)edges.size();
        const int x0 = tiles[k].z, y0 = tiles[k].w;
        if (tiles[k].y & TILE_PURE) {
            active += (int64_t)tw * th;
            continue;
        }
        for (int y = y0; y < std::min(d->ny, y0 + th); ++y) {
            const uint8_t* row = d->hmask.data() + (int64_t)y * d->nx;
            for (int seg = x0; seg < std::min(d->nx, x0 + tw); seg += 64) {
                const int end = std::min(std::min(d->nx, seg + 64), x0 + tw);
                int n_act = 0;
                bool all_interior = pair_rows && seg + 64 <= d->nx;
                for (int x = seg; x < end; ++x) {
                    if ((row[x] & TYPE_BITS) <= POROUS) ++n_act;
                    if (row[x] & 0x0E) all_interior = false;
                }
                active += n_act;
                if (!all_interior) slow += n_act;
                if (!pair_rows) continue;
                for (int x = seg; x < end; ++x) {
                    if ((row[x] & TYPE_BITS) > POROUS) continue;
                    const int xp = x & ~1;
                    const bool interior = seg + 64 <= d->nx && (row[xp] & 0x0E) == 0 && (row[xp + 1] & 0x0E) == 0;
                    if (!interior) edges.push_back((int32_t)((int64_t)y * d->nx + x));
                }
            }
        }
    }
    d->active_cells = active;
    d->slow_cells = slow;
    d->split = pair_rows && (d->prec != LBM_F32 || (double)slow > SPLIT_SHARE * (double)std::max<int64_t>(active, 1));
    d->h.split = d->split;
    if (!d->split) {  // the rows update every cell: no edge cells
        edges.clear();
        std::fill(eoff.begin(), eoff.end(), 0);
    }
    // each edge cell's neighbour types, as cell_body reads them (links 1..8,
    // periodic wrap; only for a cell marked next to a boundary)
    std::vector<uint32_t> etypes(edges.size(), 0u);
    {
        static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        for (size_t e = 0; e < edges.size(); ++e) {
            const int64_t c = edges[e];
            const int y = (int)(c / d->nx), x = (int)(c - (int64_t)y * d->nx);
            if (!(d->hmask[c] & NEAR_BOUNDARY)) continue;
            uint32_t w = 0;
            for (int i = 1; i < 9; ++i) {
                const int xn = (x + EX[i] + d->nx) % d->nx, yn = (y + EY[i] + d->ny) % d->ny;
                w |= (uint32_t)(d->hmask[(int64_t)yn * d->nx + xn] & TYPE_BITS) << (4 * (i - 1));
            }
            etypes[e] = w;
        }
    }
    eoff[tiles.size()] = (int32_t)edges.size();
    if ((int64_t)edges.size() > d->L.npad) return fail(LBM_EINVAL, "edge list overflow");
    const int per_chunk = (tw / cpt) * d->launch.block_rows;  // threads of a block
    std::vector<int4> chunks;
    for (size_t e = 0; e < edges.size(); e += (size_t)per_chunk)
        chunks.push_back(make_int4(0, TILE_EDGE, (int)e, (int)std::min<size_t>(per_chunk, edges.size() - e)));
    if ((int64_t)(chunks.size() + 2 * tiles.size()) > d->L.max_entries) return fail(LBM_EINVAL, "tile list overflow");
    // neighbour tiles in the order of the links e_1..e_8, wrapping around
    // periodic edges only (no active cell lies on a non-periodic edge, so no
    // link crosses one)
    static const int tdx[8] = {1, 0, -1, 0, 1, -1, -1, 1};
    static const int tdy[8] = {0, 1, 0, -1, 1, 1, -1, -1};
    std::vector<int> nbr(tiles.size() * 8);
    for (size_t k = 0; k < tiles.size(); ++k) {
        const int tx = tiles[k].z / tw, ty = tiles[k].w / th;
        for (int i = 0; i < 8; ++i) {
            int ux = tx + tdx[i], uy = ty + tdy[i];
            if (d->periodic_x) ux = (ux + ntx) % ntx;
            if (d->periodic_y) uy = (uy + nty) % nty;
            const bool in = ux >= 0 && ux < ntx && uy >= 0 && uy < nty;
            nbr[k * 8 + i] = in ? at[(size_t)uy * ntx + ux] : -1;
        }
    }
    // one sweep of K steps in wavefront order: position j holds band j at
    // step 0, band j - L at step 1, ..., band j - (K-1) L at step K-1.  A
    // y-periodic grid links the first and last bands, which no single
    // wavefront orders, so it sweeps one step at a time.
    int K = std::max(1, d->launch.sweep_steps);
    if (d->periodic_y) K = 1;
    const int Lg = d->launch.sweep_lag > 0 ? d->launch.sweep_lag : DEFAULT_SWEEP_LAG;
    std::vector<int> band_start(nty + 1, 0);
    for (const int4& t : tiles) band_start[t.w / th + 1] += 1;
    for (int r = 0; r < nty; ++r) band_start[r + 1] += band_start[r];
    std::vector<int4> items;
    items.reserve((size_t)K * tiles.size());
    for (int j = 0; j < nty + (K - 1) * Lg; ++j)
        for (int k = 0; k < K; ++k) {
            const int r = j - k * Lg;
            if (r < 0 || r >= nty) continue;
            for (int t = band_start[r]; t < band_start[r + 1]; ++t)
                items.push_back(make_int4(k << 24, tiles[t].y, tiles[t].z, tiles[t].w));
        }
    d->sweep_k = K;
    d->per_sweep = (int)items.size();
    d->hnbr = nbr;
    d->ntiles = (int)tiles.size();
    d->tiled_cells = cells;
    d->h.ntiles = d->ntiles;
    d->htiles = tiles;
    // per-step launch order: the tiles, boundary tiles first (the longer
    // blocks start early); then the same with the edge-cell chunks spread
    // evenly among them, so that every SM mixes their latency-bound
    // per-cell work with streaming tiles
    const std::vector<int4> tile_order = boundary_tiles_first(tiles);
    std::vector<int4> launch_order = tile_order;
    append_interleaved(launch_order, tile_order, chunks);
    if (!tiles.empty()) {
        CK(cudaMemcpyAsync(d->d_tiles, launch_order.data(), launch_order.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, d->stream));
        CK(cudaMemcpyAsync(d->d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice,
                           d->stream));
        CK(cudaMemcpyAsync(d->d_items, items.data(), items.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, d->stream));
    }
    CK(cudaMemcpyAsync(d->base + d->L.eoff, eoff.data(), eoff.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                       d->stream));
    if (!edges.empty())
        CK(cudaMemcpyAsync(d->base + d->L.etypes, etypes.data(), etypes.size() * sizeof(uint32_t),
                           cudaMemcpyHostToDevice, d->stream));
    if (!edges.empty())
        CK(cudaMemcpyAsync(d->base + d->L.edges, edges.data(), edges.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, d->stream));
    d->n_edges = (int64_t)edges.size();
    d->nchunks = (int)chunks.size();
    d->hchunks = chunks;
    // co-resident blocks of the dataflow kernel for this shape
    d->flow_grid = 0;
    if (d->coop) {
        const StepPlan pl = flow_plan(d->prec, shape_of(d->launch, d->split), d->sweep_k > 1);
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl.func,
                                                         (int)(pl.block.x * pl.block.y), pl.smem));
        if (d->launch.blocks_per_sm > 0) per_sm = std::min(per_sm, d->launch.blocks_per_sm);
        d->flow_grid = per_sm * d->num_sms;
    }
    // pageable sources: make sure the copies have consumed them before they die
    CK(cudaStreamSynchronize(d->stream));
    return LBM_OK;
}

// Link fractions of the fluid cells next to the curved cornea of the analytic
// eye (Bouzidi's interpolated bounce-back): for each link i to a cold cell,
// the fraction q at which it leaves the cornea circle, the positive root of
// |P + t e_i - C|^2 = R^2 written with the half coefficient
// (a = |e_i|^2, bh = (P - C).e_i, c = |P - C|^2 - R^2,
// t = (-bh + sqrt(bh^2 - a c)) / a); q < 1/2 links whose upstream cell is not
// active fall back to halfway (q = 1/2).  Cells with any q != 1/2 get the
// CURVED mask bit and an entry, grouped by column.  Runs on the host before
// the mask is uploaded.
static lbm_status build_curved(lbm_domain* d) {
    const int nx = d->nx, ny = d->ny;
    std::vector<int32_t> qcol(nx + 1, 0);
    std::vector<std::vector<CurvedCell>> cols(nx);
    int64_t n = 0;
    const double R = d->info.arc_r;
    if (d->info.eye_normals && R > 0.0) {
        static const int EXh[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        static const int EYh[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        auto type_at = [&](int x, int y) -> int {
            if (x < 0 || x >= nx || y < 0 || y >= ny) return ADIABATIC;
            return d->hmask[(int64_t)y * nx + x] & TYPE_BITS;
        };
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                if (type_at(x, y) != FLUID) continue;
                CurvedCell e{};
                e.y = y;
                bool any = false;
                for (int i = 1; i < 9; ++i) {
                    double q = 0.5;
                    if (type_at(x + EXh[i], y + EYh[i]) == COLD) {
                        const double dx = x - d->info.arc_xc, dy = y - d->info.arc_yc;
                        const double a = (double)(EXh[i] * EXh[i] + EYh[i] * EYh[i]);
                        const double bh = dx * EXh[i] + dy * EYh[i];
                        const double c = dx * dx + dy * dy - R * R;
                        q = (-bh + std::sqrt(bh * bh - a * c)) / a;
                        if (q < 0.5 && type_at(x - EXh[i], y - EYh[i]) > POROUS) q = 0.5;
                    }
                    e.q[i - 1] = q;
                    any = any || q != 0.5;
                }
                if (!any) continue;
                cols[x].push_back(e);
                d->hmask[(int64_t)y * nx + x] |= CURVED;
                ++n;
            }
        }
    }
    if (n > d->L.max_curved) return fail(LBM_EINVAL, "curved-wall table overflow (%lld cells)", (long long)n);
    std::vector<CurvedCell> tab;
    tab.reserve((size_t)n);
    for (int x = 0; x < nx; ++x) {
        qcol[x] = (int32_t)tab.size();
        tab.insert(tab.end(), cols[x].begin(), cols[x].end());
    }
    qcol[nx] = (int32_t)tab.size();
    d->n_curved = n;
    CK(cudaMemcpyAsync(d->base + d->L.qcol, qcol.data(), qcol.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice, d->stream));
    if (!tab.empty())
        CK(cudaMemcpyAsync(d->base + d->L.qtab, tab.data(), tab.size() * sizeof(CurvedCell),
                           cudaMemcpyHostToDevice, d->stream));
    CK(cudaStreamSynchronize(d->stream));  // pageable sources
    return LBM_OK;
}

// The 16-bit vector path's constants in heat code units (value * Tscale),
// from the descriptor's parameters and heat encoding.
static void derive_code_units(InstDesc& h) {
    h.gbc = (float)((double)h.pf.g_beta * (double)h.Tstep);
    h.dT0c = (float)((double)h.pf.dT0 * (double)h.Tscale);
    h.Trefc = (float)((double)h.pf.Tref * (double)h.Tscale);
    h.rden = (float)(1.0 / h.pd.den);
}

static lbm_status upload_desc(lbm_domain* d) {
    derive_code_units(d->h);
    CK(cudaMemcpyAsync(d->d_desc, &d->h, sizeof(InstDesc), cudaMemcpyHostToDevice, d->stream));
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// element-wise kernels: initial state, read-back, write-back, finalisation

__device__ __forceinline__ uint64_t splitmix64(uint64_t state) {
    // SplitMix64 (Steele, Lea & Flood 2014)
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class ST>
__global__ void init_kernel(const InstDesc* __restrict__ dp, double noise_amp, uint64_t seed) {
    const InstDesc d = *dp;
    using T = typename ST::T;
    T* P = static_cast<T*>(d.pops);
    const int64_t N = (int64_t)d.nx * d.ny;
    // f^eq(p_out, u = 0), Eqs. 7-8: S_i(0) = w_i ((3*0 + 4.5*0*0) - 1.5*0)
    double feq[9];
    for (int i = 0; i < 9; ++i) {
        const double Si = wgt(i) * (3.0 * 0.0 + 4.5 * 0.0 * 0.0 - 1.5 * 0.0);
        const double a = i == 0 ? -4.0 * K_SIGMA : (i <= 4 ? K_LAMBDA : K_GAMMA);
        feq[i] = a * d.pd.p_out + Si;
    }
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const bool act = (d.mask[c] & TYPE_BITS) <= POROUS;
        if (!act) {
            for (int q = 0; q < 13; ++q) P[q * d.npad + c] = T(0.0f);
            continue;
        }
        double noise = 0.0;
        if (noise_amp != 0.0) {
            const uint64_t h = splitmix64(seed ^ (uint64_t)c);
            const double u01 = (double)(h >> 11) * 0x1.0p-53;
            noise = noise_amp * (2.0 * u01 - 1.0);
        }
        const double Ti = 0.25 * (d.pd.T0 + noise);
        for (int i = 0; i < 9; ++i) ST::stf(P + i * d.npad + c, (typename ST::R)feq[i], d);
        // heat populations are stored as deviations from Tshift
        for (int i = 1; i <= 4; ++i) ST::stT(P + (8 + i) * d.npad + c, (typename ST::R)(Ti - (double)d.Tshift), d);
    }
}

// natural-order population f_i (or T_i) of cell (x, y) at the given parity
__device__ __forceinline__ int64_t slot_of(const InstDesc& d, int x, int y, int i, int parity,
                                           bool heat) {
    const int64_t c = (int64_t)y * d.nx + x;
    if (parity == 0 || i == 0) return (heat ? (8 + i) : i) * d.npad + c;
    // odd: f_i(x) sits in slot (x - e_i, opp(i))
    int xs = x - ex(i), ys = y - ey(i);
    if (xs < 0) xs += d.nx;
    if (xs >= d.nx) xs -= d.nx;
    if (ys < 0) ys += d.ny;
    if (ys >= d.ny) ys -= d.ny;
    const int o = opp(i);
    return (heat ? (8 + o) : o) * d.npad + (int64_t)ys * d.nx + xs;
}

// stored flow populations are f_i - kappa_i p_ref
__device__ __forceinline__ double kappa(int i) { return i == 0 ? -4.0 * K_SIGMA : (i <= 4 ? K_LAMBDA : K_GAMMA); }

template <class ST>
__global__ void read_pops_kernel(const InstDesc* __restrict__ dp, int parity, double p_ref, double* __restrict__ f,
                                 double* __restrict__ g) {
    const InstDesc d = *dp;
    using T = typename ST::T;
    const T* P = static_cast<const T*>(d.pops);
    const int64_t N = (int64_t)d.nx * d.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t m = d.mask[c];
        const bool act = (m & TYPE_BITS) <= POROUS;
        const int x = (int)(c % d.nx), y = (int)(c / d.nx);
        if (f) {
            double fv[9];
            for (int i = 0; i < 9; ++i)
                fv[i] = act ? (double)ST::ldf(P + slot_of(d, x, y, i, parity, false), d) + kappa(i) * p_ref : 0.0;
            if (act && d.bouzidi && (m & CURVED)) {
                const CurvedCell* ce = curved_entry(d, x, y);
                if (ce) bouzidi_read<double>(ce, fv);
            }
            for (int i = 0; i < 9; ++i) f[i * N + c] = fv[i];
        }
        for (int i = 1; i <= 4; ++i)
            if (g)
                g[(i - 1) * N + c] =
                    act ? (double)ST::ldT(P + slot_of(d, x, y, i, parity, true), d) + (double)d.Tshift : 0.0;
    }
}

template <class ST>
__global__ void write_pops_kernel(const InstDesc* __restrict__ dp, int parity, double p_ref,
                                  const double* __restrict__ f, const double* __restrict__ g) {
    const InstDesc d = *dp;
    using T = typename ST::T;
    using R = typename ST::R;
    T* P = static_cast<T*>(d.pops);
    const int64_t N = (int64_t)d.nx * d.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t m = d.mask[c];
        if ((m & TYPE_BITS) > POROUS) continue;
        const int x = (int)(c % d.nx), y = (int)(c / d.nx);
        if (f) {
            double fv[9];
            for (int i = 0; i < 9; ++i) fv[i] = f[i * N + c];
            // curved cornea: store what the next read turns back into fv
            // (the inverse of the q < 1/2 completion)
            if (d.bouzidi && (m & CURVED)) {
                const CurvedCell* ce = curved_entry(d, x, y);
                for (int i = 1; ce && i < 9; ++i) {
                    const double q = ce->q[i - 1];
                    if (q < 0.5) fv[opp(i)] = (fv[opp(i)] - (1.0 - 2.0 * q) * fv[i]) / (2.0 * q);
                }
            }
            for (int i = 0; i < 9; ++i)
                ST::stf(P + slot_of(d, x, y, i, parity, false), (R)(fv[i] - kappa(i) * p_ref), d);
        }
        if (g)
            for (int i = 1; i <= 4; ++i)
                ST::stT(P + slot_of(d, x, y, i, parity, true), (R)(g[(i - 1) * N + c] - (double)d.Tshift), d);
    }
}

// Moves the pressure reference of the stored flow populations by dp: every
// population of an active cell (found in its slot at this parity) loses
// kappa_i dp.  The q < 1/2 completion of the curved cornea interpolates two
// slots with weights that add up to 1, so it shifts alike.
template <class ST>
__global__ void shift_pressure_kernel(const InstDesc* __restrict__ dp, int parity, double dpr) {
    const InstDesc d = *dp;
    using T = typename ST::T;
    using R = typename ST::R;
    T* P = static_cast<T*>(d.pops);
    const int64_t N = (int64_t)d.nx * d.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        if ((d.mask[c] & TYPE_BITS) > POROUS) continue;
        const int x = (int)(c % d.nx), y = (int)(c / d.nx);
        for (int i = 0; i < 9; ++i) {
            T* q = P + slot_of(d, x, y, i, parity, false);
            ST::stf(q, (R)((double)ST::ldf(q, d) - kappa(i) * dpr), d);
        }
    }
}

// Eq. 9 and Eq. 13 in FP64 on the stored populations
template <class ST>
__global__ void fields_kernel(const InstDesc* __restrict__ dp, int parity, double p_ref, double* __restrict__ u,
                              double* __restrict__ p, double* __restrict__ Tf) {
    const InstDesc d = *dp;
    using T = typename ST::T;
    const T* P = static_cast<const T*>(d.pops);
    const int64_t N = (int64_t)d.nx * d.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N;
         c += (int64_t)gridDim.x * blockDim.x) {
        const bool act = (d.mask[c] & TYPE_BITS) <= POROUS;
        double ux = 0.0, uy = 0.0, pp = 0.0, TT = 0.0;
        if (act) {
            const int x = (int)(c % d.nx), y = (int)(c / d.nx);
            double fv[9], gv[4];
            for (int i = 0; i < 9; ++i) fv[i] = (double)ST::ldf(P + slot_of(d, x, y, i, parity, false), d);
            for (int i = 1; i <= 4; ++i)
                gv[i - 1] = (double)ST::ldT(P + slot_of(d, x, y, i, parity, true), d) + (double)d.Tshift;
            if (d.bouzidi && (d.mask[c] & CURVED)) {
                const CurvedCell* ce = curved_entry(d, x, y);
                if (ce) bouzidi_read<double>(ce, fv);
            }
            ux = fv[1] - fv[3] + fv[5] - fv[6] - fv[7] + fv[8];
            uy = fv[2] - fv[4] + fv[5] + fv[6] - fv[7] - fv[8];
            const double usq = ux * ux + uy * uy;
            const double S0 = K_W0 * (-1.5 * usq);
            const double s = fv[1] + fv[2] + fv[3] + fv[4] + fv[5] + fv[6] + fv[7] + fv[8];
            pp = (s + S0) / (4.0 * K_SIGMA) + p_ref;
            TT = gv[0] + gv[1] + gv[2] + gv[3];
        }
        if (u) { u[c] = ux; u[N + c] = uy; }
        if (p) p[c] = pp;
        if (Tf) Tf[c] = TT;
    }
}

// Observables of an instance from its folded partials a[NPART].
__device__ void write_obs(const InstDesc& d, const double* a) {
    double* o = d.obs;
    o[O_IOP] = a[P_N_FLUID] > 0.0 ? a[P_SUM_P] / a[P_N_FLUID] : 0.0;
    o[O_Q_IN] = a[P_Q_IN];
    o[O_Q_OUT] = a[P_Q_OUT];
    o[O_MASS] = a[P_MASS];
    o[O_PEAK] = sqrt(a[P_PEAK]);  // the partials hold max |u|^2
    o[O_WSS_C] = a[P_N_C] > 0.0 ? a[P_WSS_C] / a[P_N_C] : 0.0;
    o[O_WSS_I] = a[P_N_I] > 0.0 ? a[P_WSS_I] / a[P_N_I] : 0.0;
    o[O_RESID] = d.snap_valid ? sqrt(a[P_RESID]) : -1.0;
    o[O_N_FLUID] = a[P_N_FLUID];
    o[O_N_C] = a[P_N_C];
    o[O_N_I] = a[P_N_I];
    o[O_NAN] = (a[P_NAN] > 0.0 || !isfinite(a[P_SUM_P]) || !isfinite(a[P_MASS])) ? 1.0 : 0.0;
}

// Folds the per-tile partials of each instance in a fixed order, so the
// result does not depend on how tiles were scheduled or on which other
// instances ran.  fb blocks share an instance: block b folds the b-th of fb
// contiguous tile ranges (thread-strided, then a fixed binary tree) and
// stores its partial; the block that arrives last folds the fb partials in
// block order and writes the observables.  GB300's FP64 pipe is narrow, so
// one block per instance made this fold the long pole of a check interval
// on large grids.
__global__ void __launch_bounds__(256) finalize_kernel(const InstDesc* __restrict__ insts, int fb) {
    const int inst = blockIdx.x / fb, b = blockIdx.x - inst * fb;
    const InstDesc& d = insts[inst];
    __shared__ double sm[256][NPART];
    __shared__ int last;
    double acc[NPART];
    for (int k = 0; k < NPART; ++k) acc[k] = 0.0;
    const int nt = d.ntiles;
    const int chunk = (nt + fb - 1) / fb;
    const int t1 = min(nt, (b + 1) * chunk);
    for (int t = b * chunk + (int)threadIdx.x; t < t1; t += blockDim.x) {
        const double* q = d.partials + (int64_t)t * NPART;
        for (int k = 0; k < NSUM; ++k) acc[k] += q[k];
        for (int k = NSUM; k < NPART; ++k) acc[k] = fmax(acc[k], q[k]);
    }
    for (int k = 0; k < NPART; ++k) sm[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            for (int k = 0; k < NSUM; ++k) sm[threadIdx.x][k] += sm[threadIdx.x + s][k];
            for (int k = NSUM; k < NPART; ++k)
                sm[threadIdx.x][k] = fmax(sm[threadIdx.x][k], sm[threadIdx.x + s][k]);
        }
        __syncthreads();
    }
    if (fb == 1) {
        if (threadIdx.x == 0) write_obs(d, sm[0]);
        return;
    }
    double* const part = d.fold;
    unsigned int* const arrived = reinterpret_cast<unsigned int*>(d.fold + FOLD_MAX * NPART);
    if (threadIdx.x < NPART) part[b * NPART + threadIdx.x] = sm[0][threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(arrived, 1u) == (unsigned int)(fb - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < NPART) {
        const int k = threadIdx.x;
        double v = __ldcg(part + k);
        for (int bb = 1; bb < fb; ++bb) {
            const double w = __ldcg(part + bb * NPART + k);
            v = k < NSUM ? v + w : fmax(v, w);
        }
        sm[0][k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        write_obs(d, sm[0]);
        *arrived = 0u;  // ready for the next fold
    }
}

namespace lbm {
cudaError_t launch_finalize(const InstDesc* insts, int ninst, cudaStream_t s) {
    if (ninst <= 0) return cudaSuccess;
    // a few dozen blocks in all: one instance spreads over FOLD_MAX blocks,
    // a batch of 64 or more takes one block each
    const int fb = std::max(1, std::min(FOLD_MAX, 64 / ninst));
    finalize_kernel<<<ninst * fb, 256, 0, s>>>(insts, fb);
    return cudaGetLastError();
}
}  // namespace lbm

static int ew_grid(const lbm_domain* d) {
    const int64_t blocks = (d->N + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)d->num_sms * 16));
}

#define DISPATCH(prec, KERNEL, ...)                                                              \
    switch (prec) {                                                                              \
    case LBM_F64: KERNEL<StF64><<<ew_grid(d), 256, 0, d->stream>>>(__VA_ARGS__); break;          \
    case LBM_F32: KERNEL<StF32><<<ew_grid(d), 256, 0, d->stream>>>(__VA_ARGS__); break;          \
    case LBM_F16DEV: KERNEL<StF16><<<ew_grid(d), 256, 0, d->stream>>>(__VA_ARGS__); break;       \
    default: KERNEL<StBF16><<<ew_grid(d), 256, 0, d->stream>>>(__VA_ARGS__); break;              \
    }

// ---------------------------------------------------------------------------
// geometry (host only)

extern "C" lbm_status lbm_build_mask(const lbm_geometry_desc* desc, uint8_t* host_out,
                                     lbm_geometry_info* info) {
    if (!desc) return fail(LBM_EINVAL, "null geometry");
    std::string err;
    if (!build_mask(*desc, host_out, info, err)) return fail(LBM_EINVAL, "%s", err.c_str());
    return LBM_OK;
}

extern "C" size_t lbm_domain_bytes(const lbm_geometry_desc* desc, int32_t precision) {
    if (!desc) return 0;
    Layout L;
    if (!make_layout(desc->nx, desc->ny, precision, L)) return 0;
    return L.total;
}

// Bulk tensor copy map of the populations for the staged kernel: the 13
// planes as an nx x ny x 13 tensor, boxes of 64 x 1 x 13 (a row segment's
// own slots on an even step; out-of-grid elements are filled with zeros and
// never used).  Returns false where the driver offers no encoder or the rows
// are not 16-byte aligned; the staged kernel then copies row pieces one
// plane at a time.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn tensor_encoder() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && p)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            (void)cudaGetLastError();
    }
    return fn;
}

static bool encode_pop_map(const lbm_domain* d, CUtensorMap* map) {
    if (d->prec == LBM_F64) return false;
    const int es = (int)store_size(d->prec);
    if (d->nx % (16 / es) != 0) return false;
    const EncodeTiledFn enc = tensor_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt =
        d->prec == LBM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t dims[3] = {(cuuint64_t)d->nx, (cuuint64_t)d->ny, 13};
    const cuuint64_t strides[2] = {(cuuint64_t)d->nx * es, (cuuint64_t)d->L.npad * es};
    const cuuint32_t box[3] = {(cuuint32_t)WS_SEG, 1, 13};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, dt, 3, d->base + d->L.pops, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

extern "C" lbm_status lbm_create_domain(const lbm_geometry_desc* desc, int32_t precision,
                                        void* dev_buf, size_t bytes, void* stream,
                                        lbm_domain** out) {
    if (!desc || !out) return fail(LBM_EINVAL, "null argument");
    *out = nullptr;
    if (!store_size(precision)) return fail(LBM_EINVAL, "unknown precision %d", precision);
    lbm_domain* d = new (std::nothrow) lbm_domain();
    if (!d) return fail(LBM_ENOMEM, "host allocation failed");
    d->nx = desc->nx;
    d->ny = desc->ny;
    d->prec = precision;
    d->N = (int64_t)d->nx * d->ny;
    std::string err;
    if (d->nx <= 0 || d->ny <= 0 || !make_layout(d->nx, d->ny, precision, d->L)) {
        delete d;
        return fail(LBM_EINVAL, "invalid grid %d x %d", desc->nx, desc->ny);
    }
    d->hmask.assign((size_t)d->N, 0);
    if (!build_mask(*desc, d->hmask.data(), &d->info, err)) {
        delete d;
        return fail(LBM_EINVAL, "%s", err.c_str());
    }
    mark_near_boundary(d->hmask.data(), d->nx, d->ny);
    if (!dev_buf || bytes < d->L.total || (reinterpret_cast<uintptr_t>(dev_buf) % ALIGN) != 0) {
        const size_t need = d->L.total;
        delete d;
        return fail(LBM_ENOMEM, "device buffer too small or not 256-byte aligned (need %zu bytes)", need);
    }
    d->stream = static_cast<cudaStream_t>(stream);
    d->base = static_cast<char*>(dev_buf);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete d;
        return fail(LBM_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    d->device = dev;
    d->d_desc = reinterpret_cast<InstDesc*>(d->base + d->L.desc);
    d->d_obs = reinterpret_cast<double*>(d->base + d->L.obs);
    d->d_tiles = reinterpret_cast<int4*>(d->base + d->L.tiles);
    d->d_nbr = reinterpret_cast<int*>(d->base + d->L.nbr);
    d->d_flags = reinterpret_cast<int*>(d->base + d->L.flags);
    d->d_items = reinterpret_cast<int4*>(d->base + d->L.items);
    d->periodic_x = desc->kind == LBM_GEOM_MASK && desc->periodic_x != 0;
    d->periodic_y = desc->kind == LBM_GEOM_MASK && desc->periodic_y != 0;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess)
        d->coop = coop != 0;
    InstDesc& h = d->h;
    std::memset(&h, 0, sizeof(h));
    h.pops = d->base + d->L.pops;
    h.mask = reinterpret_cast<const uint8_t*>(d->base + d->L.mask);
    h.usnap = d->base + d->L.usnap;
    h.partials = reinterpret_cast<double*>(d->base + d->L.partials);
    h.edges = reinterpret_cast<const int32_t*>(d->base + d->L.edges);
    h.eoff = reinterpret_cast<const int32_t*>(d->base + d->L.eoff);
    h.etypes = reinterpret_cast<const uint32_t*>(d->base + d->L.etypes);
    h.obs = d->d_obs;
    h.npad = d->L.npad;
    h.nx = d->nx;
    h.ny = d->ny;
    h.inlet_dir_x = d->info.inlet_dir_x;
    h.inlet_dir_y = d->info.inlet_dir_y;
    h.inlet_profile = d->info.inlet_profile;
    h.inlet_lo = d->info.inlet_lo;
    h.inlet_width = d->info.inlet_width > 0 ? d->info.inlet_width : 1;
    h.eye_normals = d->info.eye_normals;
    h.outlet_axis = d->info.outlet_axis;
    h.arc_xc = d->info.arc_xc;
    h.arc_yc = d->info.arc_yc;
    h.fscale = precision == LBM_F16DEV ? 4096.0f : 1.0f;
    h.finv = 1.0f / h.fscale;
    lbm_status st;
    if ((st = build_curved(d)) != LBM_OK) {
        delete d;
        return st;
    }
    h.fold = reinterpret_cast<double*>(d->base + d->L.fold);
    h.qcol = reinterpret_cast<const int32_t*>(d->base + d->L.qcol);
    h.qtab = reinterpret_cast<const CurvedCell*>(d->base + d->L.qtab);
    cudaError_t ce = cudaMemcpyAsync(d->base + d->L.mask, d->hmask.data(), (size_t)d->N,
                                     cudaMemcpyHostToDevice, d->stream);
    if (ce != cudaSuccess) {
        delete d;
        return fail(LBM_ECUDA, "mask upload failed: %s", cudaGetErrorString(ce));
    }
    CUtensorMap map;
    if (encode_pop_map(d, &map)) {
        // pageable source: the copy has consumed it when the call returns
        ce = cudaMemcpy(d->base + d->L.tmap, &map, sizeof(map), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            delete d;
            return fail(LBM_ECUDA, "tensor map upload failed: %s", cudaGetErrorString(ce));
        }
        h.tmap = d->base + d->L.tmap;
    }
    ce = cudaMemsetAsync(d->base + d->L.fold, 0, ((size_t)FOLD_MAX * NPART + 1) * sizeof(double), d->stream);
    if (ce != cudaSuccess) {
        delete d;
        return fail(LBM_ECUDA, "fold counter reset failed: %s", cudaGetErrorString(ce));
    }
    ce = cudaMemsetAsync(d->d_flags, 0, sizeof(int), d->stream);
    if (ce != cudaSuccess) {
        delete d;
        return fail(LBM_ECUDA, "status word reset failed: %s", cudaGetErrorString(ce));
    }
    if ((st = build_tiles(d)) != LBM_OK || (st = upload_desc(d)) != LBM_OK) {
        delete d;
        return st;
    }
    *out = d;
    return LBM_OK;
}

static void drop_graph(lbm_domain* d) {
    if (d->graph) cudaGraphExecDestroy(d->graph);
    d->graph = nullptr;
}

extern "C" lbm_status lbm_batch_remove(lbm_batch* b, lbm_domain* d);

extern "C" void lbm_destroy_domain(lbm_domain* d) {
    if (!d) return;
    if (d->batch) lbm_batch_remove(d->batch, d);
    cudaStreamSynchronize(d->stream);
    drop_graph(d);
    if (d->pin) cudaFreeHost(d->pin);
    for (cudaEvent_t e : d->pin_ev)
        if (e) cudaEventDestroy(e);
    delete d;
}

// ---------------------------------------------------------------------------
// parameters

static bool finite_all(const lbm_params& p) {
    const double v[] = {p.tau, p.tau_T, p.g_beta, p.g_dir[0], p.g_dir[1], p.T_cold, p.T_hot,
                        p.T0, p.T_in, p.u_in_max, p.K_tm, p.porosity, p.p_out, p.drive[0],
                        p.drive[1], p.noise_amp, p.dx_m, p.dt_s, p.rho0, p.p_sc_pa};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

static void update_seepage(lbm_domain* d, double iop);

// validates p and derives the descriptor's parameter fields (no upload)
// Reference of the stored heat deviations in both parameter blocks: Tref =
// 4 Tshift (fixed when the state is initialised), dT0 = T0 - Tref.
static void sync_heat_reference(lbm_domain* d) {
    const double Tref = 4.0 * (double)d->h.Tshift;
    d->h.pd.Tref = Tref;
    d->h.pd.dT0 = d->params.T0 - Tref;
    d->h.pf.Tref = (float)Tref;
    d->h.pf.dT0 = (float)(d->params.T0 - Tref);
}

// Heat encoding fixed at initialisation: every storage but FP64 holds T_i -
// T0/4; the 16-bit storages hold it as companded 16-bit fixed point
// (enc_tfix).  |T - T0| <= span for a temperature field between the wall,
// inflow and reference temperatures, so |T_i - T0/4| <= span/4 near
// equilibrium: the fine part of the code carries that with 10 % to spare,
// plus the advective part (T/2) e.u of the equilibrium up to |u| = 0.04.
// The coarse part reaches 3.67 times as far, past the 3/4 span that
// anti-bounce-back can return while a boundary layer forms.
static void set_heat_encoding(lbm_domain* d) {
    const lbm_params& p = d->params;
    d->h.Tshift = d->prec == LBM_F64 ? 0.0f : (float)(0.25 * p.T0);
    const double span = std::max({std::fabs(p.T_cold - p.T0), std::fabs(p.T_hot - p.T0),
                                  std::fabs(p.T_in - p.T0), std::fabs(p.noise_amp)});
    const double tmax = std::max({std::fabs(p.T_cold), std::fabs(p.T_hot), std::fabs(p.T_in), std::fabs(p.T0)});
    const double fine = 1.1 * 0.25 * span + 0.02 * tmax + 1e-6;
    d->h.Tstep = (float)(fine / TFIX_KNEE);
    d->h.Tscale = 1.0f / d->h.Tstep;
    sync_heat_reference(d);
}

static lbm_status apply_params(lbm_domain* d, const lbm_params* p) {
    if (!d || !p) return fail(LBM_EINVAL, "null argument");
    if (!finite_all(*p)) return fail(LBM_EINVAL, "non-finite parameter");
    if (!(p->tau > 0.5)) return fail(LBM_EINVAL, "tau must exceed 1/2 (nu > 0, Eq. 10)");
    if (!(p->tau_T > 0.5)) return fail(LBM_EINVAL, "tau_T must exceed 1/2 (theta > 0, Eq. 14)");
    if (!(p->K_tm > 0.0)) return fail(LBM_EINVAL, "K_tm must be positive");
    const double gn = std::sqrt(p->g_dir[0] * p->g_dir[0] + p->g_dir[1] * p->g_dir[1]);
    if (p->g_beta != 0.0 && std::fabs(gn - 1.0) > 1e-9) return fail(LBM_EINVAL, "g_dir must be a unit vector");
    if (p->porosity < 0.0 || p->porosity > 1.0) return fail(LBM_EINVAL, "porosity must lie in [0, 1]");
    if (p->rho0 < 0.0 || p->dx_m < 0.0 || p->dt_s < 0.0) return fail(LBM_EINVAL, "negative unit scale");
    if (p->tm_model != 0 && p->tm_model != 1) return fail(LBM_EINVAL, "tm_model must be 0 or 1");
    if (p->tm_model == 1 && !(std::isfinite(p->h_tm) && p->h_tm > 0.0))
        return fail(LBM_EINVAL, "the lumped TM needs a positive thickness h_tm");
    if (p->bouzidi != 0 && p->bouzidi != 1) return fail(LBM_EINVAL, "bouzidi must be 0 or 1");
    d->h.tm_model = p->tm_model;
    d->h.bouzidi = p->bouzidi;
    Phys<double>& h = d->h.pd;
    h.omega = 1.0 / p->tau;
    h.omegaT = 1.0 / p->tau_T;
    h.g_beta = p->g_beta;
    h.gx = p->g_dir[0];
    h.gy = p->g_dir[1];
    h.T_cold = p->T_cold;
    h.T_hot = p->T_hot;
    h.T0 = p->T0;
    h.T_in = p->T_in;
    h.u_in_max = p->u_in_max;
    const double nu = (2.0 * p->tau - 1.0) / 6.0;  // Eq. 10
    h.cK = nu / p->K_tm;
    h.den = 1.0 + 0.5 * h.cK;
    h.p_out = p->p_out - d->p_ref;  // kernels run relative to p_ref
    h.drive_x = p->drive[0];
    h.drive_y = p->drive[1];
    h.kwss = -(1.0 - 1.0 / (2.0 * p->tau));
    Phys<float>& f = d->h.pf;
    f.omega = (float)h.omega;
    f.omegaT = (float)h.omegaT;
    f.g_beta = (float)h.g_beta;
    f.gx = (float)h.gx;
    f.gy = (float)h.gy;
    f.T_cold = (float)h.T_cold;
    f.T_hot = (float)h.T_hot;
    f.T0 = (float)h.T0;
    f.T_in = (float)h.T_in;
    f.u_in_max = (float)h.u_in_max;
    f.cK = (float)h.cK;
    f.den = (float)h.den;
    f.p_out = (float)h.p_out;
    f.drive_x = (float)h.drive_x;
    f.drive_y = (float)h.drive_y;
    f.kwss = (float)h.kwss;
    h.u_seep = d->u_seep;
    f.u_seep = (float)d->u_seep;
    d->params = *p;
    sync_heat_reference(d);
    return LBM_OK;
}

extern "C" lbm_status lbm_set_params(lbm_domain* d, const lbm_params* p) {
    if (!d || !p) return fail(LBM_EINVAL, "null argument");
    const bool changed = !d->have_params || std::memcmp(&d->params, p, sizeof(lbm_params)) != 0;
    lbm_status st = apply_params(d, p);
    if (st != LBM_OK) return st;
    const bool first = !d->have_params;
    d->have_params = true;
    if (first) return lbm_reset_state(d);
    if (changed) {
        // a new parameter set starts a new approach to steady state: the old
        // velocity snapshot no longer measures convergence, and the lumped
        // meshwork's seepage speed follows the new K, nu or h_tm at once
        d->h.snap_valid = 0;
        update_seepage(d, d->last_iop);
    }
    return upload_desc(d);
}

extern "C" lbm_status lbm_reset_state(lbm_domain* d) {
    if (!d) return fail(LBM_EINVAL, "null domain");
    if (!d->have_params) return fail(LBM_EINVAL, "set parameters before resetting the state");
    set_heat_encoding(d);
    // the initial state f = feq(p_out, 0) is all zeros relative to p_ref = p_out
    d->p_ref = d->prec == LBM_F64 ? 0.0 : d->params.p_out;
    d->checks_since_recenter = -1;
    d->h.pd.p_out = d->params.p_out - d->p_ref;
    d->h.pf.p_out = (float)d->h.pd.p_out;
    d->h.snap_valid = 0;
    d->h.parity = 0;
    d->u_seep = 0.0;
    d->last_iop = d->params.p_out;
    d->h.pd.u_seep = 0.0;
    d->h.pf.u_seep = 0.0f;
    lbm_status st = upload_desc(d);
    if (st != LBM_OK) return st;
    DISPATCH(d->prec, init_kernel, d->d_desc, d->params.noise_amp, d->params.seed);
    CK(cudaGetLastError());
    d->step = 0;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// stepping

static lbm_status step_once(lbm_domain* d, int mode) {
    CK(launch_step(d->prec, d->d_desc, d->d_tiles, d->nchunks, d->ntiles, (int)(d->step & 1), mode,
                   shape_of(d->launch, d->split), grid_cap(d), d->stream));
    if (mode == 0 || (mode & OBS_WRITE)) d->step += 1;
    return LBM_OK;
}

// Builds (once per launch shape) a graph of GRAPH_STEPS chained plain steps
// with alternating parity, replayed by lbm_step from an even step.
// A CUDA graph of n chained plain steps with alternating parity.  The steps
// are captured with programmatic dependent launch: step k + 1 may start while
// step k drains, its blocks reading their tile entry and descriptor and then
// waiting (griddepcontrol.wait) until step k has completed and its writes are
// visible, so the launch latency and block ramp-up of each step overlap the
// previous step's tail.  Falls back to plain dependencies where that is not
// available.
static cudaError_t capture_step_graph(int prec, const InstDesc* insts, const int4* all, int nchunks,
                                      int ntiles, Shape sh, int cap, int nsteps, bool pdl,
                                      cudaGraphExec_t* out) {
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return e;
    }
    const StepPlan pl = step_plan(prec, 0, sh);
    const int4* tiles = nullptr;
    int n = 0, gsz = 0;
    plan_entries(pl, all, nchunks, ntiles, cap, &tiles, &n, &gsz);
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
        const InstDesc* a0 = insts;
        const int4* a1 = tiles;
        int a2 = n, a3 = k & 1, a4 = 0;
        Shape a5 = sh;
        void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(gsz);
        cfg.blockDim = pl.block;
        cfg.dynamicSmemBytes = pl.smem;
        cfg.stream = cs;
        cfg.attrs = (pdl && k > 0) ? attr : nullptr;
        cfg.numAttrs = (pdl && k > 0) ? 1 : 0;
        e = cudaLaunchKernelExC(&cfg, pl.func, args);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return e;
}

static cudaError_t step_graph(int prec, const InstDesc* insts, const int4* all, int nchunks, int ntiles,
                              Shape sh, int cap, int nsteps, cudaGraphExec_t* out) {
    *out = nullptr;
    cudaError_t e = capture_step_graph(prec, insts, all, nchunks, ntiles, sh, cap, nsteps, true, out);
    if (e == cudaSuccess) return e;
    (void)cudaGetLastError();  // clear the failed attempt
    *out = nullptr;
    return capture_step_graph(prec, insts, all, nchunks, ntiles, sh, cap, nsteps, false, out);
}

// GRAPH_STEPS plain steps from an even step, replayed by lbm_step
static lbm_status ensure_graph(lbm_domain* d) {
    if (d->graph) return LBM_OK;
    const cudaError_t e = step_graph(d->prec, d->d_desc, d->d_tiles, d->nchunks, d->ntiles, shape_of(d->launch, d->split),
                                     grid_cap(d), GRAPH_STEPS, &d->graph);
    if (e != cudaSuccess) {
        d->graph = nullptr;
        return fail(LBM_ECUDA, "graph construction failed: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_step(lbm_domain* d, int64_t nsteps) {
    if (!d) return fail(LBM_EINVAL, "null domain");
    if (!d->have_params) return fail(LBM_EINVAL, "parameters not set");
    if (nsteps < 0) return fail(LBM_EINVAL, "negative step count");
    int64_t k = 0;
    lbm_status st;
    if (d->launch.stepping == LBM_STEP_FLOW && d->flow_grid > 0 && nsteps >= 1 && d->ntiles > 0) {
        // one dataflow launch per chunk of at most INT32_MAX / ntiles steps
        const int64_t chunk = std::max<int64_t>(1, (int64_t)INT32_MAX / d->ntiles - 1);
        while (k < nsteps) {
            const int n = (int)std::min<int64_t>(nsteps - k, chunk);
            FlowArgs fa{d->d_items, d->d_nbr, d->d_flags, d->ntiles, d->per_sweep, d->sweep_k, n,
                        (int)(d->step & 1), d->stall_tile};
            CK(launch_flow(d->prec, d->d_desc, fa, shape_of(d->launch, d->split), d->sweep_k > 1,
                           d->flow_grid, d->stream));
            d->step += n;
            k += n;
        }
        return LBM_OK;
    }
    if (nsteps >= GRAPH_STEPS + 1 && d->ntiles > 0) {
        if (d->step & 1) {
            if ((st = step_once(d, 0)) != LBM_OK) return st;
            ++k;
        }
        if ((st = ensure_graph(d)) != LBM_OK) return st;
        while (nsteps - k >= GRAPH_STEPS) {
            CK(cudaGraphLaunch(d->graph, d->stream));
            d->step += GRAPH_STEPS;
            k += GRAPH_STEPS;
        }
    }
    for (; k < nsteps; ++k)
        if ((st = step_once(d, 0)) != LBM_OK) return st;
    return LBM_OK;
}

static lbm_status check_step_status() {
    int st = 0;
    CK(take_step_status(&st));
    if (st != 0) return fail(LBM_ECUDA, "a staged population copy did not complete; results are invalid");
    return LBM_OK;
}

// Folds the observing step's partials and reads them back together with the
// dataflow status word: one host synchronisation per observation.  The staged
// kernels' status word is read only when this domain's shape may run them
// (one launch per step, one row of threads per block, FP32 arithmetic).
static lbm_status fetch_obs(lbm_domain* d, double* o) {
    CK(launch_finalize(d->d_desc, 1, d->stream));
    CK(cudaMemcpyAsync(o, d->d_obs, NOBS * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
    int fst = 0;
    CK(cudaMemcpyAsync(&fst, d->d_flags, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    if (d->prec != LBM_F64 && d->launch.block_rows == 1 && d->launch.stepping == LBM_STEP_PER_LAUNCH) {
        const lbm_status st = check_step_status();
        if (st != LBM_OK) return st;
    }
    if (fst == 0) return LBM_OK;
    CK(cudaMemsetAsync(d->d_flags, 0, sizeof(int), d->stream));
    return fail(LBM_ECUDA, "a dataflow step waited too long for its neighbourhood; results are invalid");
}

// o: the kernels' observables, relative to the pressure reference p_ref in
// effect when they were taken (the IOP and the mass carry it)
static void fill_obs(const lbm_domain* d, const double* o, int64_t step, lbm_observables* out,
                     double p_ref) {
    const lbm_params& p = d->params;
    const double scale = p.dt_s > 0.0 ? p.rho0 * (p.dx_m / p.dt_s) * (p.dx_m / p.dt_s) : 0.0;
    std::memset(out, 0, sizeof(*out));
    out->step = step;
    out->iop = o[O_IOP] + p_ref;
    out->iop_pa = p.p_sc_pa + scale * (out->iop - p.p_out);
    out->q_in = o[O_Q_IN];
    out->q_out = o[O_Q_OUT];
    // sum_{i>=1} kappa_i = 4 sigma per active cell
    out->mass = o[O_MASS] + 4.0 * K_SIGMA * p_ref * (double)d->info.n_active;
    out->peak_speed = o[O_PEAK];
    out->wss_cornea = o[O_WSS_C];
    out->wss_iris = o[O_WSS_I];
    out->wss_cornea_pa = scale * o[O_WSS_C];
    out->wss_iris_pa = scale * o[O_WSS_I];
    out->residual = o[O_RESID];
    out->n_fluid = (int64_t)o[O_N_FLUID];
    out->n_cornea = (int64_t)o[O_N_C];
    out->n_iris = (int64_t)o[O_N_I];
    out->nan_flag = o[O_NAN] != 0.0;
    out->u_seep = d->h.tm_model == 1 ? d->h.pd.u_seep : 0.0;
}

// Lumped TM (Sec. 2.3): Darcy's law across the meshwork gives the seepage
// speed for the observed IOP, u_s = K (iop - p_out) / (nu h_tm) (kinematic
// pressure, nu from Eq. 10); it applies from the next step on.
static void update_seepage(lbm_domain* d, double iop) {
    d->last_iop = iop;
    if (d->h.tm_model != 1) return;
    const lbm_params& p = d->params;
    const double nu = (2.0 * p.tau - 1.0) / 6.0;
    d->u_seep = p.K_tm * (iop - p.p_out) / (nu * p.h_tm);
    d->h.pd.u_seep = d->u_seep;
    d->h.pf.u_seep = (float)d->u_seep;
}

extern "C" lbm_status lbm_read_observables(lbm_domain* d, lbm_observables* out) {
    if (!d || !out) return fail(LBM_EINVAL, "null argument");
    if (!d->have_params) return fail(LBM_EINVAL, "parameters not set");
    const int mode = OBS_STATS | (d->h.snap_valid ? OBS_RESID : 0);
    lbm_status st = step_once(d, mode);
    if (st != LBM_OK) return st;
    double o[NOBS];
    if ((st = fetch_obs(d, o)) != LBM_OK) return st;
    fill_obs(d, o, d->step, out, d->p_ref);
    return LBM_OK;
}

// One check interval of the steady-state loop, enqueued: check_every - 1 plain
// steps, the observing step, the fold of its partials and the read-back of
// the observables and the dataflow status word into pinned slot `slot`.
static constexpr int PIN_SLOT = NOBS + 1;  // doubles per slot (last: status word)

// Re-centring of the pressure reference (FP32 and 16-bit storages): after a
// steady-state check whose IOP lies more than PREF_TOL of it away from p_ref,
// the stored populations move to p_ref = IOP.  One pass over them, enqueued
// after whatever is already queued on the domain's stream (d->step, and so
// the parity, already counts that work).  While the IOP still rises it moves
// at most once every PREF_EVERY checks, so the pass costs at most one step in
// PREF_EVERY intervals.
static constexpr double PREF_TOL = 0.01;
static constexpr int PREF_EVERY = 20;
static lbm_status maybe_recenter(lbm_domain* d, double iop) {
    if (d->prec == LBM_F64 || !std::isfinite(iop)) return LBM_OK;
    if (d->checks_since_recenter >= 0 && ++d->checks_since_recenter < PREF_EVERY) return LBM_OK;
    if (std::fabs(iop - d->p_ref) <= PREF_TOL * std::fabs(iop)) return LBM_OK;
    d->checks_since_recenter = 0;
    DISPATCH(d->prec, shift_pressure_kernel, d->d_desc, (int)(d->step & 1), iop - d->p_ref);
    CK(cudaGetLastError());
    d->p_ref = iop;
    d->h.pd.p_out = d->params.p_out - d->p_ref;
    d->h.pf.p_out = (float)d->h.pd.p_out;
    return upload_desc(d);
}

static lbm_status enqueue_interval(lbm_domain* d, int32_t check_every, int slot) {
    lbm_status st;
    if ((st = lbm_step(d, check_every - 1)) != LBM_OK) return st;
    const bool had_snap = d->h.snap_valid != 0;
    if ((st = step_once(d, OBS_STATS | OBS_SNAP | OBS_WRITE | (had_snap ? OBS_RESID : 0))) != LBM_OK)
        return st;
    CK(launch_finalize(d->d_desc, 1, d->stream));
    double* o = d->pin + slot * PIN_SLOT;
    CK(cudaMemcpyAsync(o, d->d_obs, NOBS * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaMemcpyAsync(reinterpret_cast<int*>(o + NOBS), d->d_flags, sizeof(int),
                       cudaMemcpyDeviceToHost, d->stream));
    CK(cudaEventRecord(d->pin_ev[slot], d->stream));
    d->pin_pref[slot] = d->p_ref;
    if (!had_snap) {  // a snapshot exists from this observing step on
        d->h.snap_valid = 1;
        if ((st = upload_desc(d)) != LBM_OK) return st;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_run_to_steady(lbm_domain* d, double tol, int32_t check_every,
                                        int64_t max_steps, int64_t* steps_out) {
    if (!d) return fail(LBM_EINVAL, "null domain");
    if (!d->have_params) return fail(LBM_EINVAL, "parameters not set");
    if (check_every < 1 || max_steps < 0 || !(tol >= 0.0)) return fail(LBM_EINVAL, "bad steady-state arguments");
    if (!d->pin) {
        CK(cudaHostAlloc(reinterpret_cast<void**>(&d->pin), 2 * PIN_SLOT * sizeof(double),
                         cudaHostAllocDefault));
        for (cudaEvent_t& e : d->pin_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // The lumped meshwork feeds each check's IOP into the next interval, so it
    // runs one interval at a time; otherwise the next interval is queued
    // before the host reads a check, and the loop may stop one interval after
    // the check that met the criterion (*steps_out counts it).
    const bool ahead = d->h.tm_model != 1;
    const int64_t s0 = d->step;  // interval k observes the state after s0 + k check_every - 1 steps
    int64_t taken = 0, queued = 0;
    int slot = 0;
    lbm_status st = LBM_OK;
    if (steps_out) *steps_out = 0;
    auto drain = [&]() { cudaStreamSynchronize(d->stream); };
    if (max_steps > 0) {
        const bool had = d->h.snap_valid != 0;
        if ((st = enqueue_interval(d, check_every, slot)) != LBM_OK) return st;
        queued += check_every;
        bool had_snap[2] = {had, true};
        while (taken < max_steps) {
            const int next = slot ^ 1;
            const bool more = queued < max_steps;
            if (ahead && more) {
                had_snap[next] = d->h.snap_valid != 0;
                if ((st = enqueue_interval(d, check_every, next)) != LBM_OK) { drain(); return st; }
                queued += check_every;
            }
            CK(cudaEventSynchronize(d->pin_ev[slot]));
            const double* o = d->pin + slot * PIN_SLOT;
            const int fst = *reinterpret_cast<const int*>(o + NOBS);
            taken += check_every;
            if (steps_out) *steps_out = queued;
            if (d->prec != LBM_F64 && d->launch.block_rows == 1 &&
                d->launch.stepping == LBM_STEP_PER_LAUNCH && (st = check_step_status()) != LBM_OK) {
                drain();
                return st;
            }
            if (fst != 0) {
                drain();
                CK(cudaMemsetAsync(d->d_flags, 0, sizeof(int), d->stream));
                return fail(LBM_ECUDA, "a dataflow step waited too long for its neighbourhood; results are invalid");
            }
            if (o[O_NAN] != 0.0) {
                drain();
                return fail(LBM_EUNSTABLE, "NaN in the pressure field after %lld steps", (long long)taken);
            }
            fill_obs(d, o, s0 + taken - 1, &d->last_obs, d->pin_pref[slot]);
            d->have_last_obs = true;
            update_seepage(d, d->last_obs.iop);
            if (d->h.tm_model == 1) {
                if ((st = upload_desc(d)) != LBM_OK) return st;
            }
            if (had_snap[slot] && o[O_RESID] < tol) {
                drain();
                if (queued > taken) {  // the interval queued ahead has run too: take its check
                    const double* t = d->pin + next * PIN_SLOT;
                    if (*reinterpret_cast<const int*>(t + NOBS) != 0) {
                        CK(cudaMemsetAsync(d->d_flags, 0, sizeof(int), d->stream));
                        return fail(LBM_ECUDA, "a dataflow step waited too long for its neighbourhood; results are invalid");
                    }
                    if (t[O_NAN] != 0.0)
                        return fail(LBM_EUNSTABLE, "NaN in the pressure field after %lld steps", (long long)queued);
                    fill_obs(d, t, s0 + queued - 1, &d->last_obs, d->pin_pref[next]);
                    update_seepage(d, d->last_obs.iop);
                }
                return LBM_OK;
            }
            if ((st = maybe_recenter(d, d->last_obs.iop)) != LBM_OK) { drain(); return st; }
            if (!ahead && more) {
                had_snap[next] = d->h.snap_valid != 0;
                if ((st = enqueue_interval(d, check_every, next)) != LBM_OK) return st;
                queued += check_every;
            }
            slot = next;
            if (taken >= queued) break;
        }
    }
    drain();
    return fail(LBM_ENOTCONVERGED, "not steady after %lld steps", (long long)queued);
}

// ---------------------------------------------------------------------------
// read-back, write-back, checkpoints

extern "C" lbm_status lbm_read_field(lbm_domain* d, double* u, double* p, double* T) {
    if (!d) return fail(LBM_EINVAL, "null domain");
    DISPATCH(d->prec, fields_kernel, d->d_desc, (int)(d->step & 1), d->p_ref, u, p, T);
    CK(cudaGetLastError());
    return LBM_OK;
}

extern "C" lbm_status lbm_read_populations(lbm_domain* d, double* f, double* g) {
    if (!d) return fail(LBM_EINVAL, "null domain");
    DISPATCH(d->prec, read_pops_kernel, d->d_desc, (int)(d->step & 1), d->p_ref, f, g);
    CK(cudaGetLastError());
    return LBM_OK;
}

extern "C" lbm_status lbm_write_populations(lbm_domain* d, const double* f, const double* g) {
    if (!d) return fail(LBM_EINVAL, "null domain");
    if (!d->have_params) return fail(LBM_EINVAL, "parameters not set");
    DISPATCH(d->prec, write_pops_kernel, d->d_desc, (int)(d->step & 1), d->p_ref, f, g);
    CK(cudaGetLastError());
    return LBM_OK;
}

namespace {
struct StateHeader {
    char magic[8];
    int32_t nx, ny, prec, snap_valid;
    int64_t step, npad;
    double Tshift;
    double u_seep;
    lbm_params params;
    double Tstep;  // 16-bit storages: step of the heat codes
    double p_ref;  // pressure reference of the stored flow populations
};
}  // namespace

extern "C" size_t lbm_state_bytes(const lbm_domain* d) {
    if (!d) return 0;
    return sizeof(StateHeader) + 13 * (size_t)d->L.npad * store_size(d->prec);
}

extern "C" lbm_status lbm_save_state(lbm_domain* d, void* host_buf, size_t bytes) {
    if (!d || !host_buf) return fail(LBM_EINVAL, "null argument");
    if (!d->have_params) return fail(LBM_EINVAL, "parameters not set");
    if (bytes < lbm_state_bytes(d)) return fail(LBM_ENOMEM, "state buffer too small");
    StateHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "LBMSTAT2", 8);
    hd.nx = d->nx;
    hd.ny = d->ny;
    hd.prec = d->prec;
    hd.snap_valid = 0;
    hd.step = d->step;
    hd.npad = d->L.npad;
    hd.Tshift = d->h.Tshift;
    hd.Tstep = d->h.Tstep;
    hd.p_ref = d->p_ref;
    hd.u_seep = d->u_seep;
    hd.params = d->params;
    std::memcpy(host_buf, &hd, sizeof(hd));
    CK(cudaMemcpyAsync(static_cast<char*>(host_buf) + sizeof(hd), d->h.pops,
                       13 * (size_t)d->L.npad * store_size(d->prec), cudaMemcpyDeviceToHost, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_load_state(lbm_domain* d, const void* host_buf, size_t bytes) {
    if (!d || !host_buf) return fail(LBM_EINVAL, "null argument");
    if (bytes < lbm_state_bytes(d)) return fail(LBM_ENOMEM, "state buffer too small");
    StateHeader hd;
    std::memcpy(&hd, host_buf, sizeof(hd));
    if (std::memcmp(hd.magic, "LBMSTAT2", 8) != 0 || hd.nx != d->nx || hd.ny != d->ny ||
        hd.prec != d->prec || hd.npad != d->L.npad)
        return fail(LBM_EINVAL, "checkpoint does not match this domain");
    d->u_seep = hd.u_seep;
    d->p_ref = hd.p_ref;  // before apply_params, which sets the kernels' outlet pressure from it
    lbm_status st = apply_params(d, &hd.params);  // no reset: populations come from the buffer
    if (st != LBM_OK) return st;
    d->have_params = true;
    d->h.Tshift = (float)hd.Tshift;
    d->h.Tstep = (float)hd.Tstep;
    d->h.Tscale = hd.Tstep > 0.0 ? (float)(1.0 / hd.Tstep) : 0.0f;
    sync_heat_reference(d);
    d->h.snap_valid = 0;
    d->step = hd.step;
    if ((st = upload_desc(d)) != LBM_OK) return st;
    CK(cudaMemcpyAsync(d->h.pops, static_cast<const char*>(host_buf) + sizeof(hd),
                       13 * (size_t)d->L.npad * store_size(d->prec), cudaMemcpyHostToDevice, d->stream));
    CK(cudaStreamSynchronize(d->stream));
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// launch shape and introspection

extern "C" lbm_status lbm_set_launch(lbm_domain* d, const lbm_launch* l) {
    if (!d || !l) return fail(LBM_EINVAL, "null argument");
    if (!launch_ok(*l, d->prec)) return fail(LBM_EINVAL, "invalid launch shape");
    CK(cudaStreamSynchronize(d->stream));
    drop_graph(d);
    d->launch = *l;
    lbm_status st = build_tiles(d);
    if (st != LBM_OK) return st;
    return upload_desc(d);
}

extern "C" lbm_status lbm_get_launch(const lbm_domain* d, lbm_launch* l) {
    if (!d || !l) return fail(LBM_EINVAL, "null argument");
    *l = d->launch;
    return LBM_OK;
}

extern "C" int64_t lbm_get_step(const lbm_domain* d) { return d ? d->step : -1; }

extern "C" lbm_status lbm_debug_stall_tile(lbm_domain* d, int32_t tile) {
    if (!d) return fail(LBM_EINVAL, "null domain");
    if (tile < -1 || tile >= d->ntiles) return fail(LBM_EINVAL, "tile %d out of range", tile);
    d->stall_tile = tile;
    return LBM_OK;
}

extern "C" lbm_status lbm_get_info(const lbm_domain* d, lbm_geometry_info* info) {
    if (!d || !info) return fail(LBM_EINVAL, "null argument");
    *info = d->info;
    return LBM_OK;
}

extern "C" int64_t lbm_get_tile_count(const lbm_domain* d) { return d ? d->ntiles : -1; }

extern "C" int64_t lbm_get_edge_cell_count(const lbm_domain* d) { return d ? d->n_edges : -1; }

extern "C" double lbm_step_bytes(const lbm_domain* d) {
    if (!d) return 0.0;
    return (double)d->info.n_active * (26.0 * (double)store_size(d->prec) + 1.0);
}

// ---------------------------------------------------------------------------
// internal accessors for the allocation-free observables entry point
namespace lbm {
lbm_status set_error(lbm_status s, const char* msg) { return fail(s, "%s", msg); }

bool domain_parts(const lbm_domain* d, const InstDesc** desc, int* precision, int* ny,
                  int* parity, int* snap_valid, cudaStream_t* stream, int* device) {
    if (!d) { fail(LBM_EINVAL, "null domain"); return false; }
    if (!d->have_params) { fail(LBM_EINVAL, "parameters not set"); return false; }
    *device = d->device;
    *desc = d->d_desc;
    *precision = d->prec;
    *ny = d->ny;
    *parity = (int)(d->step & 1);
    *snap_valid = d->h.snap_valid;
    *stream = d->stream;
    return true;
}

bool domain_vortex_parts(const lbm_domain* d, const uint8_t** mask, int* nx, int* ny,
                         int* periodic_x, int* periodic_y, double** scratch,
                         int64_t* scratch_doubles, double* dx_m, double* dt_s,
                         cudaStream_t* stream) {
    if (!d) { fail(LBM_EINVAL, "null domain"); return false; }
    *mask = d->h.mask;
    *nx = d->nx;
    *ny = d->ny;
    *periodic_x = d->periodic_x;
    *periodic_y = d->periodic_y;
    *scratch = d->h.partials;
    *scratch_doubles = d->L.max_tiles * NPART;
    *dx_m = d->have_params ? d->params.dx_m : 0.0;
    *dt_s = d->have_params ? d->params.dt_s : 0.0;
    *stream = d->stream;
    return true;
}

void fill_observables(const lbm_domain* d, const double* o, lbm_observables* out) {
    fill_obs(d, o, d->step, out, d->p_ref);
}
}  // namespace lbm

// ---------------------------------------------------------------------------
// batches: many domains advanced by one launch per step over a merged tile list

static constexpr int BATCH_GRAPH_STEPS = 32;

struct lbm_batch {
    int prec = 0;
    int max_inst = 0;
    int64_t max_tiles = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 1;
    char* base = nullptr;
    InstDesc* d_table = nullptr;
    double* d_obs = nullptr;
    int4* d_tiles = nullptr;
    int* d_nbr = nullptr;              // dataflow: 8 neighbour tiles per tile (batch indices)
    int* d_flags = nullptr;            // dataflow: status, abort and progress words
    int4* d_items = nullptr;           // dataflow: one item per tile, step by step
    bool coop = false;
    int flow_grid = 0;
    std::vector<lbm_domain*> members;  // table order
    std::vector<InstDesc> htable;
    std::vector<double> hobs;
    lbm_launch launch{128, 1, 2, 0, LBM_STEP_PER_LAUNCH, 1, 0};
    int ntiles = 0;
    int nchunks = 0;  // edge-cell chunks in d_tiles' second part
    int split = 0;    // plain steps take the edge-cell chunks (Shape::split)
    bool dirty = true;
    // per-step launches take the tiles holding boundary cells (the slower
    // general update) first, then the pure tiles; the autotuner tries both
    bool boundary_first = false;
    cudaGraphExec_t graph = nullptr;
};

struct BatchLayout {
    size_t table, obs, tiles, nbr, flags, items, total;
};

static BatchLayout batch_layout(int max_inst, int64_t max_tiles) {
    BatchLayout L;
    size_t off = 0;
    L.table = off; off = align_up(off + (size_t)max_inst * sizeof(InstDesc));
    L.obs = off; off = align_up(off + (size_t)max_inst * NOBS * sizeof(double));
    // per-step list: the tiles, then the tiles with up to as many edge-cell
    // chunks spread among them
    L.tiles = off; off = align_up(off + (size_t)3 * max_tiles * sizeof(int4));
    L.nbr = off; off = align_up(off + (size_t)max_tiles * 8 * sizeof(int));
    L.flags = off; off = align_up(off + (size_t)(max_tiles + 2) * sizeof(int));
    L.items = off; off = align_up(off + (size_t)max_tiles * sizeof(int4));
    L.total = off;
    return L;
}

extern "C" size_t lbm_batch_bytes(int32_t max_instances, int64_t max_tiles) {
    if (max_instances <= 0 || max_tiles <= 0 || max_tiles > INT32_MAX) return 0;
    return batch_layout(max_instances, max_tiles).total;
}

extern "C" lbm_status lbm_batch_create(int32_t precision, int32_t max_instances, int64_t max_tiles,
                                       const lbm_launch* launch, void* dev_buf, size_t bytes,
                                       void* stream, lbm_batch** out) {
    if (!out) return fail(LBM_EINVAL, "null argument");
    *out = nullptr;
    if (!store_size(precision)) return fail(LBM_EINVAL, "unknown precision %d", precision);
    if (max_instances <= 0 || max_tiles <= 0 || max_tiles > INT32_MAX)
        return fail(LBM_EINVAL, "bad batch capacity");
    if (launch && !launch_ok(*launch, precision)) return fail(LBM_EINVAL, "invalid launch shape");
    const BatchLayout L = batch_layout(max_instances, max_tiles);
    if (!dev_buf || bytes < L.total || (reinterpret_cast<uintptr_t>(dev_buf) % ALIGN) != 0)
        return fail(LBM_ENOMEM, "batch buffer too small or not 256-byte aligned (need %zu bytes)", L.total);
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return fail(LBM_ENOMEM, "host allocation failed");
    b->prec = precision;
    b->max_inst = max_instances;
    b->max_tiles = max_tiles;
    b->stream = static_cast<cudaStream_t>(stream);
    b->base = static_cast<char*>(dev_buf);
    b->d_table = reinterpret_cast<InstDesc*>(b->base + L.table);
    b->d_obs = reinterpret_cast<double*>(b->base + L.obs);
    b->d_tiles = reinterpret_cast<int4*>(b->base + L.tiles);
    b->d_nbr = reinterpret_cast<int*>(b->base + L.nbr);
    b->d_flags = reinterpret_cast<int*>(b->base + L.flags);
    b->d_items = reinterpret_cast<int4*>(b->base + L.items);
    if (launch) b->launch = *launch;
    int dev = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flags, 0, sizeof(int), b->stream);
    b->coop = coop != 0;
    if (e != cudaSuccess) {
        delete b;
        return fail(LBM_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    *out = b;
    return LBM_OK;
}

static void batch_drop_graph(lbm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

extern "C" lbm_status lbm_batch_add(lbm_batch* b, lbm_domain* d) {
    if (!b || !d) return fail(LBM_EINVAL, "null argument");
    if (d->batch) return fail(LBM_EBUSY, "domain already belongs to a batch");
    if (d->prec != b->prec) return fail(LBM_EINVAL, "domain precision differs from the batch's");
    if (!d->have_params) return fail(LBM_EINVAL, "set the domain's parameters before adding it");
    if ((int)b->members.size() >= b->max_inst) return fail(LBM_EBUSY, "batch is full");
    lbm_status st;
    if (std::memcmp(&d->launch, &b->launch, sizeof(lbm_launch)) != 0 &&
        (st = lbm_set_launch(d, &b->launch)) != LBM_OK)
        return st;
    int64_t total = d->ntiles;
    for (lbm_domain* m : b->members) total += m->ntiles;
    if (total > b->max_tiles) return fail(LBM_EBUSY, "batch tile capacity exceeded (%lld tiles)", (long long)total);
    CK(cudaStreamSynchronize(d->stream));  // order the domain's earlier work before the batch's
    d->own_stream = d->stream;
    d->stream = b->stream;
    d->batch = b;
    b->members.push_back(d);
    b->dirty = true;
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_remove(lbm_batch* b, lbm_domain* d) {
    if (!b || !d) return fail(LBM_EINVAL, "null argument");
    auto it = std::find(b->members.begin(), b->members.end(), d);
    if (it == b->members.end()) return fail(LBM_EINVAL, "domain is not a member of this batch");
    CK(cudaStreamSynchronize(b->stream));
    b->members.erase(it);
    d->stream = d->own_stream;
    d->batch = nullptr;
    b->dirty = true;
    return LBM_OK;
}

extern "C" int32_t lbm_batch_size(const lbm_batch* b) { return b ? (int32_t)b->members.size() : -1; }

// merged tile list: member k's local tile t becomes (k, t, x0, y0); for
// dataflow steps, the members' neighbour lists shifted to batch indices and
// one work item per tile (batch index | TILE_PURE)
static lbm_status batch_rebuild(lbm_batch* b) {
    if (!b->dirty) return LBM_OK;
    std::vector<int4> tiles, items, chunks;
    std::vector<int> nbr;
    for (size_t k = 0; k < b->members.size(); ++k) {
        const lbm_domain* m = b->members[k];
        for (const int4& c : m->hchunks) chunks.push_back(make_int4((int)k, c.y, c.z, c.w));
        const int base = (int)tiles.size();
        for (size_t j = 0; j < m->htiles.size(); ++j) {
            const int4& t = m->htiles[j];
            const int g = base + (int)j;
            tiles.push_back(make_int4((int)k, t.y, t.z, t.w));
            items.push_back(make_int4((int)k, g | (t.y & TILE_PURE), t.z, t.w));
            for (int i = 0; i < 8; ++i) {
                const int u = m->hnbr[j * 8 + i];
                nbr.push_back(u < 0 ? -1 : base + u);
            }
        }
    }
    if ((int64_t)tiles.size() > b->max_tiles) return fail(LBM_EBUSY, "batch tile capacity exceeded");
    if (b->boundary_first) {  // per-step order only: the dataflow items keep their wavefront order
        std::stable_partition(tiles.begin(), tiles.end(), [](const int4& t) { return !(t.y & TILE_PURE); });
    }
    // the split kernels when any member takes edge-cell chunks (each member
    // keeps its own choice, so it computes the same alone and in the batch)
    b->split = 0;
    for (const lbm_domain* m : b->members) b->split |= m->split;
    if ((int64_t)chunks.size() > b->max_tiles)
        return fail(LBM_EBUSY, "batch tile capacity exceeded (edge-cell chunks)");
    // per-step list: the tiles, then the tiles with the members' edge-cell
    // chunks spread among them
    std::vector<int4> order = tiles;
    append_interleaved(order, tiles, chunks);
    if (!tiles.empty()) {
        CK(cudaMemcpyAsync(b->d_tiles, order.data(), order.size() * sizeof(int4), cudaMemcpyHostToDevice,
                           b->stream));
        CK(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, b->stream));
        CK(cudaMemcpyAsync(b->d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice,
                           b->stream));
    }
    b->flow_grid = 0;
    if (b->coop) {
        const StepPlan pl = flow_plan(b->prec, shape_of(b->launch, b->split), false);
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl.func,
                                                         (int)(pl.block.x * pl.block.y), pl.smem));
        if (b->launch.blocks_per_sm > 0) per_sm = std::min(per_sm, b->launch.blocks_per_sm);
        b->flow_grid = per_sm * b->num_sms;
    }
    CK(cudaStreamSynchronize(b->stream));
    b->ntiles = (int)tiles.size();
    b->nchunks = (int)chunks.size();

    batch_drop_graph(b);
    b->dirty = false;
    return LBM_OK;
}

// table entry k = member k's descriptor with its current step parity and a
// slot of the batch's contiguous observables array
static lbm_status batch_upload_table(lbm_batch* b) {
    b->htable.resize(b->members.size());
    int32_t base = 0;  // the member's first tile in the merged list (batch_rebuild's order)
    for (size_t k = 0; k < b->members.size(); ++k) {
        InstDesc t = b->members[k]->h;
        derive_code_units(t);
        t.tile_base = base;
        base += b->members[k]->ntiles;
        t.parity = (int)(b->members[k]->step & 1);
        t.obs = b->d_obs + k * NOBS;
        b->htable[k] = t;
    }
    if (!b->htable.empty())
        CK(cudaMemcpyAsync(b->d_table, b->htable.data(), b->htable.size() * sizeof(InstDesc),
                           cudaMemcpyHostToDevice, b->stream));
    return LBM_OK;
}

static int batch_cap(const lbm_batch* b) {
    return b->launch.blocks_per_sm > 0 ? b->launch.blocks_per_sm * b->num_sms : 0;
}

static lbm_status batch_ensure_graph(lbm_batch* b) {
    if (b->graph) return LBM_OK;
    const cudaError_t e = step_graph(b->prec, b->d_table, b->d_tiles, b->nchunks, b->ntiles, shape_of(b->launch, b->split),
                                     batch_cap(b), BATCH_GRAPH_STEPS, &b->graph);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return fail(LBM_ECUDA, "batch graph construction failed: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps) {
    if (!b) return fail(LBM_EINVAL, "null batch");
    if (nsteps < 0) return fail(LBM_EINVAL, "negative step count");
    if (b->members.empty() || nsteps == 0) return LBM_OK;
    lbm_status st;
    if ((st = batch_rebuild(b)) != LBM_OK || (st = batch_upload_table(b)) != LBM_OK) return st;
    int64_t k = 0;
    if (b->launch.stepping == LBM_STEP_FLOW && b->flow_grid > 0 && b->ntiles > 0) {
        // dataflow launches, step by step (each member's own parity is in its
        // table entry)
        const int64_t chunk = (int64_t)INT32_MAX / 8 - 1;
        while (k < nsteps) {
            const int n = (int)std::min<int64_t>(nsteps - k, chunk);
            FlowArgs fa{b->d_items, b->d_nbr, b->d_flags, b->ntiles, b->ntiles, 1, n, 0, -1};
            CK(launch_flow(b->prec, b->d_table, fa, shape_of(b->launch, b->split), false, b->flow_grid,
                           b->stream));
            k += n;
        }
    }
    if (nsteps - k >= BATCH_GRAPH_STEPS && b->ntiles > 0) {
        if ((st = batch_ensure_graph(b)) != LBM_OK) return st;
        for (; nsteps - k >= BATCH_GRAPH_STEPS; k += BATCH_GRAPH_STEPS)
            CK(cudaGraphLaunch(b->graph, b->stream));
    }
    for (; k < nsteps; ++k)
        CK(launch_step(b->prec, b->d_table, b->d_tiles, b->nchunks, b->ntiles, (int)(k & 1), 0,
                       shape_of(b->launch, b->split), batch_cap(b), b->stream));
    for (lbm_domain* m : b->members) m->step += nsteps;
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_check(lbm_batch* b, int32_t check_every) {
    if (!b) return fail(LBM_EINVAL, "null batch");
    if (check_every < 1) return fail(LBM_EINVAL, "check_every must be >= 1");
    if (b->members.empty()) return LBM_OK;
    lbm_status st;
    if ((st = lbm_batch_step(b, check_every - 1)) != LBM_OK) return st;
    if ((st = batch_rebuild(b)) != LBM_OK || (st = batch_upload_table(b)) != LBM_OK) return st;
    CK(launch_step(b->prec, b->d_table, b->d_tiles, b->nchunks, b->ntiles, 0,
                   OBS_STATS | OBS_SNAP | OBS_WRITE | OBS_RESID, shape_of(b->launch, b->split), batch_cap(b),
                   b->stream));
    for (lbm_domain* m : b->members) m->step += 1;
    const int n = (int)b->members.size();
    CK(launch_finalize(b->d_table, n, b->stream));
    b->hobs.resize((size_t)n * NOBS);
    CK(cudaMemcpyAsync(b->hobs.data(), b->d_obs, b->hobs.size() * sizeof(double), cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if ((st = check_step_status()) != LBM_OK) return st;
    {
        int fs = 0;
        CK(cudaMemcpyAsync(&fs, b->d_flags, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        if (fs != 0) {
            CK(cudaMemsetAsync(b->d_flags, 0, sizeof(int), b->stream));
            return fail(LBM_ECUDA, "a dataflow step waited too long for its neighbourhood; results are invalid");
        }
    }
    for (int k = 0; k < n; ++k) {
        lbm_domain* m = b->members[k];
        // the observing step ran at step - 1 (pre-collision state of that step)
        fill_obs(m, b->hobs.data() + (size_t)k * NOBS, m->step - 1, &m->last_obs, m->p_ref);
        m->have_last_obs = true;
        update_seepage(m, m->last_obs.iop);
        if (!m->h.snap_valid || m->h.tm_model == 1) {
            m->h.snap_valid = 1;
            if ((st = upload_desc(m)) != LBM_OK) return st;
        }
        if ((st = maybe_recenter(m, m->last_obs.iop)) != LBM_OK) return st;
    }
    // the members' descriptors may have changed (snapshot, seepage, p_ref)
    return batch_upload_table(b);
}

extern "C" lbm_status lbm_last_observables(const lbm_domain* d, lbm_observables* out) {
    if (!d || !out) return fail(LBM_EINVAL, "null argument");
    if (!d->have_last_obs) return fail(LBM_EINVAL, "no steady-state check has observed this domain yet");
    *out = d->last_obs;
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_get_launch(const lbm_batch* b, lbm_launch* l) {
    if (!b || !l) return fail(LBM_EINVAL, "null argument");
    *l = b->launch;
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_set_launch(lbm_batch* b, const lbm_launch* l) {
    if (!b || !l) return fail(LBM_EINVAL, "null argument");
    if (!launch_ok(*l, b->prec)) return fail(LBM_EINVAL, "invalid launch shape");
    int64_t total = 0;
    for (lbm_domain* m : b->members) {
        lbm_status st = lbm_set_launch(m, l);
        if (st != LBM_OK) return st;
        total += m->ntiles;
    }
    if (total > b->max_tiles) return fail(LBM_EBUSY, "batch tile capacity exceeded for this shape");
    b->launch = *l;
    b->dirty = true;
    return LBM_OK;
}

extern "C" double lbm_batch_step_bytes(const lbm_batch* b) {
    if (!b) return 0.0;
    double s = 0.0;
    for (const lbm_domain* m : b->members) s += lbm_step_bytes(m);
    return s;
}

extern "C" int64_t lbm_batch_active_cells(const lbm_batch* b) {
    if (!b) return -1;
    int64_t s = 0;
    for (const lbm_domain* m : b->members) s += m->info.n_active;
    return s;
}

// Autotuner: time each candidate shape on the current members (the timed
// steps are real steps of the members) and keep the fastest.
extern "C" lbm_status lbm_batch_tune(lbm_batch* b, int32_t steps_per_candidate, lbm_launch* chosen) {
    if (!b) return fail(LBM_EINVAL, "null batch");
    if (steps_per_candidate < 2) return fail(LBM_EINVAL, "steps_per_candidate must be >= 2");
    if (b->members.empty()) return fail(LBM_EINVAL, "empty batch");
    // one launch per step on most shapes, dataflow stepping on the ones that suit it
    // (sweep_steps 0, sweep_lag 0: one step per sweep, the default lag)
    static const lbm_launch cand[] = {
        {128, 2, 2, 0, LBM_STEP_PER_LAUNCH, 0, 0}, {64, 2, 2, 0, LBM_STEP_PER_LAUNCH, 0, 0},
        {64, 4, 1, 0, LBM_STEP_PER_LAUNCH, 0, 0},  {64, 4, 2, 0, LBM_STEP_PER_LAUNCH, 0, 0},
        {128, 1, 4, 0, LBM_STEP_PER_LAUNCH, 0, 0}, {128, 1, 8, 0, LBM_STEP_PER_LAUNCH, 0, 0},
        {256, 1, 8, 0, LBM_STEP_PER_LAUNCH, 0, 0}, {64, 4, 2, 0, LBM_STEP_FLOW, 0, 0},
        {64, 4, 3, 0, LBM_STEP_FLOW, 0, 0},        {128, 2, 2, 0, LBM_STEP_FLOW, 0, 0},
        // 16-bit storages only: eight cells per thread on 256-cell rows
        {256, 4, 1, 0, LBM_STEP_PER_LAUNCH, 0, 0}, {256, 4, 2, 0, LBM_STEP_PER_LAUNCH, 0, 0},
        {256, 8, 1, 0, LBM_STEP_PER_LAUNCH, 0, 0}, {256, 4, 2, 0, LBM_STEP_FLOW, 0, 0}};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    lbm_launch best = b->launch;
    bool best_bfirst = b->boundary_first;
    lbm_status st = LBM_OK;
    for (const lbm_launch& c : cand) {
        if (!launch_ok(c, b->prec)) continue;  // a shape of another storage
        // one launch per step: raster order and boundary tiles first
        for (int order = 0; order < (c.stepping == LBM_STEP_PER_LAUNCH ? 2 : 1) && st == LBM_OK; ++order) {
            b->boundary_first = order == 1;
            b->dirty = true;
            if ((st = lbm_batch_set_launch(b, &c)) != LBM_OK) {
                if (st == LBM_EBUSY) st = LBM_OK;  // shape needs more tiles than fit
                break;
            }
            if ((st = lbm_batch_step(b, 2)) != LBM_OK) break;  // warm-up, builds the tile list
            cudaEventRecord(e0, b->stream);
            if ((st = lbm_batch_step(b, steps_per_candidate)) != LBM_OK) break;
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) { best_ms = ms; best = c; best_bfirst = b->boundary_first; }
        }
        if (st != LBM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBM_OK) return st;
    b->boundary_first = best_bfirst;
    b->dirty = true;
    if ((st = lbm_batch_set_launch(b, &best)) != LBM_OK) return st;
    if (chosen) *chosen = best;
    return LBM_OK;
}

extern "C" void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (lbm_domain* m : b->members) {
        m->stream = m->own_stream;
        m->batch = nullptr;
    }
    batch_drop_graph(b);
    delete b;
}
