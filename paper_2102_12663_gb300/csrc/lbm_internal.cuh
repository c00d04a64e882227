// Internal declarations shared by the library's translation units: the
// per-instance descriptor read by the kernels, the mask encoding, the
// storage-precision traits and the launcher entry points.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Mask byte: bits 0-2 cell type (lbm_cell_type), bit 3 set when at least one
// of the eight neighbours is not an active (fluid or porous) cell.
constexpr uint8_t TYPE_BITS = 7;
constexpr uint8_t NEAR_BOUNDARY = 8;
constexpr uint8_t CURVED = 16;  // fluid cell with a link to the curved cornea (q != 1/2)

// Link fractions of one curved cell: q[i-1] for link i, 1/2 where the
// halfway rule applies.  Entries are grouped by column (qcol prefix sums).
struct CurvedCell {
    int32_t y, pad;
    double q[8];
};
enum : int { FLUID = 0, POROUS = 1, COLD = 2, HOT = 3, ADIABATIC = 4, INLET = 5, OUTLET = 6 };

// Observation modes of the fused step (bit set).
enum : int {
    OBS_STATS = 1,  // per-tile partial sums of the observables
    OBS_RESID = 2,  // max |u - u_snapshot|
    OBS_SNAP = 4,   // store u as the new snapshot
    OBS_WRITE = 8   // also perform the step (else observe only)
};

// Per-tile partial slots (FP64).  P_PEAK and P_RESID hold the maxima of the
// squared norms; the fold takes their square roots.
enum : int {
    P_SUM_P = 0, P_N_FLUID, P_MASS, P_Q_IN, P_Q_OUT, P_WSS_C, P_N_C, P_WSS_I, P_N_I,
    P_NAN, P_PEAK, P_RESID, NPART
};
constexpr int NSUM = P_PEAK;  // slots [0, NSUM) add, the rest take the max

// Finalised observables (FP64) as written by the finalize kernel.
enum : int {
    O_IOP = 0, O_Q_IN, O_Q_OUT, O_MASS, O_PEAK, O_WSS_C, O_WSS_I, O_RESID,
    O_N_FLUID, O_N_C, O_N_I, O_NAN, NOBS
};

// Physical parameters in the arithmetic precision of a kernel (derived once on
// the host, so no kernel converts between FP64 and FP32 per cell).
template <class R>
struct Phys {
    R omega, omegaT;      // 1/tau, 1/tau_T
    R g_beta, gx, gy;
    R T_cold, T_hot, T0, T_in;
    R u_in_max;
    R cK, den;            // nu/K and 1 + nu/(2K)
    R p_out;
    R drive_x, drive_y;
    R kwss;               // -(1 - 1/(2 tau))
    R u_seep;             // lumped TM: seepage speed out of the outlets
    // Heat populations are stored (and, with FP32 arithmetic, collided) as
    // deviations T_i - Tref/4 from a reference temperature fixed when the
    // state is initialised (0 for FP64, T0 otherwise); dT0 = T0 - Tref.
    R Tref, dT0;
};

// Everything a kernel needs to update one problem instance.  Lives in device
// memory (one per domain, one table per batch); copied to shared memory by
// every block that works on the instance.
struct InstDesc {
    void* pops;          // 13 planes of npad elements: f_0..f_8, T_1..T_4
    const uint8_t* mask; // npad bytes
    void* usnap;         // 2 planes of npad compute-precision values
    double* partials;    // NPART doubles per tile of this instance
    double* obs;         // NOBS finalised observables
    int64_t npad;
    int32_t ntiles;      // tiles of this instance (partials rows)
    int32_t nx, ny;
    int32_t parity;      // parity of the instance's step counter at launch base
    int32_t snap_valid;
    int32_t inlet_dir_x, inlet_dir_y, inlet_profile, inlet_lo, inlet_width;
    int32_t eye_normals;
    int32_t tm_model;    // 0 porous TM cells, 1 lumped TM (seepage-velocity outlets)
    int32_t outlet_axis; // outlets drain along x (0) or y (1)
    int32_t bouzidi;     // interpolated bounce-back on the curved cornea
    const int32_t* qcol; // nx + 1 prefix sums into qtab (curved cells per column)
    const CurvedCell* qtab;
    double arc_xc, arc_yc;
    Phys<double> pd;
    Phys<float> pf;
    // 16-bit storage of the flow populations: stored = value * fscale.  Tshift
    // = Tref / 4: every storage but FP64 holds T_i - Tshift
    float fscale, finv, Tshift, pad1;
    // bulk tensor copy map of the populations (staged kernel), or null; last,
    // so that adding it moved no field the other kernels read
    const void* tmap;
    // FOLD_MAX x NPART doubles of per-block partials for the observables'
    // fold, then its arrival counter (zero between folds)
    double* fold;
    // 16-bit storages: heat deviations as 16-bit fixed point,
    // code = round(value * Tscale), value = code * Tstep
    float Tstep, Tscale;
    // the same run's constants for the 16-bit vector path, whose collision
    // takes the heat deviations in code units (value * Tscale): g beta Tstep,
    // (T0 - Tref) Tscale and Tref Tscale, and 1 / den of the Darcy drag (set
    // from the fields above whenever the descriptor is uploaded)
    float gbc, dT0c, Trefc, rden;
    // Edge cells of the FP32-arithmetic plain steps (cell indices y nx + x):
    // the active cells that no interior cell pair of the pair or vector path
    // covers, in tile order, those of local tile t at edges[eoff[t] ..
    // eoff[t + 1]).  Per-step launches hand them out in entries of the tile
    // list flagged TILE_EDGE (one cell per thread of a block); the dataflow
    // kernel updates a tile's own after its rows.
    const int32_t* edges;
    // per edge cell: its eight neighbours' cell types, 4 bits each in link
    // order (0 for a cell not next to a boundary), as the per-cell update
    // would read them from the mask
    const uint32_t* etypes;
    const int32_t* eoff;
    // first tile of this instance in a batch's merged tile list (0 for a
    // domain): the dataflow items carry merged indices, eoff local ones
    int32_t tile_base;
    // this instance's plain steps take its edge-cell chunks (FP32: the
    // host's choice for the grid; always for the 16-bit storages); else its
    // rows update every cell and it has no edge cells
    int32_t split;
};
// most blocks that fold one instance's tile partials
constexpr int FOLD_MAX = 32;
static_assert(sizeof(InstDesc) % 8 == 0, "descriptor must be 8-byte sized");

template <class R>
__host__ __device__ __forceinline__ const Phys<R>& phys(const InstDesc& d);
template <>
__host__ __device__ __forceinline__ const Phys<double>& phys<double>(const InstDesc& d) { return d.pd; }
template <>
__host__ __device__ __forceinline__ const Phys<float>& phys<float>(const InstDesc& d) { return d.pf; }

// Tile list entries are int4 {instance, local tile | TILE_PURE, x0, y0}.
// TILE_PURE marks a tile that lies wholly inside the grid and holds only
// fluid cells none of which links to a boundary: the FP32-arithmetic kernels
// update it by the pair path without reading its mask.
constexpr int TILE_PURE = 1 << 30;
// an edge-cell chunk {instance, TILE_EDGE, first, count}: cells edges[first ..
// first + count) of the instance, one per thread, in plain steps of the
// FP32-arithmetic kernels (spread among the tiles in a second part of the
// tile list; the other kernels are launched on the first part, the tiles alone)
constexpr int TILE_EDGE = 1 << 29;
constexpr int TILE_INDEX = TILE_EDGE - 1;

struct Shape {
    int tw, bh, rpt;  // tile = tw x (bh * rpt) cells, block = (tw / V) x bh threads
    // plain FP32-arithmetic steps with edge-cell chunks (the host's choice
    // for the grid: every 16-bit storage, FP32 grids with many cells in row
    // segments next to a boundary); 0: the rows update every cell
    int split = 0;
};

// Cells per thread along x: the FP32-arithmetic kernels take cell pairs
// (vector loads and stores, warp shuffles), the FP64 kernel single cells, and
// the 16-bit storages on 256- or 128-cell tile rows eight or four cells (one
// 16- or 8-byte vector per plane; 32 threads per row).
__host__ __device__ constexpr int vec16_cells(int tile_w) {
    return tile_w == 256 ? 8 : (tile_w == 128 ? 4 : 0);
}
__host__ __device__ constexpr int cells_per_thread(int precision, int tile_w) {
    return precision == 0 ? 1 : ((precision >= 2 && vec16_cells(tile_w) > 0) ? vec16_cells(tile_w) : 2);
}

// ---- storage traits --------------------------------------------------------
// Store cache policy of a storage trait.  ST_STREAM: evict-first streaming
// stores (with one step per pass over the grid, the next step reads the slot
// back from DRAM anyway).  ST_KEEP: ordinary L2 stores (a sweep of several
// steps reads the slot back while it is still in L2).
enum : int { ST_STREAM = 0, ST_KEEP = 1 };
template <int POL, class V>
__device__ __forceinline__ void st_pol(V* p, V v) {
    if constexpr (POL == ST_STREAM) __stcs(p, v);
    else __stcg(p, v);
}

// Heat deviations T_i - Tshift of the 16-bit storages: 16-bit fixed point,
// companded.  The deviations of a run lie in a range known from its boundary
// temperatures: near equilibrium |T_i - T0/4| <= span/4 (span: the largest
// distance of a wall, inflow or reference temperature from T0), and the
// steady state's heat depends on the rounding of these values through the
// slowest diffusive modes, which amplify it by about 1/theta.  So the inner
// three quarters of the codes (|code| <= TFIX_KNEE) carry that range with a
// uniform step, several times finer than FP16's rounding at its ends.  While
// a thermal boundary layer forms, anti-bounce-back at a wall of temperature
// T_w returns deviations up to (T_w - T0)/2 - d*, up to 3/4 of span: the
// outer codes cover them with a step TFIX_COARSE times coarser, out to about
// span.  Codes saturate at the ends of the 16-bit range.
constexpr float TFIX_KNEE = 24576.0f;
constexpr float TFIX_COARSE = 8.0f;
// In code units (value * Tscale): the code of q is q inside the knee and
// knee + (|q| - knee) / 8 outside it, i.e. c = k + (q - k) / 8 with k = q
// clamped to the knee; rounded to the nearest integer, saturated to the
// 16-bit range (the float-to-integer conversion saturates).  The value of
// code c is c + 7 (c - k), k = c clamped to the knee (exact in FP32).
__device__ __forceinline__ float tcode_fold(float q) {
    const float k = fminf(fmaxf(q, -TFIX_KNEE), TFIX_KNEE);
    return fmaf(q - k, 1.0f / TFIX_COARSE, k);
}
__device__ __forceinline__ float tcode_unfold(float c) {
    const float k = fminf(fmaxf(c, -TFIX_KNEE), TFIX_KNEE);
    return fmaf(c - k, TFIX_COARSE - 1.0f, c);
}
// two codes from two values in code units (a in the low half)
__device__ __forceinline__ uint32_t enc_tcode2(float a, float b) {
    uint32_t w;
    asm("{\n\t.reg .s16 lo, hi;\n\t"
        "cvt.rni.s16.f32 lo, %1;\n\t"
        "cvt.rni.s16.f32 hi, %2;\n\t"
        "mov.b32 %0, {lo, hi};\n\t}"
        : "=r"(w)
        : "f"(tcode_fold(a)), "f"(tcode_fold(b)));
    return w;
}
// the two values in code units of a word of two codes
__device__ __forceinline__ float2 dec_tcode2(uint32_t w) {
    float a, b;
    asm("{\n\t.reg .s16 lo, hi;\n\t"
        "mov.b32 {lo, hi}, %2;\n\t"
        "cvt.rn.f32.s16 %0, lo;\n\t"
        "cvt.rn.f32.s16 %1, hi;\n\t}"
        : "=f"(a), "=f"(b)
        : "r"(w));
    return make_float2(tcode_unfold(a), tcode_unfold(b));
}
__device__ __forceinline__ unsigned int enc_tfix(float v, const InstDesc& d) {
    short c;
    asm("cvt.rni.s16.f32 %0, %1;" : "=h"(c) : "f"(tcode_fold(v * d.Tscale)));
    return (unsigned int)(unsigned short)c;
}
__device__ __forceinline__ float dec_tfix(unsigned int h, const InstDesc& d) {
    return tcode_unfold((float)(short)(unsigned short)h) * d.Tstep;
}

// Populations are read through L2 only: each slot is read once per step, and
// the dataflow kernel reads slots that other SMs wrote during the same launch.
template <int POL = ST_STREAM>
struct StF64T {
    using T = double;
    using R = double;
    using A = double;  // per-thread and per-warp partials of the observables
    static constexpr int kPol = POL;
    static __device__ __forceinline__ R ldf(const T* p, const InstDesc&) { return __ldcg(p); }
    static __device__ __forceinline__ void stf(T* p, R v, const InstDesc&) { st_pol<POL>(p, v); }
    static __device__ __forceinline__ R ldT(const T* p, const InstDesc&) { return __ldcg(p); }
    static __device__ __forceinline__ void stT(T* p, R v, const InstDesc&) { st_pol<POL>(p, v); }
};
// The FP32-arithmetic storages read populations through L2 only (each slot
// is read once per step, so L1 would only hold dead lines) and write them as
// streaming stores (evict-first: the next step reads them from DRAM anyway).
template <int POL = ST_STREAM>
struct StF32T {
    using T = float;
    using R = float;
    using A = float;  // per-thread and per-warp partials (tiles fold in FP64)
    static constexpr int kPol = POL;
    static __device__ __forceinline__ R ldf(const T* p, const InstDesc&) { return __ldcg(p); }
    static __device__ __forceinline__ void stf(T* p, R v, const InstDesc&) { st_pol<POL>(p, v); }
    static __device__ __forceinline__ R ldT(const T* p, const InstDesc&) { return __ldcg(p); }
    static __device__ __forceinline__ void stT(T* p, R v, const InstDesc&) { st_pol<POL>(p, v); }
    // two neighbouring cells (p 8-byte aligned)
    static __device__ __forceinline__ float2 ldf2(const T* p, const InstDesc&) {
        return __ldcg(reinterpret_cast<const float2*>(p));
    }
    static __device__ __forceinline__ void stf2(T* p, float a, float b, const InstDesc&) {
        st_pol<POL>(reinterpret_cast<float2*>(p), make_float2(a, b));
    }
    static __device__ __forceinline__ float2 ldT2(const T* p, const InstDesc& d) { return ldf2(p, d); }
    static __device__ __forceinline__ void stT2(T* p, float a, float b, const InstDesc& d) { stf2(p, a, b, d); }
    // decode a value staged in shared memory (plain load: not a global address)
    static __device__ __forceinline__ R sldf(const T* p, const InstDesc&) { return *p; }
    static __device__ __forceinline__ R sldT(const T* p, const InstDesc&) { return *p; }
};
template <int POL = ST_STREAM>
struct StF16T {
    using T = __half;
    using R = float;
    using A = float;  // per-thread and per-warp partials (tiles fold in FP64)
    static constexpr int kPol = POL;
    // stored flow value = value * 2^kLog2S (the host's fscale)
    static constexpr int kLog2S = 12;
    // packed pairs of 16-bit codes (the vector path): the lower column in the
    // low half of a 32-bit word; the _raw forms convert the stored values
    // without the scale (the vector path's collision takes them scaled)
    static __device__ __forceinline__ uint32_t encf2_raw(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    static __device__ __forceinline__ float2 decf2_raw(uint32_t w) {
        return __half22float2(*reinterpret_cast<const __half2*>(&w));
    }
    static __device__ __forceinline__ uint32_t encf2(float a, float b, const InstDesc& d) {
        const __half2 h = __floats2half2_rn(a * d.fscale, b * d.fscale);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    static __device__ __forceinline__ float2 decf2(uint32_t w, const InstDesc& d) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w));
        return make_float2(v.x * d.finv, v.y * d.finv);
    }
    static __device__ __forceinline__ R ldf(const T* p, const InstDesc& d) {
        return __half2float(__ldcg(p)) * d.finv;
    }
    static __device__ __forceinline__ void stf(T* p, R v, const InstDesc& d) {
        st_pol<POL>(p, __float2half_rn(v * d.fscale));
    }
    static __device__ __forceinline__ float2 ldf2(const T* p, const InstDesc& d) {
        const float2 v = __half22float2(__ldcg(reinterpret_cast<const __half2*>(p)));
        return make_float2(v.x * d.finv, v.y * d.finv);
    }
    static __device__ __forceinline__ void stf2(T* p, float a, float b, const InstDesc& d) {
        st_pol<POL>(reinterpret_cast<__half2*>(p), __floats2half2_rn(a * d.fscale, b * d.fscale));
    }
    static __device__ __forceinline__ R sldf(const T* p, const InstDesc& d) { return __half2float(*p) * d.finv; }
    // heat deviations: 16-bit companded fixed point (enc_tfix / dec_tfix)
    static __device__ __forceinline__ uint32_t encT2(float a, float b, const InstDesc& d) {
        return enc_tcode2(a * d.Tscale, b * d.Tscale);
    }
    static __device__ __forceinline__ float2 decT2(uint32_t w, const InstDesc& d) {
        const float2 v = dec_tcode2(w);
        return make_float2(v.x * d.Tstep, v.y * d.Tstep);
    }
    static __device__ __forceinline__ R ldT(const T* p, const InstDesc& d) {
        return dec_tfix(__ldcg(reinterpret_cast<const unsigned short*>(p)), d);
    }
    static __device__ __forceinline__ void stT(T* p, R v, const InstDesc& d) {
        st_pol<POL>(reinterpret_cast<unsigned short*>(p), (unsigned short)enc_tfix(v, d));
    }
    static __device__ __forceinline__ float2 ldT2(const T* p, const InstDesc& d) {
        return decT2(__ldcg(reinterpret_cast<const unsigned int*>(p)), d);
    }
    static __device__ __forceinline__ void stT2(T* p, float a, float b, const InstDesc& d) {
        st_pol<POL>(reinterpret_cast<unsigned int*>(p), encT2(a, b, d));
    }
    static __device__ __forceinline__ R sldT(const T* p, const InstDesc& d) {
        return dec_tfix(*reinterpret_cast<const unsigned short*>(p), d);
    }
};
template <int POL = ST_STREAM>
struct StBF16T {
    using T = __nv_bfloat16;
    using R = float;
    using A = float;  // per-thread and per-warp partials (tiles fold in FP64)
    static constexpr int kPol = POL;
    static constexpr int kLog2S = 0;  // stored unscaled (fscale 1)
    static __device__ __forceinline__ uint32_t encf2_raw(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    static __device__ __forceinline__ float2 decf2_raw(uint32_t w) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    }
    static __device__ __forceinline__ uint32_t encf2(float a, float b, const InstDesc& d) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a * d.fscale, b * d.fscale);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    static __device__ __forceinline__ float2 decf2(uint32_t w, const InstDesc& d) {
        const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
        return make_float2(v.x * d.finv, v.y * d.finv);
    }
    static __device__ __forceinline__ R ldf(const T* p, const InstDesc& d) {
        return __bfloat162float(__ldcg(p)) * d.finv;
    }
    static __device__ __forceinline__ void stf(T* p, R v, const InstDesc& d) {
        st_pol<POL>(p, __float2bfloat16_rn(v * d.fscale));
    }
    static __device__ __forceinline__ float2 ldf2(const T* p, const InstDesc& d) {
        const float2 v = __bfloat1622float2(__ldcg(reinterpret_cast<const __nv_bfloat162*>(p)));
        return make_float2(v.x * d.finv, v.y * d.finv);
    }
    static __device__ __forceinline__ void stf2(T* p, float a, float b, const InstDesc& d) {
        st_pol<POL>(reinterpret_cast<__nv_bfloat162*>(p), __floats2bfloat162_rn(a * d.fscale, b * d.fscale));
    }
    static __device__ __forceinline__ R sldf(const T* p, const InstDesc& d) {
        return __bfloat162float(*p) * d.finv;
    }
    // heat deviations: 16-bit companded fixed point (enc_tfix / dec_tfix)
    static __device__ __forceinline__ uint32_t encT2(float a, float b, const InstDesc& d) {
        return enc_tcode2(a * d.Tscale, b * d.Tscale);
    }
    static __device__ __forceinline__ float2 decT2(uint32_t w, const InstDesc& d) {
        const float2 v = dec_tcode2(w);
        return make_float2(v.x * d.Tstep, v.y * d.Tstep);
    }
    static __device__ __forceinline__ R ldT(const T* p, const InstDesc& d) {
        return dec_tfix(__ldcg(reinterpret_cast<const unsigned short*>(p)), d);
    }
    static __device__ __forceinline__ void stT(T* p, R v, const InstDesc& d) {
        st_pol<POL>(reinterpret_cast<unsigned short*>(p), (unsigned short)enc_tfix(v, d));
    }
    static __device__ __forceinline__ float2 ldT2(const T* p, const InstDesc& d) {
        return decT2(__ldcg(reinterpret_cast<const unsigned int*>(p)), d);
    }
    static __device__ __forceinline__ void stT2(T* p, float a, float b, const InstDesc& d) {
        st_pol<POL>(reinterpret_cast<unsigned int*>(p), encT2(a, b, d));
    }
    static __device__ __forceinline__ R sldT(const T* p, const InstDesc& d) {
        return dec_tfix(*reinterpret_cast<const unsigned short*>(p), d);
    }
};

using StF64 = StF64T<ST_STREAM>;
using StF32 = StF32T<ST_STREAM>;
using StF16 = StF16T<ST_STREAM>;
using StBF16 = StBF16T<ST_STREAM>;

// ---- launchers (one translation unit per arithmetic precision) -----------
// precision: 0 f64, 1 f32, 2 f16-dev, 3 bf16-dev.
// all: nchunks edge-cell chunks, then ntiles tiles; cap: most blocks (0: one per entry)
cudaError_t launch_step(int precision, const InstDesc* insts, const int4* all, int nchunks, int ntiles,
                        int flip, int mode, Shape shape, int cap, cudaStream_t s);
cudaError_t launch_finalize(const InstDesc* insts, int ninst, cudaStream_t s);

// Kernel, block shape and dynamic shared memory of one step launch (also the
// parameters of a CUDA graph kernel node).
struct StepPlan {
    const void* func;
    dim3 block;
    size_t smem;
    int max_grid = 0;  // persistent kernels: co-resident blocks on the device (0: no cap)
    bool edges = false;  // runs the tile list's second part, tiles and edge-cell chunks
};
// mode: the step's observation mode (0 for a plain step)
StepPlan step_plan(int precision, int mode, Shape shape);
// status word of the staged kernel: 0, or 1 after one of its waits expired
// (read and cleared)
cudaError_t take_step_status(int* status);
StepPlan step_plan_f64(int mode, Shape shape);
StepPlan step_plan_lp(int precision, int mode, Shape shape);
// Dataflow kernel advancing a tile list by many steps in one cooperative
// launch; keep = L2-resident stores (sweeps of several steps).
StepPlan flow_plan(int precision, Shape shape, bool keep);
StepPlan flow_plan_f64(Shape shape, bool keep);
StepPlan flow_plan_lp(int precision, Shape shape, bool keep);

// Work items of a dataflow sweep: x = (k << 24) | instance (k: step of the
// sweep), y = tile index in the tile list (| TILE_PURE), z, w = tile origin.
constexpr int SWEEP_MAX = 8;
struct FlowArgs {
    const int4* items;  // per_sweep items of one sweep, in issue order
    const int* nbr;     // 8 neighbour tiles per tile, -1: none
    int* flags;         // status, abort, then one progress word per tile
    int ntiles, per_sweep, sweep_steps, nsteps, flip;
    int stall_tile;     // test hook: this tile never reports progress (-1: none)
};
cudaError_t launch_flow(int precision, const InstDesc* insts, const FlowArgs& fa, Shape shape,
                        bool keep, int grid, cudaStream_t s);

}  // namespace lbm
