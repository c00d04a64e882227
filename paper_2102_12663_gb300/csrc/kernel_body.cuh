// The fused time step: one kernel updates every active cell of a tile list
// (one or many problem instances) by Guo's incompressible D2Q9 BGK model with
// Boussinesq forcing (arXiv 2102.12663, Eqs. 6-10, 15-17), mid-step Darcy drag
// in porous cells (Eq. 4), the D2Q4 heat BGK model (Eqs. 11-14) and link-wise
// boundary rules, streaming in place with the AA pattern:
//   even step: read f_i(x) from slot (x, i), write post-collision f*_i to
//              slot (x, opp(i));
//   odd step:  read f_i(x) from slot (x - e_i, opp(i)), write f*_i to slot
//              (x + e_i, i).
// Each cell reads and writes the same set of slots, so the update is race
// free in place.  A link that ends in a boundary cell is resolved at write
// time: the reflected value goes to the slot the next step reads for the
// reversed population (slot (x + e_i, i) after an even step, (x, opp(i))
// after an odd one), so reads never branch on the mask.
//
// Evaluation order.  Every expression below is evaluated in the same order as
// the definitions it implements (moments summed over i = 1..8 in index order,
// S_i = w_i ((3 e.u + 4.5 (e.u) e.u) - 1.5 |u|^2), collision
// (f - omega (f - feq)) + F_i, ...).  Built without FMA contraction the FP64
// instantiation therefore reproduces a plain sequential FP64 evaluation of the
// model bit for bit; the FP32 instantiation may contract.
#pragma once

#include <type_traits>

#include "lbm_internal.cuh"

// Resident blocks of 256 threads the kernels are compiled for (register
// budget 65536 / (256 * n)): the two-cell pair path keeps 26 populations and
// the collision temporaries of two cells live.  FP32 storage, one launch per
// step: 4 (64 registers, a few spilled bytes; more warps to hide memory
// latency measured faster than 3).  FP32 dataflow kernel: 3 (its per-tile
// waits and barriers do better with fewer, fatter blocks).  FP64: 3.
#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 4
#endif
#ifndef LBM_FLOW_MIN_BLOCKS
#define LBM_FLOW_MIN_BLOCKS 3
#endif
// the 16-bit storages: 2 (128 registers), for the eight-cell vector path,
// which keeps 13 planes of eight packed codes live
#ifndef LBM_STEP_MIN_BLOCKS_16
#define LBM_STEP_MIN_BLOCKS_16 2
#endif

namespace lbm {

template <class ST>
constexpr int step_min_blocks() {
    return sizeof(typename ST::T) == 2 ? LBM_STEP_MIN_BLOCKS_16
                                       : (sizeof(typename ST::T) == 4 ? LBM_STEP_MIN_BLOCKS : 3);
}
template <class ST>
constexpr int flow_min_blocks() {
    return sizeof(typename ST::T) == 2 ? LBM_STEP_MIN_BLOCKS_16 : (sizeof(typename ST::T) == 4 ? LBM_FLOW_MIN_BLOCKS : 3);
}

// Free constants of Eq. 7 (lambda + gamma = sigma, lambda + 2 gamma = 1/2)
// and the D2Q9 weights of Eq. 8.
constexpr double K_SIGMA = 5.0 / 12.0;
constexpr double K_LAMBDA = 1.0 / 3.0;
constexpr double K_GAMMA = 1.0 / 12.0;
constexpr double K_W0 = 4.0 / 9.0;
constexpr double K_W1 = 1.0 / 9.0;
constexpr double K_W5 = 1.0 / 36.0;

__device__ __forceinline__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
__device__ __forceinline__ constexpr int ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ constexpr int ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ constexpr double wgt(int i) {
    return i == 0 ? K_W0 : (i <= 4 ? K_W1 : K_W5);
}

// Arithmetic rounded one operation at a time: no multiply and add of an Rn
// expression is ever fused, so a function written in Rn computes the same
// bits in every kernel that inlines it (the compiler's contraction choices
// depend on the surrounding code).  Operands of an operation must both be Rn;
// mixing in a plain R or double does not compile.
template <class R>
struct Rn {
    R v;
    Rn() = default;
    __host__ __device__ constexpr Rn(R a) : v(a) {}
    template <class U>
    __host__ __device__ constexpr explicit Rn(U a) : v(R(a)) {}
};
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }
template <class R>
__device__ __forceinline__ Rn<R> operator+(Rn<R> a, Rn<R> b) { return Rn<R>(rn_add(a.v, b.v)); }
template <class R>
__device__ __forceinline__ Rn<R> operator-(Rn<R> a, Rn<R> b) { return Rn<R>(rn_sub(a.v, b.v)); }
template <class R>
__device__ __forceinline__ Rn<R> operator*(Rn<R> a, Rn<R> b) { return Rn<R>(rn_mul(a.v, b.v)); }
template <class R>
__device__ __forceinline__ Rn<R> operator/(Rn<R> a, Rn<R> b) { return Rn<R>(rn_div(a.v, b.v)); }
template <class R>
__device__ __forceinline__ Rn<R> operator-(Rn<R> a) { return Rn<R>(-a.v); }

// FP64 partials: a shuffle tree per warp, then one across the warps.
__device__ __forceinline__ void warp_block_reduce_f64(double* acc, double (*red)[NPART], double* out) {
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (nthreads + 31) >> 5;
    // lanes present in this warp (a block of fewer than 32 threads, or a last
    // partial warp, has fewer)
    const int width = min(32, nthreads - (warp << 5));
    const unsigned mask = width == 32 ? 0xffffffffu : ((1u << width) - 1u);
#pragma unroll
    for (int k = 0; k < NPART; ++k) {
        double v = acc[k];
        // most slots (wall shear, fluxes, counts of boundary cells) are zero
        // in a whole warp away from the walls: skip their FP64 shuffle tree
        if (__any_sync(mask, v != 0.0)) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double o = __shfl_down_sync(mask, v, off);
                if (lane + off < width) v = k < NSUM ? v + o : fmax(v, o);
            }
        } else {
            v = 0.0;
        }
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NPART; ++k) {
            double v = lane < nwarps ? red[lane][k] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double o = __shfl_down_sync(mask, v, off);
                if (lane + off < width) v = k < NSUM ? v + o : fmax(v, o);
            }
            if (lane == 0) out[k] = v;
        }
    }
}

__device__ __forceinline__ double amax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float amax(float a, float b) { return fmaxf(a, b); }

// Block reduction of the per-thread partials acc (A: the storage's
// accumulator type) into out[NPART] (FP64): sums for slots < NSUM, maxima
// for the rest.  FP64 partials reduce by a shuffle tree per warp and one more
// across warps.  FP32 partials (the FP32-arithmetic storages) reduce by an
// FP32 shuffle tree per warp, then one thread per slot folds the warps'
// values in FP64 in warp order: GB300's FP64 pipe is narrow, and FP64
// shuffle trees over every tile made the observing step FP64-bound.
template <class A>
__device__ __forceinline__ void warp_block_reduce(A* acc, double (*red)[NPART], double* out) {
    if constexpr (std::is_same<A, double>::value) {
        warp_block_reduce_f64(acc, red, out);
    } else {
        const int nthreads = blockDim.x * blockDim.y;
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        const int lane = tid & 31, warp = tid >> 5;
        const int nwarps = (nthreads + 31) >> 5;
        const int width = min(32, nthreads - (warp << 5));
        const unsigned mask = width == 32 ? 0xffffffffu : ((1u << width) - 1u);
#pragma unroll
        for (int k = 0; k < NPART; ++k) {
            A v = acc[k];
            if (__any_sync(mask, v != A(0))) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const A o = __shfl_down_sync(mask, v, off);
                    if (lane + off < width) v = k < NSUM ? v + o : amax(v, o);
                }
            } else {
                v = A(0);
            }
            if (lane == 0) red[warp][k] = (double)v;
        }
        __syncthreads();
        if (tid < NPART) {
            double v = red[0][tid];
            for (int w = 1; w < nwarps; ++w) v = tid < NSUM ? v + red[w][tid] : fmax(v, red[w][tid]);
            out[tid] = v;
        }
    }
}

// Programmatic dependent launch: allow the dependent grid to launch, and wait
// until the prerequisite grid has completed with its memory visible.  Both
// are no-ops for a kernel launched without a programmatic dependency.
__device__ __forceinline__ void grid_dependents_go() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// neighbour indices of cell (x, y) (wrap-around only ever triggers on
// periodic edges: a non-periodic edge holds no active cell)
__device__ __forceinline__ void neighbours(const InstDesc& d, int x, int y, int* nb) {
    const int nx = d.nx, ny = d.ny;
    const int xl = x == 0 ? nx - 1 : x - 1;
    const int xr = x == nx - 1 ? 0 : x + 1;
    const int yd = (y == 0 ? ny - 1 : y - 1) * nx;
    const int yu = (y == ny - 1 ? 0 : y + 1) * nx;
    const int yc = y * nx;
    nb[0] = yc + x;
    nb[1] = yc + xr;
    nb[2] = yu + x;
    nb[3] = yc + xl;
    nb[4] = yd + x;
    nb[5] = yu + xr;
    nb[6] = yu + xl;
    nb[7] = yd + xl;
    nb[8] = yd + xr;
}

// Curved-cell entry of cell (x, y) (a short scan of its column), or null.
__device__ __forceinline__ const CurvedCell* curved_entry(const InstDesc& d, int x, int y) {
    for (int k = d.qcol[x]; k < d.qcol[x + 1]; ++k)
        if (d.qtab[k].y == y) return d.qtab + k;
    return nullptr;
}

// Bouzidi's rule for a wall at fraction q < 1/2 of link i, applied when the
// cell reads its populations: the slot of f_o (o = opp(i)) holds the cell's
// own post-collision f*_i of the previous step (written there as halfway
// bounce-back), and f_i holds f*_i of the upstream cell x - e_i, streamed in;
// f_o = 2q f*_i(x) + (1 - 2q) f*_i(x - e_i).  Links with q < 1/2 always have
// an active upstream cell, so the opposite link is no wall link of this kind
// and the corrections of one cell do not feed each other.
template <class V>
__device__ __forceinline__ void bouzidi_read(const CurvedCell* ce, V* f) {
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const double q = ce->q[i - 1];
        if (q < 0.5) {
            const V qq = V(q);
            f[opp(i)] = (V(2.0) * qq) * f[opp(i)] + (V(1.0) - V(2.0) * qq) * f[i];
        }
    }
}

// Load the mask byte and the 13 populations of cell nb[0] (AA read pattern).
// The mask and all populations are requested together (every slot index is
// in range for any cell of the grid), so an active cell pays one memory round
// trip; a solid cell inside a launched tile discards them.
template <class ST, int PAR>
__device__ __forceinline__ void load_cell(const InstDesc& d, const int* nb, typename ST::R* f,
                                          typename ST::R* g, uint8_t& m) {
    using T = typename ST::T;
    const T* const P = static_cast<const T*>(d.pops);
    const int np = (int)d.npad;  // 13 * npad < 2^31 (checked at creation)
    const int c = nb[0];
    m = d.mask[c];
    if (PAR == 0) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = ST::ldf(P + i * np + c, d);
#pragma unroll
        for (int i = 1; i <= 4; ++i) g[i - 1] = ST::ldT(P + (8 + i) * np + c, d);
    } else {
        f[0] = ST::ldf(P + c, d);
#pragma unroll
        for (int i = 1; i < 9; ++i) f[i] = ST::ldf(P + opp(i) * np + nb[opp(i)], d);
#pragma unroll
        for (int i = 1; i <= 4; ++i) g[i - 1] = ST::ldT(P + (8 + opp(i)) * np + nb[opp(i)], d);
    }
}

// Everything after the load: observables, collision, boundary rules, stores.
// The arithmetic runs in Rn<R> (each operation rounded on its own), so the
// update is the same function of the loaded populations in every kernel that
// inlines it.
template <class ST, bool OBS, int PAR, class A = double>
__device__ __forceinline__ void cell_body(const InstDesc& d, int x, int y,
                                          const typename ST::R* fin, const typename ST::R* gin,
                                          uint8_t m, int mode, A* acc,
                                          int64_t ntw = -1) {
    using T = typename ST::T;
    using R = typename ST::R;
    using E = Rn<R>;
    const int nx = d.nx, ny = d.ny;
    int nb[9];
    neighbours(d, x, y, nb);
    const int c = nb[0];
    const int xl = x == 0 ? nx - 1 : x - 1;
    const int xr = x == nx - 1 ? 0 : x + 1;
    T* const P = static_cast<T*>(d.pops);
    const int np = (int)d.npad;
    const Phys<R>& ph = phys<R>(d);
    const int type = m & TYPE_BITS;
    if (type > POROUS) return;
    E f[9], g[4];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = fin[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) g[i] = gin[i];
    // interpolated bounce-back on the curved cornea (Bouzidi): q < 1/2 links
    // are completed here, q > 1/2 links when they are written below
    const CurvedCell* ce = nullptr;
    if (d.bouzidi && (m & CURVED)) {
        ce = curved_entry(d, x, y);
        if (ce) bouzidi_read<E>(ce, f);
    }

    // ---- moments, Eq. 9 and Eq. 13 ------------------------------------------
    const E ux = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const E uy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    const E usq = ux * ux + uy * uy;
    const E S0 = E(K_W0) * (E(-1.5) * usq);
    const E sum18 = f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    // p = [sum_{i>=1} f_i + S_0(u)] / (4 sigma); the FP32 form multiplies by 0.6.
    // Pressure parts of feq_1..8: lambda p (axis) and gamma p (diagonal).  In
    // FP64 they are formed from p as Eq. 7 writes them.  In FP32 (whose
    // rounded constants 0.6, 1/3 and 1/12 all lie above the exact values) they
    // are formed from P4 = 4 sigma p = sum18 + S_0: lambda p = P4 / 5, and
    // gamma p = P4 / 4 - lambda p, an exact subtraction (Sterbenz), so the
    // eight parts add up to P4 exactly.
    const E P4 = sum18 + S0;
    const E p = sizeof(R) == 8 ? P4 / E(4.0 * K_SIGMA) : P4 * E(0.6);
    const E pax = sizeof(R) == 8 ? E(K_LAMBDA) * p : P4 * E(0.2);
    const E pdg = sizeof(R) == 8 ? E(K_GAMMA) * p : P4 * E(0.25) - pax;
    // T - Tref (Eq. 13 on the stored deviations; Tref = 0 for FP64)
    const E Tm = g[0] + g[1] + g[2] + g[3];

    // e_i . u for i = 0..8
    E eu[9];
    eu[0] = E(0.0);
    eu[1] = ux;
    eu[2] = uy;
    eu[3] = -ux;
    eu[4] = -uy;
    eu[5] = ux + uy;
    eu[6] = -ux + uy;
    eu[7] = -ux - uy;
    eu[8] = ux - uy;

    // equilibrium, Eqs. 7-8
    E feq[9];
    feq[0] = (sizeof(R) == 8 ? E(-4.0 * K_SIGMA) * p : -P4) + S0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const E Si = E(wgt(i)) * (E(3.0) * eu[i] + E(4.5) * eu[i] * eu[i] - E(1.5) * usq);
        feq[i] = (i <= 4 ? pax : pdg) + Si;
    }

    // neighbour types (only next to a boundary)
    // (ntw >= 0: the host's word of them, an edge cell's; else read here)
    uint32_t ntypes = 0, bnd = 0;
    if (m & NEAR_BOUNDARY) {
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const uint32_t tn = ntw >= 0 ? ((uint32_t)ntw >> (4 * (i - 1))) & 15u : d.mask[nb[i]] & TYPE_BITS;
            ntypes |= tn << (4 * (i - 1));
            if (tn > POROUS) bnd |= 1u << i;
        }
    }

    // ---- observables of the pre-collision state -----------------------------
    if (OBS) {
        if (mode & OBS_STATS) {
            acc[P_MASS] += (A)sum18.v;
            // max of |u|^2; the fold takes one square root (sqrt is monotone)
            acc[P_PEAK] = amax(acc[P_PEAK], (A)usq.v);
            if (type == FLUID) {
                acc[P_SUM_P] += (A)p.v;
                acc[P_N_FLUID] += A(1);
                if (!isfinite((double)p.v)) acc[P_NAN] += A(1);
                if (bnd) {
                    bool hit_c = false, hit_h = false;
                    double ac_x = 0.0, ac_y = 0.0, ah_x = 0.0, ah_y = 0.0;
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        const uint32_t tn = (ntypes >> (4 * (i - 1))) & 15u;
                        if (tn == COLD) { hit_c = true; ac_x += ex(i); ac_y += ey(i); }
                        if (tn == HOT) { hit_h = true; ah_x += ex(i); ah_y += ey(i); }
                    }
                    if (hit_c || hit_h) {
                        // non-equilibrium stress sigma = -(1 - 1/(2 tau)) sum e e (f - feq)
                        const double d1 = (double)(f[1] - feq[1]).v, d2 = (double)(f[2] - feq[2]).v;
                        const double d3 = (double)(f[3] - feq[3]).v, d4 = (double)(f[4] - feq[4]).v;
                        const double d5 = (double)(f[5] - feq[5]).v, d6 = (double)(f[6] - feq[6]).v;
                        const double d7 = (double)(f[7] - feq[7]).v, d8 = (double)(f[8] - feq[8]).v;
                        const double pxx = d1 + d3 + d5 + d6 + d7 + d8;
                        const double pxy = d5 - d6 + d7 - d8;
                        const double pyy = d2 + d4 + d5 + d6 + d7 + d8;
                        const double kw = d.pd.kwss;
                        const double sxx = kw * pxx, sxy = kw * pxy, syy = kw * pyy;
                        if (hit_c) {
                            double ax = ac_x, ay = ac_y;
                            if (d.eye_normals) { ax = x - d.arc_xc; ay = y - d.arc_yc; }
                            const double r = sqrt(ax * ax + ay * ay);
                            const double nxw = r > 0.0 ? ax / r : 0.0, nyw = r > 0.0 ? ay / r : 0.0;
                            acc[P_WSS_C] += (A)fabs(-nyw * (sxx * nxw + sxy * nyw) + nxw * (sxy * nxw + syy * nyw));
                            acc[P_N_C] += A(1);
                        }
                        if (hit_h) {
                            double ax = ah_x, ay = ah_y;
                            if (d.eye_normals) { ax = 0.0; ay = 1.0; }
                            const double r = sqrt(ax * ax + ay * ay);
                            const double nxw = r > 0.0 ? ax / r : 0.0, nyw = r > 0.0 ? ay / r : 0.0;
                            acc[P_WSS_I] += (A)fabs(-nyw * (sxx * nxw + sxy * nyw) + nxw * (sxy * nxw + syy * nyw));
                            acc[P_N_I] += A(1);
                        }
                    }
                }
            }
        }
        if (mode & (OBS_RESID | OBS_SNAP)) {
            R* U = static_cast<R*>(d.usnap);
            if ((mode & OBS_RESID) && d.snap_valid) {
                const double dx = (double)ux.v - (double)U[c];
                const double dy = (double)uy.v - (double)U[np + c];
                acc[P_RESID] = amax(acc[P_RESID], (A)(dx * dx + dy * dy));
            }
            if (mode & OBS_SNAP) {
                U[c] = ux.v;
                U[np + c] = uy.v;
            }
        }
    }

    // ---- body force, Eqs. 15-17: F_i = (1/2) e_i . F on the axis links --------
    const E gb = E(ph.g_beta) * (Tm - E(ph.dT0));
    const E Fx = E(ph.drive_x) - gb * E(ph.gx);
    const E Fy = E(ph.drive_y) - gb * E(ph.gy);
    const E F1 = E(0.5) * Fx, F2 = E(0.5) * Fy;

    // ---- flow collision, Eq. 6 --------------------------------------------
    const E om = E(ph.omega);
    E fs[9];
    if constexpr (sizeof(R) == 8) {
#pragma unroll
        for (int i = 0; i < 9; ++i) fs[i] = f[i] - om * (f[i] - feq[i]);
    } else {
        // FP32: the mean of the rounded non-equilibrium parts f_i - feq_i
        // (zero in exact arithmetic) is taken out, so that the rounded
        // equilibrium adds no mass (the pair path does the same)
        E nq[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) nq[i] = f[i] - feq[i];
        const E nm = (((nq[1] + nq[3]) + (nq[2] + nq[4])) + ((nq[5] + nq[7]) + (nq[6] + nq[8]))) * E(0.125);
        fs[0] = f[0] - om * (f[0] - feq[0]);
#pragma unroll
        for (int i = 1; i < 9; ++i) fs[i] = f[i] - om * (nq[i] - nm);
    }
    fs[1] = fs[1] + F1;
    fs[2] = fs[2] + F2;
    fs[3] = fs[3] + (-F1);
    fs[4] = fs[4] + (-F2);

    // ---- Darcy drag in porous cells, Eq. 4 at the mid-step velocity ---------
    // (the lumped meshwork of Sec. 2.3 resolves no flow resistance in the TM)
    if (type == POROUS && d.tm_model == 0) {
        const E den = E(ph.den), cK = E(ph.cK);
        const E umx = (ux + E(0.5) * Fx) / den;
        const E umy = (uy + E(0.5) * Fy) / den;
        const E FDx = -cK * umx;
        const E FDy = -cK * umy;
        const E a1 = E(3.0 * K_W1), a5 = E(3.0 * K_W5);
        fs[1] = fs[1] + a1 * FDx;
        fs[2] = fs[2] + a1 * FDy;
        fs[3] = fs[3] + a1 * (-FDx);
        fs[4] = fs[4] + a1 * (-FDy);
        fs[5] = fs[5] + a5 * (FDx + FDy);
        fs[6] = fs[6] + a5 * (-FDx + FDy);
        fs[7] = fs[7] + a5 * (-FDx - FDy);
        fs[8] = fs[8] + a5 * (FDx - FDy);
    }

    // ---- heat collision, Eqs. 11-12 ----------------------------------------
    const E omT = E(ph.omegaT);
    const E Tq = E(0.25) * Tm;
    E gs[4];
    if constexpr (sizeof(R) == 8) {
#pragma unroll
        for (int i = 1; i <= 4; ++i) {
            const E teq = Tq * (E(1.0) + E(2.0) * eu[i]);
            gs[i - 1] = g[i - 1] - omT * (g[i - 1] - teq);
        }
    } else {
        // FP32, on the deviations from Tref/4: T_i^eq - Tref/4 =
        // (T - Tref)/4 + (T/2) e_i.u; the mean of the rounded non-equilibrium
        // parts is taken out, so that the rounded equilibrium adds no heat
        const E Th = E(0.5) * (Tm + E(ph.Tref));
        E nt[4];
#pragma unroll
        for (int i = 1; i <= 4; ++i) nt[i - 1] = g[i - 1] - (Tq + Th * eu[i]);
        const E mt = ((nt[0] + nt[2]) + (nt[1] + nt[3])) * E(0.25);
#pragma unroll
        for (int i = 0; i < 4; ++i) gs[i] = g[i] - omT * (nt[i] - mt);
    }

    const bool write = !OBS || (mode & OBS_WRITE);

    // ---- stream (AA write pattern) with link-wise boundary rules ----------
    if (write) ST::stf(P + c, fs[0].v, d);
    double q_in = 0.0, q_out = 0.0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const bool is_bnd = (bnd >> i) & 1u;
        E v = fs[i];
        if (is_bnd) {
            const uint32_t tn = (ntypes >> (4 * (i - 1))) & 15u;
            if (tn == INLET) {
                // moving-wall bounce-back; 6 w_i e_i.u is the odd part of feq
                const int xn = ex(i) == 1 ? xr : (ex(i) == -1 ? xl : x);
                const int ynb = ey(i) == 1 ? (y == ny - 1 ? 0 : y + 1)
                                           : (ey(i) == -1 ? (y == 0 ? ny - 1 : y - 1) : y);
                E shape = E(1.0);
                if (d.inlet_profile == 1) {
                    const int cg = d.inlet_dir_x == 0 ? xn : ynb;
                    const E s = (E(cg - d.inlet_lo) + E(0.5)) / E(d.inlet_width);
                    shape = E(4.0) * s * (E(1.0) - s);
                }
                const E uin = E(ph.u_in_max) * shape;
                const E uix = uin * E(d.inlet_dir_x), uiy = uin * E(d.inlet_dir_y);
                v = fs[i] - E(6.0 * wgt(i)) * (E(ex(i)) * uix + E(ey(i)) * uiy);
                if (OBS) q_in += (double)(v - fs[i]).v;
            } else if (tn == OUTLET && d.tm_model == 1) {
                // lumped TM (Sec. 2.3): the seepage velocity, out of the domain
                // along the outlet axis, as a moving wall
                const E uwx = d.outlet_axis == 0 ? E(ph.u_seep) * E(ex(i)) : E(0.0);
                const E uwy = d.outlet_axis == 1 ? E(ph.u_seep) * E(ey(i)) : E(0.0);
                v = fs[i] - E(6.0 * wgt(i)) * (E(ex(i)) * uwx + E(ey(i)) * uwy);
                if (OBS) q_out += (double)(fs[i] - v).v;
            } else if (tn == OUTLET) {
                // pressure anti-bounce-back: minus f* plus the even part of feq(p_out, u)
                const E kap = i <= 4 ? E(K_LAMBDA) : E(K_GAMMA);
                v = -fs[i] + E(2.0) * (kap * E(ph.p_out) +
                                       E(wgt(i)) * (E(4.5) * eu[i] * eu[i] - E(1.5) * usq));
                if (OBS) q_out += (double)(fs[i] - v).v;
            } else if (tn == COLD && ce) {
                // curved cornea, wall beyond the link's midpoint (q > 1/2):
                // f_o = f*_i / (2q) + (2q - 1)/(2q) f*_o; q < 1/2 stays halfway
                // here and is completed when the cell next reads its populations
                const double q = ce->q[i - 1];
                if (q > 0.5) {
                    const E qq = E(q);
                    v = (E(1.0) / (E(2.0) * qq)) * fs[i] + ((E(2.0) * qq - E(1.0)) / (E(2.0) * qq)) * fs[opp(i)];
                }
            }
            // any other wall: halfway bounce-back, v = f*_i
        }
        if (write) {
            const bool to_own = (PAR == 0) != is_bnd;  // even+stream or odd+boundary
            if (to_own) ST::stf(P + opp(i) * np + c, v.v, d);
            else ST::stf(P + i * np + nb[i], v.v, d);
        }
    }
#pragma unroll
    for (int i = 1; i <= 4; ++i) {
        const bool is_bnd = (bnd >> i) & 1u;
        E v = gs[i - 1];
        if (is_bnd) {
            const uint32_t tn = (ntypes >> (4 * (i - 1))) & 15u;
            // anti-bounce-back of the deviations: T_w - Tref at the wall
            if (tn == COLD) v = -gs[i - 1] + E(0.5) * (E(ph.T_cold) - E(ph.Tref));
            else if (tn == HOT) v = -gs[i - 1] + E(0.5) * (E(ph.T_hot) - E(ph.Tref));
            else if (tn == INLET) v = -gs[i - 1] + E(0.5) * (E(ph.T_in) - E(ph.Tref));
            else if (tn == OUTLET) v = -gs[i - 1] + E(0.5) * Tm;
            // adiabatic: bounce-back, zero heat flux
        }
        if (write) {
            const bool to_own = (PAR == 0) != is_bnd;
            if (to_own) ST::stT(P + (8 + opp(i)) * np + c, v.v, d);
            else ST::stT(P + (8 + i) * np + nb[i], v.v, d);
        }
    }
    if (OBS && (mode & OBS_STATS)) {
        acc[P_Q_IN] += (A)q_in;
        acc[P_Q_OUT] += (A)q_out;
    }
}

template <class ST, bool OBS, int PAR, class A = double>
__device__ __forceinline__ void update_cell(const InstDesc& d, int x, int y, int mode, A* acc,
                                            int64_t ntw = -1) {
    using R = typename ST::R;
    int nb[9];
    neighbours(d, x, y, nb);
    R f[9], g[4];
    uint8_t m;
    load_cell<ST, PAR>(d, nb, f, g, m);
    cell_body<ST, OBS, PAR, A>(d, x, y, f, g, m, mode, acc, ntw);
}

// ---------------------------------------------------------------------------
// Interior fast path of the FP32-arithmetic kernels: one thread updates two
// neighbouring cells (x, x+1) of a row, both active and with no boundary
// neighbour, and every lane of its warp does the same on consecutive pairs of
// that row.  Populations move as 2-cell vectors.  On an odd step the
// x-shifted reads and writes are assembled from the neighbouring lane's pair
// by warp shuffles; the warp's first and last lanes fetch or store the one
// element that lies outside the warp.  Same model as update_cell (Eqs. 4,
// 6-17), with the equilibrium evaluated per opposite-link pair
// (feq_i, feq_opp(i) = common +- odd part).

// Flow collision (Eqs. 6-9, 15-17), Darcy drag (Eq. 4) and heat collision
// (Eqs. 11-13) of one interior cell, in place: q = 0..8 flow, 9..12 T_1..T_4.
// LOG2S: the flow values come and go scaled by S = 2^LOG2S (as a 16-bit
// storage holds them).  Every intermediate of the flow collision is then S
// times, or for the square of the velocity S^2 times, the unscaled one, with
// the same rounding: the constants that meet a product of two scaled values
// carry 1/S, the force terms S.  TCODE: the heat deviations come and go in
// code units (value * Tscale, the 16-bit storages' heat codes), with the
// run's constants gbc, dT0c, Trefc; else in the units of T.
template <int LOG2S = 0, bool TCODE = false>
__device__ __forceinline__ void collide_interior(float* f, bool porous, const InstDesc& d) {
    const Phys<float>& ph = d.pf;
    constexpr float S = float(1 << LOG2S), iS = 1.0f / float(1 << LOG2S);
    const float ux = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const float uy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    const float usq = ux * ux + uy * uy;
    const float e5 = ux + uy, e6 = uy - ux;
    // even parts w_i (4.5 (e_i.u)^2 - 1.5 |u|^2) of S_i, one per opposite pair
    constexpr float a1 = float(4.5 * K_W1) * iS, b1 = float(1.5 * K_W1) * iS;
    constexpr float a5 = float(4.5 * K_W5) * iS, b5 = float(1.5 * K_W5) * iS;
    const float h1 = a1 * ux * ux - b1 * usq;
    const float h2 = a1 * uy * uy - b1 * usq;
    const float h5 = a5 * e5 * e5 - b5 * usq;
    const float h6 = a5 * e6 * e6 - b5 * usq;
    // S_0 = -sum_{i>=1} S_i (the S_i of Eq. 8 sum to zero), from the rounded even parts
    const float S0 = -2.0f * ((h1 + h2) + (h5 + h6));
    const float sum18 = f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    // pressure parts lambda p = P4 / 5 and gamma p = P4 / 20 of P4 = 4 sigma p
    // (Eq. 9); gamma p = P4 / 4 - lambda p is exact (Sterbenz), so the eight
    // pressure parts add up to P4 exactly
    const float P4 = sum18 + S0;
    const float pax = P4 * 0.2f;
    const float pdg = P4 * 0.25f - pax;
    const float Tm = f[9] + f[10] + f[11] + f[12];  // T - Tref (stored deviations)
    const float om = ph.omega;
    // equilibrium per opposite pair: common = kappa p + even part, odd = 3 w eu
    const float q1 = pax + h1, o1 = float(3.0 * K_W1) * ux;
    const float q2 = pax + h2, o2 = float(3.0 * K_W1) * uy;
    const float q5 = pdg + h5, o5 = float(3.0 * K_W5) * e5;
    const float q6 = pdg + h6, o6 = float(3.0 * K_W5) * e6;
    const float feq0 = -P4 + S0;
    // body force F = drive - g beta (T - T0) g_hat; F_i = (1/2) e_i . F on the axis links
    const float gb = TCODE ? d.gbc * (Tm - d.dT0c) : ph.g_beta * (Tm - ph.dT0);
    const float Fx = ph.drive_x - gb * ph.gx;
    const float Fy = ph.drive_y - gb * ph.gy;
    const float F1 = (0.5f * S) * Fx, F2 = (0.5f * S) * Fy;
    // Non-equilibrium parts n_i = f_i - feq_i (exact subtractions: f_i and
    // feq_i are close).  Their sum vanishes in exact arithmetic (the
    // equilibrium carries the cell's mass sum_{i>=1} f_i, Eq. 9), but the
    // rounded equilibrium misses it by a few units in the last place of the
    // populations, with a bias that survives the sum over cells and steps: a
    // mass source whose steady outflow raises the IOP.  So the mean of the
    // rounded n_i is taken out before the relaxation; what remains of the
    // collision's mass error is the final rounding of each f_i.
    const float n1 = f[1] - (q1 + o1), n3 = f[3] - (q1 - o1);
    const float n2 = f[2] - (q2 + o2), n4 = f[4] - (q2 - o2);
    const float n5 = f[5] - (q5 + o5), n7 = f[7] - (q5 - o5);
    const float n6 = f[6] - (q6 + o6), n8 = f[8] - (q6 - o6);
    const float nm = (((n1 + n3) + (n2 + n4)) + ((n5 + n7) + (n6 + n8))) * 0.125f;
    f[0] = f[0] - om * (f[0] - feq0);
    f[1] = f[1] - om * (n1 - nm) + F1;
    f[3] = f[3] - om * (n3 - nm) - F1;
    f[2] = f[2] - om * (n2 - nm) + F2;
    f[4] = f[4] - om * (n4 - nm) - F2;
    f[5] = f[5] - om * (n5 - nm);
    f[7] = f[7] - om * (n7 - nm);
    f[6] = f[6] - om * (n6 - nm);
    f[8] = f[8] - om * (n8 - nm);
    if (porous) {
        // mid-step velocity (u + F/2) / (1 + nu / (2K)), F1 = S Fx / 2
        const float umx = (ux + F1) / ph.den;
        const float umy = (uy + F2) / ph.den;
        const float FDx = -ph.cK * umx, FDy = -ph.cK * umy;
        const float c1 = float(3.0 * K_W1), c5 = float(3.0 * K_W5);
        f[1] += c1 * FDx;
        f[3] -= c1 * FDx;
        f[2] += c1 * FDy;
        f[4] -= c1 * FDy;
        f[5] += c5 * (FDx + FDy);
        f[7] -= c5 * (FDx + FDy);
        f[6] += c5 * (FDy - FDx);
        f[8] -= c5 * (FDy - FDx);
    }
    // heat: the same for the D2Q4 populations, whose equilibria carry T.  They
    // are stored and collided as deviations from Tref/4, so their rounding is
    // that of T - Tref: T_i^eq - Tref/4 = (T - Tref)/4 + (T/2) e_i.u (the
    // velocity's scale S taken out of T/2)
    const float omT = ph.omegaT, Tq = 0.25f * Tm;
    const float Th = (0.5f * iS) * (Tm + (TCODE ? d.Trefc : ph.Tref));
    const float m1 = f[9] - (Tq + Th * ux), m3 = f[11] - (Tq - Th * ux);
    const float m2 = f[10] - (Tq + Th * uy), m4 = f[12] - (Tq - Th * uy);
    const float mm = ((m1 + m3) + (m2 + m4)) * 0.25f;
    f[9] = f[9] - omT * (m1 - mm);
    f[10] = f[10] - omT * (m2 - mm);
    f[11] = f[11] - omT * (m3 - mm);
    f[12] = f[12] - omT * (m4 - mm);
}

// The same collision for two cells at once, with Blackwell's paired FP32
// operations (component x: one cell, y: the other; one instruction per pair
// of operations, each component rounded as its scalar operation).  por: bit 0
// the first cell is porous, bit 1 the second.  The Darcy drag multiplies by
// the descriptor's 1 / den instead of dividing by den.
__device__ __forceinline__ float2 p2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p2(float s) { return make_float2(s, s); }

template <int LOG2S = 0, bool TCODE = false>
__device__ __forceinline__ void collide_interior2(float2* f, uint32_t por, const InstDesc& d) {
    const Phys<float>& ph = d.pf;
    constexpr float S = float(1 << LOG2S), iS = 1.0f / float(1 << LOG2S);
    const float2 d13 = p2sub(f[1], f[3]), d24 = p2sub(f[2], f[4]);
    const float2 d57 = p2sub(f[5], f[7]), d68 = p2sub(f[6], f[8]);
    const float2 ux = p2add(d13, p2sub(d57, d68));
    const float2 uy = p2add(d24, p2add(d57, d68));
    const float2 usq = p2fma(ux, ux, p2mul(uy, uy));
    const float2 e5 = p2add(ux, uy), e6 = p2sub(uy, ux);
    // even parts w_i (4.5 (e_i.u)^2 - 1.5 |u|^2), one per opposite pair
    constexpr float a1 = float(4.5 * K_W1) * iS, b1 = float(1.5 * K_W1) * iS;
    constexpr float a5 = float(4.5 * K_W5) * iS, b5 = float(1.5 * K_W5) * iS;
    const float2 t1 = p2mul(p2(-b1), usq), t5 = p2mul(p2(-b5), usq);
    const float2 h1 = p2fma(p2mul(p2(a1), ux), ux, t1);
    const float2 h2 = p2fma(p2mul(p2(a1), uy), uy, t1);
    const float2 h5 = p2fma(p2mul(p2(a5), e5), e5, t5);
    const float2 h6 = p2fma(p2mul(p2(a5), e6), e6, t5);
    // S_0 = -sum_{i>=1} S_i from the rounded even parts
    const float2 S0 = p2mul(p2(-2.0f), p2add(p2add(h1, h2), p2add(h5, h6)));
    const float2 sum18 = p2add(p2add(p2add(f[1], f[3]), p2add(f[2], f[4])),
                               p2add(p2add(f[5], f[7]), p2add(f[6], f[8])));
    // pressure parts lambda p = P4 / 5, gamma p = P4 / 4 - lambda p (exact)
    const float2 P4 = p2add(sum18, S0);
    const float2 pax = p2mul(P4, p2(0.2f));
    const float2 pdg = p2fma(P4, p2(0.25f), p2mul(pax, p2(-1.0f)));
    const float2 Tm = p2add(p2add(f[9], f[11]), p2add(f[10], f[12]));
    const float2 q1 = p2add(pax, h1), o1 = p2mul(p2(float(3.0 * K_W1)), ux);
    const float2 q2 = p2add(pax, h2), o2 = p2mul(p2(float(3.0 * K_W1)), uy);
    const float2 q5 = p2add(pdg, h5), o5 = p2mul(p2(float(3.0 * K_W5)), e5);
    const float2 q6 = p2add(pdg, h6), o6 = p2mul(p2(float(3.0 * K_W5)), e6);
    const float2 feq0 = p2sub(S0, P4);
    // body force F = drive - g beta (T - T0) g_hat; F_i = S (1/2) e_i . F
    const float2 gb = TCODE ? p2mul(p2(d.gbc), p2sub(Tm, p2(d.dT0c))) : p2mul(p2(ph.g_beta), p2sub(Tm, p2(ph.dT0)));
    const float2 F1 = p2mul(p2(0.5f * S), p2fma(gb, p2(-ph.gx), p2(ph.drive_x)));
    const float2 F2 = p2mul(p2(0.5f * S), p2fma(gb, p2(-ph.gy), p2(ph.drive_y)));
    // non-equilibrium parts, their mean taken out before the relaxation
    const float2 n1 = p2sub(f[1], p2add(q1, o1)), n3 = p2sub(f[3], p2sub(q1, o1));
    const float2 n2 = p2sub(f[2], p2add(q2, o2)), n4 = p2sub(f[4], p2sub(q2, o2));
    const float2 n5 = p2sub(f[5], p2add(q5, o5)), n7 = p2sub(f[7], p2sub(q5, o5));
    const float2 n6 = p2sub(f[6], p2add(q6, o6)), n8 = p2sub(f[8], p2sub(q6, o6));
    const float2 nm = p2mul(p2add(p2add(p2add(n1, n3), p2add(n2, n4)), p2add(p2add(n5, n7), p2add(n6, n8))),
                            p2(0.125f));
    const float2 mom = p2(-ph.omega);
    f[0] = p2fma(mom, p2sub(f[0], feq0), f[0]);
    f[1] = p2add(p2fma(mom, p2sub(n1, nm), f[1]), F1);
    f[3] = p2sub(p2fma(mom, p2sub(n3, nm), f[3]), F1);
    f[2] = p2add(p2fma(mom, p2sub(n2, nm), f[2]), F2);
    f[4] = p2sub(p2fma(mom, p2sub(n4, nm), f[4]), F2);
    f[5] = p2fma(mom, p2sub(n5, nm), f[5]);
    f[7] = p2fma(mom, p2sub(n7, nm), f[7]);
    f[6] = p2fma(mom, p2sub(n6, nm), f[6]);
    f[8] = p2fma(mom, p2sub(n8, nm), f[8]);
    if (por & 3u) {
        // mid-step velocity (u + F/2) / den, drag -cK u_m on the porous cell(s) only
        const float2 k = make_float2((por & 1u) ? -ph.cK * d.rden : 0.0f, (por & 2u) ? -ph.cK * d.rden : 0.0f);
        const float2 FDx = p2mul(p2add(ux, F1), k), FDy = p2mul(p2add(uy, F2), k);
        const float2 c1 = p2(float(3.0 * K_W1)), c5 = p2(float(3.0 * K_W5));
        const float2 sp = p2add(FDx, FDy), sm = p2sub(FDy, FDx);
        f[1] = p2fma(c1, FDx, f[1]);
        f[3] = p2sub(f[3], p2mul(c1, FDx));
        f[2] = p2fma(c1, FDy, f[2]);
        f[4] = p2sub(f[4], p2mul(c1, FDy));
        f[5] = p2fma(c5, sp, f[5]);
        f[7] = p2sub(f[7], p2mul(c5, sp));
        f[6] = p2fma(c5, sm, f[6]);
        f[8] = p2sub(f[8], p2mul(c5, sm));
    }
    // heat: deviations from Tref/4, T_i^eq - Tref/4 = (T - Tref)/4 + (T/2) e_i.u
    const float2 Tq = p2mul(p2(0.25f), Tm);
    const float2 Th = p2mul(p2(0.5f * iS), p2add(Tm, p2(TCODE ? d.Trefc : ph.Tref)));
    const float2 Tn = p2mul(p2(-0.5f * iS), p2add(Tm, p2(TCODE ? d.Trefc : ph.Tref)));
    const float2 m1 = p2sub(f[9], p2fma(Th, ux, Tq)), m3 = p2sub(f[11], p2fma(Tn, ux, Tq));
    const float2 m2 = p2sub(f[10], p2fma(Th, uy, Tq)), m4 = p2sub(f[12], p2fma(Tn, uy, Tq));
    const float2 mm = p2mul(p2add(p2add(m1, m3), p2add(m2, m4)), p2(0.25f));
    const float2 momT = p2(-ph.omegaT);
    f[9] = p2fma(momT, p2sub(m1, mm), f[9]);
    f[10] = p2fma(momT, p2sub(m2, mm), f[10]);
    f[11] = p2fma(momT, p2sub(m3, mm), f[11]);
    f[12] = p2fma(momT, p2sub(m4, mm), f[12]);
}

// Collision of a cell pair (cells x and x+1, 13 values each) and its AA-pattern
// stores; every lane of the warp takes part (odd steps assemble x-shifted
// links by shuffles).
template <class ST, int PAR, bool MASK = false>
__device__ __forceinline__ void pair_collide_store(const InstDesc& d, int x, int y, float* a,
                                                   float* b, bool por0, bool por1, bool mine_in = true) {
    // MASK: some lanes' pairs are not interior (their stores are left out);
    // else every lane stores (the code of the unmasked pair path)
    const bool mine = MASK ? mine_in : true;
    using T = typename ST::T;
    const int nx = d.nx, ny = d.ny;
    const int np = (int)d.npad;
    T* const P = static_cast<T*>(d.pops);
    const int lane = threadIdx.x & 31;
    const int row = y * nx;
    const int rowu = (y == ny - 1 ? 0 : y + 1) * nx;
    const int rowd = (y == 0 ? ny - 1 : y - 1) * nx;
    const int xl = x == 0 ? nx - 1 : x - 1;
    const int xr = x + 2 == nx ? 0 : x + 2;
    if constexpr (sizeof(T) == 2) {
        // 16-bit storages: the paired collision (the FP32 kernel measured
        // faster with the scalar one)
        float2 v[13];
#pragma unroll
        for (int k = 0; k < 13; ++k) v[k] = make_float2(a[k], b[k]);
        collide_interior2<0, false>(v, (por0 ? 1u : 0u) | (por1 ? 2u : 0u), d);
#pragma unroll
        for (int k = 0; k < 13; ++k) {
            a[k] = v[k].x;
            b[k] = v[k].y;
        }
    } else {
        collide_interior(a, por0, d);
        collide_interior(b, por1, d);
    }

    // ---- store --------------------------------------------------------------
    // Only the results of cells whose pair is interior (mine) are stored; a
    // store that combines this lane's cell with the neighbouring lane's
    // (odd steps, x-shifted links) writes each half only for its own pair.
    if (PAR == 0) {
        if (mine) {
#pragma unroll
            for (int q = 0; q < 9; ++q) ST::stf2(P + opp(q) * np + row + x, a[q], b[q], d);
#pragma unroll
            for (int i = 1; i <= 4; ++i) ST::stT2(P + (8 + opp(i)) * np + row + x, a[8 + i], b[8 + i], d);
        }
    } else {
        const bool left_ok = (MASK ? __shfl_up_sync(0xffffffffu, mine, 1) != 0 : true) && lane != 0;
        const bool right_ok = (MASK ? __shfl_down_sync(0xffffffffu, mine, 1) != 0 : true) && lane != 31;
        if (mine) ST::stf2(P + row + x, a[0], b[0], d);
#pragma unroll
        for (int k = 1; k < 13; ++k) {
            const bool heat = k > 8;
            const int i = heat ? k - 8 : k;
            const int pl = heat ? 8 + i : i;           // f*_i(x) goes to slot (x + e_i, i)
            const int dr = ey(i) == 1 ? rowu : (ey(i) == -1 ? rowd : row);
            T* dst = P + pl * np + dr;
            if (ex(i) == 0) {
                if (mine) {
                    if (heat) ST::stT2(dst + x, a[k], b[k], d);
                    else ST::stf2(dst + x, a[k], b[k], d);
                }
            } else if (ex(i) == 1) {  // destination columns x+1, x+2
                const float left = __shfl_up_sync(0xffffffffu, b[k], 1);
                if (mine && left_ok) {
                    if (heat) ST::stT2(dst + x, left, a[k], d);
                    else ST::stf2(dst + x, left, a[k], d);
                } else {
                    if (mine) {
                        if (heat) ST::stT(dst + x + 1, a[k], d);
                        else ST::stf(dst + x + 1, a[k], d);
                    }
                    if (left_ok) {
                        if (heat) ST::stT(dst + x, left, d);
                        else ST::stf(dst + x, left, d);
                    }
                }
                if (lane == 31 && mine) {
                    if (heat) ST::stT(dst + xr, b[k], d);
                    else ST::stf(dst + xr, b[k], d);
                }
            } else {                  // destination columns x-1, x
                const float right = __shfl_down_sync(0xffffffffu, a[k], 1);
                if (mine && right_ok) {
                    if (heat) ST::stT2(dst + x, b[k], right, d);
                    else ST::stf2(dst + x, b[k], right, d);
                } else {
                    if (mine) {
                        if (heat) ST::stT(dst + x, b[k], d);
                        else ST::stf(dst + x, b[k], d);
                    }
                    if (right_ok) {
                        if (heat) ST::stT(dst + x + 1, right, d);
                        else ST::stf(dst + x + 1, right, d);
                    }
                }
                if (lane == 0 && mine) {
                    if (heat) ST::stT(dst + xl, a[k], d);
                    else ST::stf(dst + xl, a[k], d);
                }
            }
        }
    }
}

// Observables of an interior cell pair before its collision (the observing
// check step of the steady-state loop): mass, peak |u|^2, pressure sum and
// count over fluid cells, NaN count, residual against and update of the
// velocity snapshot.  Interior cells have no wall, inlet or outlet link, so
// they add nothing to the wall shear stress or the fluxes.  Same definitions
// as cell_body (Eq. 9), evaluated in the pair path's FP32 arithmetic.  The
// two cells are combined first (a sum of two values, a maximum, a count) and
// enter the partials (type A) once per pair: GB300's FP64 pipe is narrow, and
// per-cell FP64 updates made this step FP64-bound.
template <class ST, class A>
__device__ __forceinline__ void pair_observe(const InstDesc& d, int x, int y, const float* a,
                                             const float* b, uint32_t m2, int mode, A* acc) {
    const int np = (int)d.npad;
    const int c = y * d.nx + x;
    float ux2[2], uy2[2], mass = 0.0f, psum = 0.0f, pk = 0.0f;
    int nfl = 0;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float* f = j == 0 ? a : b;
        const float ux = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
        const float uy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
        const float usq = ux * ux + uy * uy;
        const float S0 = float(K_W0) * (-1.5f * usq);
        const float sum18 = f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
        const float p = (sum18 + S0) * 0.6f;
        ux2[j] = ux;
        uy2[j] = uy;
        mass += sum18;
        pk = fmaxf(pk, usq);
        if (((m2 >> (8 * j)) & TYPE_BITS) == FLUID) {
            psum += p;
            ++nfl;
            bad = bad || !isfinite(p);
        }
    }
    if (mode & OBS_STATS) {
        acc[P_MASS] += (A)mass;
        acc[P_PEAK] = amax(acc[P_PEAK], (A)pk);
        acc[P_SUM_P] += (A)psum;
        acc[P_N_FLUID] += (A)nfl;
        if (bad) acc[P_NAN] += A(1);
    }
    if (mode & (OBS_RESID | OBS_SNAP)) {
        float* U = static_cast<float*>(d.usnap);
        if ((mode & OBS_RESID) && d.snap_valid) {
            float r2 = 0.0f;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float dx = ux2[j] - U[c + j];
                const float dy = uy2[j] - U[np + c + j];
                r2 = fmaxf(r2, dx * dx + dy * dy);
            }
            acc[P_RESID] = amax(acc[P_RESID], (A)r2);
        }
        if (mode & OBS_SNAP) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                U[c + j] = ux2[j];
                U[np + c + j] = uy2[j];
            }
        }
    }
}

template <class ST, int PAR, bool OBS = false, class A = double, bool MASK = false>
__device__ __forceinline__ void update_pair_interior(const InstDesc& d, int x, int y, bool por0,
                                                     bool por1, uint32_t m2 = 0, int mode = 0,
                                                     A* acc = nullptr, bool mine = true) {
    using T = typename ST::T;
    const int nx = d.nx, ny = d.ny;
    const int np = (int)d.npad;
    T* const P = static_cast<T*>(d.pops);
    const int lane = threadIdx.x & 31;
    const int row = y * nx;
    const int rowu = (y == ny - 1 ? 0 : y + 1) * nx;
    const int rowd = (y == 0 ? ny - 1 : y - 1) * nx;
    const int xl = x == 0 ? nx - 1 : x - 1;     // column left of the pair
    const int xr = x + 2 == nx ? 0 : x + 2;     // column right of the pair
    float a[13], b[13];                          // cells x and x+1; 9..12 = T_1..T_4

    // ---- load ---------------------------------------------------------------
    if (PAR == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float2 v = ST::ldf2(P + q * np + row + x, d);
            a[q] = v.x;
            b[q] = v.y;
        }
#pragma unroll
        for (int i = 1; i <= 4; ++i) {
            const float2 v = ST::ldT2(P + (8 + i) * np + row + x, d);
            a[8 + i] = v.x;
            b[8 + i] = v.y;
        }
    } else {
        {
            const float2 v = ST::ldf2(P + row + x, d);
            a[0] = v.x;
            b[0] = v.y;
        }
#pragma unroll
        for (int k = 1; k < 13; ++k) {
            const bool heat = k > 8;
            const int i = heat ? k - 8 : k;            // lattice direction
            const int pl = heat ? 8 + opp(i) : opp(i); // f_i(x) sits in slot (x - e_i, opp(i))
            const int sr = ey(i) == 1 ? rowd : (ey(i) == -1 ? rowu : row);
            const T* src = P + pl * np + sr;
            const float2 v = heat ? ST::ldT2(src + x, d) : ST::ldf2(src + x, d);
            if (ex(i) == 0) {
                a[k] = v.x;
                b[k] = v.y;
            } else if (ex(i) == 1) {  // source columns x-1, x
                float left = __shfl_up_sync(0xffffffffu, v.y, 1);
                if (lane == 0) left = heat ? ST::ldT(src + xl, d) : ST::ldf(src + xl, d);
                a[k] = left;
                b[k] = v.x;
            } else {                  // source columns x+1, x+2
                float right = __shfl_down_sync(0xffffffffu, v.x, 1);
                if (lane == 31) right = heat ? ST::ldT(src + xr, d) : ST::ldf(src + xr, d);
                a[k] = v.y;
                b[k] = right;
            }
        }
    }

    if constexpr (OBS) {
        if (!MASK || mine) pair_observe<ST, A>(d, x, y, a, b, m2, mode, acc);
    }
    pair_collide_store<ST, PAR, MASK>(d, x, y, a, b, por0, por1, mine);
}

// ---------------------------------------------------------------------------
// Interior path of the 16-bit storages on 256-cell tile rows: one lane updates
// eight neighbouring cells x0 .. x0 + 7 (x0 a multiple of 8), and every plane
// moves as one 16-byte vector of eight packed 16-bit codes, i.e. 13 vector
// loads and 13 vector stores per eight cells.  The codes stay packed in
// registers (w[plane][word], two codes per 32-bit word, the lower column in
// the low half), and the two cells of a word are decoded, collided and
// encoded together, their results replacing the word they came from, so only
// two cells' 13 values are live as FP32 at a time.  On an odd step the
// x-shifted links are assembled from the neighbouring lane's words (one
// shuffle per plane and __byte_perm), and the warp's first and last lanes
// load or store the one code outside the warp's 256 cells.  Same model and
// operations as the pair path (collide_interior), run on the values as
// stored: the flow populations with their power-of-two scale (the same
// rounding as unscaled), the heat deviations in code units, so that decoding
// and encoding are bare conversions (and the heat codes' clamp of the knee).

// the code pair (b of lo, a of hi): word whose low half is the high half of
// lo and whose high half is the low half of hi (a one-code shift)
__device__ __forceinline__ uint32_t shift_pair(uint32_t lo, uint32_t hi) { return __byte_perm(lo, hi, 0x5432); }

// NW packed 32-bit words (2 NW cells) per plane and lane: one 16-byte (NW = 4)
// or 8-byte (NW = 2) vector access
template <int NW>
__device__ __forceinline__ void ld_words(const void* p, uint32_t* w) {
    if constexpr (NW == 4) {
        const uint4 v = __ldcg(reinterpret_cast<const uint4*>(p));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else {
        const uint2 v = __ldcg(reinterpret_cast<const uint2*>(p));
        w[0] = v.x; w[1] = v.y;
    }
}
template <int POL, int NW>
__device__ __forceinline__ void st_words(void* p, const uint32_t* w) {
    if constexpr (NW == 4) st_pol<POL>(reinterpret_cast<uint4*>(p), make_uint4(w[0], w[1], w[2], w[3]));
    else st_pol<POL>(reinterpret_cast<uint2*>(p), make_uint2(w[0], w[1]));
}

template <class ST, int PAR, int NW>
__device__ __forceinline__ void update_vec16_interior(const InstDesc& d, int x0, int y, uint32_t por) {
    using T = typename ST::T;
    static_assert(sizeof(T) == 2, "16-bit storages only");
    static_assert(NW == 2 || NW == 4, "8-byte or 16-byte vectors");
    constexpr int POL = ST::kPol;
    constexpr int C = 2 * NW;  // cells per lane
    const int nx = d.nx, ny = d.ny;
    const int np = (int)d.npad;
    T* const P = static_cast<T*>(d.pops);
    const int lane = threadIdx.x & 31;
    const int row = y * nx;
    const int rowu = (y == ny - 1 ? 0 : y + 1) * nx;
    const int rowd = (y == 0 ? ny - 1 : y - 1) * nx;
    const int xl = x0 == 0 ? nx - 1 : x0 - 1;  // column left of the lane's cells
    const int xr = x0 + C == nx ? 0 : x0 + C;  // column right of them
    uint32_t w[13][NW];

    // ---- load -------------------------------------------------------------
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        if (PAR == 0 || k == 0) {
            ld_words<NW>(P + k * np + row + x0, w[k]);
        } else {
            const bool heat = k > 8;
            const int i = heat ? k - 8 : k;             // lattice direction
            const int pl = heat ? 8 + opp(i) : opp(i);  // f_i(x) sits in slot (x - e_i, opp(i))
            const int sr = ey(i) == 1 ? rowd : (ey(i) == -1 ? rowu : row);
            const T* src = P + pl * np + sr;
            uint32_t v[NW];
            ld_words<NW>(src + x0, v);
            if (ex(i) == 0) {
#pragma unroll
                for (int j = 0; j < NW; ++j) w[k][j] = v[j];
            } else if (ex(i) == 1) {  // source columns x0 - 1 .. x0 + C - 2
                uint32_t prev = __shfl_up_sync(0xffffffffu, v[NW - 1], 1);
                if (lane == 0) prev = (uint32_t)__ldcg(reinterpret_cast<const unsigned short*>(src + xl)) << 16;
                w[k][0] = shift_pair(prev, v[0]);
#pragma unroll
                for (int j = 1; j < NW; ++j) w[k][j] = shift_pair(v[j - 1], v[j]);
            } else {                  // source columns x0 + 1 .. x0 + C
                uint32_t next = __shfl_down_sync(0xffffffffu, v[0], 1);
                if (lane == 31) next = (uint32_t)__ldcg(reinterpret_cast<const unsigned short*>(src + xr));
#pragma unroll
                for (int j = 0; j < NW - 1; ++j) w[k][j] = shift_pair(v[j], v[j + 1]);
                w[k][NW - 1] = shift_pair(v[NW - 1], next);
            }
        }
    }

    // ---- collide, two cells (one packed word per plane) at a time -----------
    // w[k] holds the inputs of direction k (even step: slot k = plane k; odd
    // step: assembled from plane opp(k)); the result of direction k goes to
    // plane opp(k) of the cells' own columns on an even step and to plane k,
    // shifted by e_k, on an odd step.  Each pass takes word 0 of every plane
    // (two cells) and moves the result word to the back, so after NW passes
    // every plane's words are the results in their own places.  The pass loop
    // is not unrolled: every register index stays static, and the body (two
    // inlined collisions) stays small enough for the instruction cache.
#pragma unroll 1
    for (int q = 0; q < NW; ++q) {
        float2 v[13];
        // flow values as stored (scaled by 2^kLog2S), heat in code units
#pragma unroll
        for (int k = 0; k < 9; ++k) v[k] = ST::decf2_raw(w[k][0]);
#pragma unroll
        for (int k = 9; k < 13; ++k) v[k] = dec_tcode2(w[k][0]);
        collide_interior2<ST::kLog2S, true>(v, (por >> (2 * q)) & 3u, d);
        uint32_t o[13];
#pragma unroll
        for (int k = 0; k < 13; ++k) {
            const int dst = PAR == 0 ? (k < 9 ? opp(k) : 8 + opp(k - 8)) : k;
            o[dst] = k < 9 ? ST::encf2_raw(v[k].x, v[k].y) : enc_tcode2(v[k].x, v[k].y);
        }
#pragma unroll
        for (int k = 0; k < 13; ++k) {
#pragma unroll
            for (int j = 0; j < NW - 1; ++j) w[k][j] = w[k][j + 1];
            w[k][NW - 1] = o[k];
        }
    }

    // ---- store ------------------------------------------------------------
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        if (PAR == 0 || k == 0) {
            st_words<POL, NW>(P + k * np + row + x0, w[k]);
            continue;
        }
        const bool heat = k > 8;
        const int i = heat ? k - 8 : k;
        const int dr = ey(i) == 1 ? rowu : (ey(i) == -1 ? rowd : row);  // f*_i(x) goes to slot (x + e_i, i)
        T* const dst = P + k * np + dr;
        if (ex(i) == 0) {
            st_words<POL, NW>(dst + x0, w[k]);
        } else if (ex(i) == 1) {  // destination columns x0 + 1 .. x0 + C
            const uint32_t prev = __shfl_up_sync(0xffffffffu, w[k][NW - 1], 1);
            uint32_t o[NW];
            o[0] = shift_pair(prev, w[k][0]);
#pragma unroll
            for (int j = 1; j < NW; ++j) o[j] = shift_pair(w[k][j - 1], w[k][j]);
            if (lane != 0) {
                st_words<POL, NW>(dst + x0, o);
            } else {  // column x0 belongs to the cell left of the warp
                st_pol<POL>(reinterpret_cast<unsigned short*>(dst + x0 + 1), (unsigned short)(o[0] >> 16));
                st_pol<POL>(reinterpret_cast<unsigned int*>(dst + x0 + 2), o[1]);
                if constexpr (NW == 4) st_pol<POL>(reinterpret_cast<uint2*>(dst + x0 + 4), make_uint2(o[2], o[3]));
            }
            if (lane == 31)
                st_pol<POL>(reinterpret_cast<unsigned short*>(dst + xr), (unsigned short)(w[k][NW - 1] >> 16));
        } else {                  // destination columns x0 - 1 .. x0 + C - 2
            const uint32_t next = __shfl_down_sync(0xffffffffu, w[k][0], 1);
            uint32_t o[NW];
#pragma unroll
            for (int j = 0; j < NW - 1; ++j) o[j] = shift_pair(w[k][j], w[k][j + 1]);
            o[NW - 1] = shift_pair(w[k][NW - 1], next);
            if (lane != 31) {
                st_words<POL, NW>(dst + x0, o);
            } else {  // column x0 + C - 1 belongs to the cell right of the warp
                if constexpr (NW == 4) {
                    st_pol<POL>(reinterpret_cast<uint2*>(dst + x0), make_uint2(o[0], o[1]));
                    st_pol<POL>(reinterpret_cast<unsigned int*>(dst + x0 + 4), o[2]);
                    st_pol<POL>(reinterpret_cast<unsigned short*>(dst + x0 + 6), (unsigned short)(o[3] & 0xFFFFu));
                } else {
                    st_pol<POL>(reinterpret_cast<unsigned int*>(dst + x0), o[0]);
                    st_pol<POL>(reinterpret_cast<unsigned short*>(dst + x0 + 2), (unsigned short)(o[1] & 0xFFFFu));
                }
            }
            if (lane == 0)
                st_pol<POL>(reinterpret_cast<unsigned short*>(dst + xl), (unsigned short)(w[k][0] & 0xFFFFu));
        }
    }
}

// The masked pair row is rare (rows next to a boundary) and is called out of
// line: its registers are then allocated apart from the interior pair path's.
template <class ST, int PAR, bool OBS, class A>
__device__ __noinline__ void pair_row_masked(const InstDesc& sd, int x, int y, bool por0, bool por1, uint32_t m2,
                                             int mode, A* acc, bool mine) {
    update_pair_interior<ST, PAR, OBS, A, true>(sd, x, y, por0, por1, m2, mode, acc, mine);
}

// The per-cell update of a pair of a plain step's row without the pair path
// (rare: grids of odd width, tiles 32 wide), out of line.
template <class ST, int PAR>
__device__ __noinline__ void cell_pair_slow(const InstDesc& sd, int x, int y) {
    if (x < sd.nx && y < sd.ny) update_cell<ST, false, PAR, double>(sd, x, y, 0, nullptr);
    if (x + 1 < sd.nx && y < sd.ny) update_cell<ST, false, PAR, double>(sd, x + 1, y, 0, nullptr);
}

// One row of cell pairs (x, x + 1) of a warp that covers a 64-cell segment.
// With the pair path (vec_ok), a segment whose pairs are all interior (both
// cells fluid or porous, not next to a boundary) takes it.  Otherwise:
// - an instance that takes edge-cell chunks (SPLIT kernels, sd.split): the
//   interior pairs of a segment that lies wholly in the grid take the pair
//   path, the warp's other lanes taking part in its loads and shuffles but
//   storing nothing; its other cells are edge cells, updated elsewhere;
// - else every cell of the segment takes the per-cell update.
template <class ST, bool OBS, int PAR, class A, bool SPLIT>
__device__ __forceinline__ void pair_row(const InstDesc& sd, int x, int y, bool pure, bool vec_ok, int mode,
                                         A* acc) {
    bool split = SPLIT;
    if constexpr (SPLIT && sizeof(typename ST::T) == 4) split = sd.split != 0;
    bool fast = false;
    if (vec_ok) {
        uint32_t m2 = 0u;
        if (pure) {
            fast = true;
        } else {
            const bool in = y < sd.ny && x + 1 < sd.nx;
            if (in) m2 = *reinterpret_cast<const uint16_t*>(sd.mask + (int64_t)y * sd.nx + x);
            else m2 = 0xFFFFu;
            // both cells fluid or porous (type bits 1-2 clear) and not next to a boundary (bit 3)
            const bool mine = (m2 & 0x0E0Eu) == 0u;
            fast = __all_sync(0xffffffffu, mine);
            if constexpr (SPLIT) {
                // every lane in the grid: the segment lies wholly in it
                if (!fast && split && __all_sync(0xffffffffu, in) && __any_sync(0xffffffffu, mine))
                    pair_row_masked<ST, PAR, OBS, A>(sd, x, y, (m2 & 1u) != 0 && sd.tm_model == 0,
                                                     (m2 & 0x100u) != 0 && sd.tm_model == 0, m2, mode, acc, mine);
            }
        }
        if (fast)
            update_pair_interior<ST, PAR, OBS, A>(sd, x, y, (m2 & 1u) != 0 && sd.tm_model == 0,
                                                  (m2 & 0x100u) != 0 && sd.tm_model == 0, m2, mode, acc);
    }
    if (!fast && !(split && vec_ok)) {
        if constexpr (SPLIT) {
            cell_pair_slow<ST, PAR>(sd, x, y);
        } else {
            if (x < sd.nx && y < sd.ny) update_cell<ST, OBS, PAR, A>(sd, x, y, mode, acc);
            if (x + 1 < sd.nx && y < sd.ny) update_cell<ST, OBS, PAR, A>(sd, x + 1, y, mode, acc);
        }
    }
}

// The edge cells of one tile (the dataflow kernel, after the tile's rows):
// one per thread of the block, through the per-cell update.  Out of line, so
// that its registers are allocated apart from the rows'.
template <class ST, int PAR>
__device__ __noinline__ void tile_edge_cells(const InstDesc& sd, int li) {
    if (li < 0 || li >= sd.ntiles) return;  // not a tile of this instance
    const int e1 = sd.eoff[li + 1];
    const int nthreads = blockDim.x * blockDim.y;
    for (int e = sd.eoff[li] + (int)(threadIdx.y * blockDim.x + threadIdx.x); e < e1; e += nthreads) {
        const int c = sd.edges[e];
        const int y = c / sd.nx;
        update_cell<ST, false, PAR, double>(sd, c - y * sd.nx, y, 0, nullptr, sd.etypes[e]);
    }
}

// An edge-cell chunk {instance, TILE_EDGE, first, count}: one edge cell per
// thread of the block, through the per-cell update (a plain step).
template <class ST, int PAR>
__device__ __noinline__ void edge_block(const InstDesc& sd, int4 te) {
    const int k = (int)(threadIdx.y * blockDim.x + threadIdx.x);
    if (k < te.w) {
        const int c = sd.edges[te.z + k];
        const int y = c / sd.nx;
        update_cell<ST, false, PAR, double>(sd, c - y * sd.nx, y, 0, nullptr, sd.etypes[te.z + k]);
    }
}

// SPLIT: a plain step whose edge cells come in chunks of their own (pair_row)
template <class ST, bool OBS, int PAR, class A = double, bool SPLIT = false>
__device__ __forceinline__ void tile_rows(const InstDesc& sd, const int4& te, int mode, const Shape& shape,
                                          A* acc) {
    const int rpt = shape.rpt;
    if constexpr (sizeof(typename ST::R) == 4) {
        // the pair path needs whole warps on one row and even rows; an
        // observing step takes it too when it also writes (the steady-state
        // check), while observe-only reads stay on the per-cell path
        const bool vec_ok = (!OBS || (mode & OBS_WRITE)) && (blockDim.x & 31) == 0 && (sd.nx & 1) == 0;
        // a pure tile (every cell fluid, in the grid, away from boundaries)
        // takes the pair path without reading its mask
        const bool pure = (te.y & TILE_PURE) != 0;
        const int V16 = sizeof(typename ST::T) == 2 ? vec16_cells(shape.tw) : 0;
        if (V16 > 0) {
            // 16-bit storage, V16 = 8 or 4 cells per lane (blockDim.x == 32):
            // plain steps of rows whose 32 V16 cells are all interior take the
            // vector path; the others, and observing steps, take V16 / 2
            // 64-cell pair rows
            const int x0 = te.z + V16 * threadIdx.x;
            const bool v16_ok = !OBS && (sd.nx % (V16 > 0 ? V16 : 1)) == 0;
            for (int r = 0; r < rpt; ++r) {
                const int y = te.w + threadIdx.y + r * blockDim.y;
                bool fast = false;
                uint32_t por = 0u;
                if constexpr (!OBS && sizeof(typename ST::T) == 2) {
                    if (v16_ok) {
                        if (pure) {
                            fast = true;
                        } else {
                            uint64_t m8 = ~0ull;
                            const int64_t mo = (int64_t)y * sd.nx + x0;
                            if (y < sd.ny && x0 + V16 <= sd.nx)
                                m8 = V16 == 8 ? __ldg(reinterpret_cast<const unsigned long long*>(sd.mask + mo))
                                              : (uint64_t)__ldg(reinterpret_cast<const unsigned int*>(sd.mask + mo));
                            const uint64_t busy = V16 == 8 ? 0x0E0E0E0E0E0E0E0Eull : 0x0E0E0E0Eull;
                            fast = __all_sync(0xffffffffu, (m8 & busy) == 0ull);
                            if (sd.tm_model == 0)
#pragma unroll
                                for (int j = 0; j < 8; ++j) por |= (uint32_t)((m8 >> (8 * j)) & 1u) << j;
                        }
                        if (fast) {
                            if (V16 == 8) update_vec16_interior<ST, PAR, 4>(sd, x0, y, por);
                            else update_vec16_interior<ST, PAR, 2>(sd, x0, y, por);
                        }
                    }
                }
                if (!fast) {
#pragma unroll 1
                    for (int s = 0; s < V16 / 2; ++s)
                        pair_row<ST, OBS, PAR, A, SPLIT>(sd, te.z + 64 * s + 2 * (int)threadIdx.x, y, pure, vec_ok, mode, acc);
                }
            }
        } else {
            const int x = te.z + 2 * threadIdx.x;
            for (int r = 0; r < rpt; ++r) {
                const int y = te.w + threadIdx.y + r * blockDim.y;
                pair_row<ST, OBS, PAR, A, SPLIT>(sd, x, y, pure, vec_ok, mode, acc);
            }
        }
    } else {
        const int x = te.z + threadIdx.x;
        for (int r = 0; r < rpt; ++r) {
            const int y = te.w + threadIdx.y + r * blockDim.y;
            if (x < sd.nx && y < sd.ny) update_cell<ST, OBS, PAR, A>(sd, x, y, mode, acc);
        }
    }
}

// ---------------------------------------------------------------------------
// Staged step of the FP32-arithmetic kernels (launch shapes with one row of
// threads per block and tiles at least 64 cells wide): every warp runs its
// own copy pipeline through shared memory.
//
// The unit of work is a row segment: 64 cells of one row of a tile (32 cell
// pairs, one per lane).  The segments of the block's tiles (blockIdx.x,
// + gridDim.x, ...) are numbered tile by tile, row by row; warp w takes
// segments w, w + WS_WARPS, w + 2 WS_WARPS, ...  Each warp keeps WS_DEPTH
// shared-memory stages.  For a segment it stages what the segment's cells
// read with bulk copies that complete on the stage's barrier: on an even step
// the cells' own slots of all 13 planes (one bulk tensor copy,
// cp.async.bulk.tensor), on an odd step the x-shifted links' sources, plane p
// from row y + ey(p) and widened by a 16-byte halo on both sides (one
// cp.async.bulk per plane), and for tiles that are not pure the mask row.  It then waits for its oldest stage, updates
// that segment's pairs from shared memory, stores them in the AA pattern to
// global memory, and refills the stage with the segment WS_DEPTH ahead.  So
// WS_DEPTH segments per warp are in flight while it computes, no register
// waits on a load, and a warp held up by boundary cells delays only itself.
//
// Each slot is read and written in a step only by the cell that owns it, so
// staging later segments before earlier segments' stores land is exact; halo
// and out-of-grid elements are copied (or zero-filled) but never used.
// Whole-warp interior segments take the pair path's collision and stores;
// other active cells take cell_body with the staged populations; pairs at a
// periodic edge (whose wrap-around column is not staged) and instances whose
// rows are not 16-byte aligned take the direct path.  Every barrier wait is
// bounded: an expired wait sets the device status word, the warp waits
// (bounded) for the copies it may still have in flight and leaves, and the
// host reports the error instead of hanging.

#ifndef LBM_WS_WARPS
#define LBM_WS_WARPS 8
#endif
#ifndef LBM_WS_DEPTH
#define LBM_WS_DEPTH 3
#endif
#ifndef LBM_WS_MINB
#define LBM_WS_MINB 2
#endif
constexpr int WS_SEG = 64;               // cells per segment (32 pairs: one warp)
constexpr int WS_WARPS = LBM_WS_WARPS;   // warps per block
constexpr int WS_DEPTH = LBM_WS_DEPTH;   // stages per warp
constexpr int WS_THREADS = 32 * WS_WARPS;
constexpr uint32_t TMA_WAIT_LIMIT = 1u << 22;

// elements per 16-byte chunk
template <class T>
__host__ __device__ constexpr int chunk_elems() { return 16 / (int)sizeof(T); }

// Stage layout, in elements of T from the stage base (128-byte aligned, as
// bulk tensor copies need).  Even step: plane p's 64 cells at p * 64.  Odd
// step: plane p's row piece at p * ws_odd_pe (the segment and a 16-byte chunk
// of halo on both sides).  The mask row follows the odd layout.
__host__ __device__ constexpr int ws_align128(int b) { return (b + 127) / 128 * 128; }
template <class T>
__host__ __device__ constexpr int ws_odd_pe() { return WS_SEG + 2 * chunk_elems<T>(); }
template <class T, int PAR>
__host__ __device__ constexpr int ws_plane_off(int p) { return p * (PAR == 0 ? WS_SEG : ws_odd_pe<T>()); }
template <class T>
__host__ __device__ constexpr int ws_mask_off() { return 13 * ws_odd_pe<T>() * (int)sizeof(T); }
template <class T>
__host__ __device__ constexpr int ws_stage_bytes() { return ws_align128(ws_mask_off<T>() + WS_SEG); }
// dynamic shared memory of a block (and room to align the ring)
template <class T>
__host__ __device__ constexpr int ws_smem_bytes() { return WS_WARPS * WS_DEPTH * ws_stage_bytes<T>() + 128; }
static_assert(ws_mask_off<float>() % 16 == 0 && ws_mask_off<__half>() % 16 == 0, "stage layout");

// What a stage holds, written by the producer before it arrives on the
// stage's full barrier.
struct WsMeta {
    int inst, flags, x, y;  // instance, WS_* flags, segment origin
};
enum : int {
    WS_PURE = 1,    // pure tile: every cell an interior fluid cell, no mask needed
    WS_MASK = 2,    // the mask row is staged after the planes
    WS_DIRECT = 4,  // nothing staged: the warp takes the direct path
    WS_SKIP = 8,    // segment outside the grid: nothing to do
    WS_END = 16     // no more segments for this warp
};

// Non-zero after a staged wait expired; read and cleared by the host
// (take_step_status).  Only the FP32-arithmetic unit instantiates the staged
// kernel, so its copy of this word is the one that is used.
static __device__ int g_step_status = 0;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < TMA_WAIT_LIMIT; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// source row of plane p for target row y on an odd step: f_i(x) sits in slot
// (x - e_i, opp(i)), i.e. plane p = opp(i) holds it at row y - ey(i) = y + ey(p)
__device__ __forceinline__ constexpr int plane_dir(int p) { return p < 9 ? p : p - 8; }

// Populations of the cell pair at segment column c (cells c, c + 1): own
// slots on an even step, the x-shifted links' sources on an odd step.
template <class ST, int PAR>
__device__ __forceinline__ void ws_load(const InstDesc& d, const typename ST::T* stage, int c, float* a,
                                        float* b) {
    using T = typename ST::T;
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        const bool heat = k > 8;
        const int i = heat ? k - 8 : k;
        const int pl = PAR == 0 ? k : (heat ? 8 + opp(i) : opp(i));
        const int col = PAR == 0 ? c : c + chunk_elems<T>() - ex(i);
        const T* src = stage + ws_plane_off<T, PAR>(pl) + col;
        a[k] = heat ? ST::sldT(src, d) : ST::sldf(src, d);
        b[k] = heat ? ST::sldT(src + 1, d) : ST::sldf(src + 1, d);
    }
}

// AA-pattern stores of a collided interior pair by one lane on its own (no
// shuffles: the lanes of a warp need not all take this path).
template <class ST, int PAR>
__device__ __forceinline__ void pair_store_lane(const InstDesc& d, int x, int y, const float* a,
                                                const float* b) {
    using T = typename ST::T;
    T* const P = static_cast<T*>(d.pops);
    const int np = (int)d.npad;
    const int nx = d.nx, ny = d.ny;
    const int row = y * nx;
    if (PAR == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) ST::stf2(P + opp(q) * np + row + x, a[q], b[q], d);
#pragma unroll
        for (int i = 1; i <= 4; ++i) ST::stT2(P + (8 + opp(i)) * np + row + x, a[8 + i], b[8 + i], d);
    } else {
        const int rowu = (y == ny - 1 ? 0 : y + 1) * nx;
        const int rowd = (y == 0 ? ny - 1 : y - 1) * nx;
        ST::stf2(P + row + x, a[0], b[0], d);
#pragma unroll
        for (int k = 1; k < 13; ++k) {
            const bool heat = k > 8;
            const int i = heat ? k - 8 : k;
            const int pl = heat ? 8 + i : i;  // f*_i(x) goes to slot (x + e_i, i)
            const int dr = ey(i) == 1 ? rowu : (ey(i) == -1 ? rowd : row);
            T* dst = P + pl * np + dr + x;
            if (ex(i) == 0) {
                if (heat) ST::stT2(dst, a[k], b[k], d);
                else ST::stf2(dst, a[k], b[k], d);
            } else {
                const int o = ex(i);
                if (heat) {
                    ST::stT(dst + o, a[k], d);
                    ST::stT(dst + 1 + o, b[k], d);
                } else {
                    ST::stf(dst + o, a[k], d);
                    ST::stf(dst + 1 + o, b[k], d);
                }
            }
        }
    }
}

// One warp's staged segment: lane l updates cells x = m.x + 2 l, x + 1.
template <class ST, int PAR>
__device__ __forceinline__ void ws_segment(const InstDesc& d, const typename ST::T* stage,
                                           const unsigned char* smask, const WsMeta& m) {
    const int lane = threadIdx.x & 31;
    const int nx = d.nx;
    const int c = 2 * lane;  // column of cell x in the segment
    const int x = m.x + c, y = m.y;
    if (m.flags & WS_DIRECT) {
        if (x < nx) update_cell<ST, false, PAR, double>(d, x, y, 0, nullptr);
        if (x + 1 < nx) update_cell<ST, false, PAR, double>(d, x + 1, y, 0, nullptr);
        return;
    }
    // a staged instance has nx a multiple of the 16-byte chunk, hence even:
    // x < nx implies x + 1 < nx
    const bool in = x < nx;
    uint32_t m2 = 0xFFFFu;
    if (m.flags & WS_PURE) m2 = 0u;
    else if (in)
        m2 = (m.flags & WS_MASK) ? *reinterpret_cast<const uint16_t*>(smask + c)
                                 : *reinterpret_cast<const uint16_t*>(d.mask + (int64_t)y * nx + x);
    const bool edge = x == 0 || x + 2 >= nx;
    // both cells fluid or porous (type bits 1-2 clear), not next to a boundary (bit 3)
    const bool interior = in && !edge && (m2 & 0x0E0Eu) == 0u;
    const bool por0 = (m2 & 1u) != 0 && d.tm_model == 0;
    const bool por1 = (m2 & 0x100u) != 0 && d.tm_model == 0;
    float a[13], b[13];
    if (__all_sync(0xffffffffu, interior)) {
        ws_load<ST, PAR>(d, stage, c, a, b);
        pair_collide_store<ST, PAR>(d, x, y, a, b, por0, por1);
        return;
    }
    if (!in) return;
    if ((m2 & TYPE_BITS) > POROUS && ((m2 >> 8) & TYPE_BITS) > POROUS) return;  // neither cell active
    if (edge) {
        update_cell<ST, false, PAR, double>(d, x, y, 0, nullptr);
        update_cell<ST, false, PAR, double>(d, x + 1, y, 0, nullptr);
        return;
    }
    ws_load<ST, PAR>(d, stage, c, a, b);
    if (interior) {
        collide_interior(a, por0, d);
        collide_interior(b, por1, d);
        pair_store_lane<ST, PAR>(d, x, y, a, b);
        return;
    }
    // at least one cell next to a boundary: general update of each cell
#pragma unroll 1
    for (int v = 0; v < 2; ++v) {
        const float* c = v == 0 ? a : b;
        float f[9], g[4];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = c[i];
#pragma unroll
        for (int i = 0; i < 4; ++i) g[i] = c[9 + i];
        cell_body<ST, false, PAR, double>(d, x + v, y, f, g, (uint8_t)(m2 >> (8 * v)), 0, nullptr);
    }
}

__device__ __forceinline__ void warp_copy_desc(InstDesc* dst, const InstDesc* src) {
    const uint64_t* s = reinterpret_cast<const uint64_t*>(src);
    uint64_t* o = reinterpret_cast<uint64_t*>(dst);
    __syncwarp();
    for (int k = threadIdx.x & 31; k < (int)(sizeof(InstDesc) / 8); k += 32) o[k] = s[k];
    __syncwarp();
}

__device__ __forceinline__ void bulk_tensor_load(void* dst, const void* map, int x, int y, int z,
                                                 uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];\n" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Posts one segment (or the end marker) into stage `st` of the calling warp,
// completing on barrier `bar`.  te is the segment's tile entry (read ahead by
// the caller), r and sx its row and segment in the tile; idesc holds the
// descriptor of the instance last posted (refreshed here when it changes).
// On an even step every plane is read at row y, and with the instance's
// tensor map one bulk tensor copy (64 x 1 x 13 planes) stages them all.  On
// an odd step (or without a map) lanes 0-12 copy one plane's row piece each
// (plane p from row y + ey(p), widened by a 16-byte halo on both sides).
// Lane 13 copies the mask row of a tile that is not pure.
template <class ST>
__device__ __forceinline__ void ws_post(const InstDesc* __restrict__ insts, InstDesc& idesc, int& iheld,
                                        const int4& te, bool valid, int r, int sx, int flip,
                                        unsigned char* st, WsMeta& meta, uint64_t* bar) {
    using T = typename ST::T;
    constexpr int CHE = chunk_elems<T>();
    constexpr int ES = (int)sizeof(T);
    const int lane = threadIdx.x & 31;
    if (!valid) {
        if (lane == 0) {
            meta = WsMeta{-1, WS_END, 0, 0};
            mbar_arrive(bar);
        }
        return;
    }
    if (te.x != iheld) {
        warp_copy_desc(&idesc, insts + te.x);
        iheld = te.x;
    }
    const int nx = idesc.nx, ny = idesc.ny;
    const int y = te.w + r, xs = te.z + sx * WS_SEG;
    if (y >= ny || xs >= nx) {
        if (lane == 0) {
            meta = WsMeta{te.x, WS_SKIP, xs, y};
            mbar_arrive(bar);
        }
        return;
    }
    const bool staged = (nx % CHE) == 0;  // plane rows start on 16-byte boundaries
    const bool pure = (te.y & TILE_PURE) != 0;
    const bool smask = !pure && (nx % 16) == 0;
    if (!staged) {
        if (lane == 0) {
            meta = WsMeta{te.x, WS_DIRECT, xs, y};
            mbar_arrive(bar);
        }
        return;
    }
    const int parity = (idesc.parity ^ flip) & 1;
    const uint32_t mbytes = smask ? (uint32_t)min(WS_SEG, nx - xs) : 0u;
    const bool tensor = parity == 0 && idesc.tmap != nullptr;
    // row pieces of the one-plane-at-a-time copies
    const int lo = parity ? max(xs - CHE, 0) : xs;
    const int hi = parity ? min(xs + WS_SEG + CHE, nx) : min(xs + WS_SEG, nx);
    const uint32_t bytes = (uint32_t)(hi - lo) * (uint32_t)ES;
    const uint32_t total = tensor ? (uint32_t)(13 * WS_SEG * ES) + mbytes : 13u * bytes + mbytes;
    if (lane == 0) {
        meta = WsMeta{te.x, (pure ? WS_PURE : 0) | (smask ? WS_MASK : 0), xs, y};
        mbar_expect_tx(bar, total);
    }
    __syncwarp();
    T* const stage = reinterpret_cast<T*>(st);
    if (tensor) {
        if (lane == 0) {
            // the warp's earlier reads of this stage precede the copy into it
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            bulk_tensor_load(stage, idesc.tmap, xs, y, 0, bar);
        }
    } else if (lane < 13) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        const T* P = static_cast<const T*>(idesc.pops);
        int row = y;
        T* dst = stage + ws_plane_off<T, 0>(lane);
        if (parity) {
            row = y + ey(plane_dir(lane));
            if (row < 0) row += ny;
            if (row >= ny) row -= ny;
            dst = stage + ws_plane_off<T, 1>(lane) + (lo - (xs - CHE));
        }
        bulk_load(dst, P + lane * idesc.npad + (int64_t)row * nx + lo, bytes, bar);
    }
    if (lane == 13 && mbytes != 0u) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        bulk_load(st + ws_mask_off<T>(), idesc.mask + (int64_t)y * nx + xs, mbytes, bar);
    }
}

template <class ST>
__global__ void __launch_bounds__(WS_THREADS, LBM_WS_MINB) step_kernel_ws(const InstDesc* __restrict__ insts,
                                                                         const int4* __restrict__ tiles,
                                                                         int ntiles, int flip, int mode,
                                                                         Shape shape) {
    using T = typename ST::T;
    constexpr int SB = ws_stage_bytes<T>();
    constexpr uint32_t D = WS_DEPTH;
    extern __shared__ __align__(128) unsigned char ws_smem[];
    __shared__ __align__(16) InstDesc cdesc[WS_WARPS], idesc[WS_WARPS];
    __shared__ __align__(16) WsMeta meta[WS_WARPS][WS_DEPTH];
    __shared__ __align__(8) uint64_t bars[WS_WARPS][WS_DEPTH];
    (void)mode;
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    // stages start on 128-byte boundaries (bulk tensor copy destinations)
    unsigned char* const ring =
        ws_smem + ((128u - (smem_addr(ws_smem) & 127u)) & 127u) + (size_t)warp * D * SB;
    uint64_t* const bar = bars[warp];
    if (lane == 0) {
        for (uint32_t k = 0; k < D; ++k) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncwarp();
    // programmatic dependent launch (graph replays): let the next step launch,
    // and wait for the previous one before the first copy
    grid_dependents_go();
    grid_dependency_wait();
    asm volatile("fence.proxy.async.global;\n" ::: "memory");

    // segment numbering: item i -> tile ordinal i / ipt, row, segment
    const int nseg = shape.tw / WS_SEG;
    const int ipt = shape.rpt * nseg;
    auto tile_of = [&](int64_t i) -> int64_t { return (int64_t)blockIdx.x + (i / ipt) * (int64_t)gridDim.x; };
    int iheld = -1, cheld = -1;
    int64_t next = warp;  // next item to post
    for (uint32_t k = 0; k < D; ++k, next += WS_WARPS) {
        const int64_t t = tile_of(next);
        const bool valid = t < ntiles;
        const int4 te = valid ? tiles[t] : make_int4(0, 0, 0, 0);
        const int rem = (int)(next % ipt);
        ws_post<ST>(insts, idesc[warp], iheld, te, valid, rem / nseg, rem % nseg, flip, ring + k * SB,
                    meta[warp][k], &bar[k]);
    }
    for (uint32_t j = 0;; ++j) {
        const uint32_t s = j % D;
        // tile entry of the segment posted after this one, read ahead
        const int64_t tn = tile_of(next);
        const bool vn = tn < ntiles;
        int4 ten = make_int4(0, 0, 0, 0);
        if (vn) ten = tiles[tn];
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[s], (j / D) & 1u))) {
            if (lane == 0) {
                atomicExch(&g_step_status, 1);
                for (uint32_t q = 1; q < D; ++q) {  // the other stages may still be in flight
                    const uint32_t jq = j + q;
                    (void)mbar_wait_bounded(&bar[jq % D], (jq / D) & 1u);
                }
            }
            return;
        }
        const WsMeta m = meta[warp][s];
        if (m.flags & WS_END) return;  // every later stage holds an end marker too
        if (!(m.flags & WS_SKIP)) {
            if (m.inst != cheld) {
                warp_copy_desc(&cdesc[warp], insts + m.inst);
                cheld = m.inst;
            }
            const unsigned char* st = ring + s * SB;
            const T* stage = reinterpret_cast<const T*>(st);
            const unsigned char* smk = st + ws_mask_off<T>();
            if ((cdesc[warp].parity ^ flip) & 1) ws_segment<ST, 1>(cdesc[warp], stage, smk, m);
            else ws_segment<ST, 0>(cdesc[warp], stage, smk, m);
        }
        __syncwarp();
        const int rem = (int)(next % ipt);
        ws_post<ST>(insts, idesc[warp], iheld, ten, vn, rem / nseg, rem % nseg, flip, ring + s * SB,
                    meta[warp][s], &bar[s]);
        next += WS_WARPS;
    }
}

// One time step of a tile list.  OBS adds the observables of the
// pre-collision state, with per-thread and per-warp partials of type A: FP64
// for observe-only reads, the storage's accumulator type for the steady-state
// check step (which also writes).
// MB > 0: resident blocks of 256 threads to compile for (a register budget
// chosen per launch geometry), else the storage's default
// SPLIT (plain FP32-arithmetic steps): the launch runs the edge-cell chunks
// spread among the tiles, and the rows update interior pairs only
template <class ST, bool OBS, class A = double, int MB = 0, bool SPLIT = false>
__global__ void __launch_bounds__(256, MB > 0 ? MB : (OBS ? 2 : step_min_blocks<ST>())) step_kernel(const InstDesc* __restrict__ insts,
                                                    const int4* __restrict__ tiles, int ntiles,
                                                    int flip, int mode, Shape shape) {
    __shared__ __align__(16) InstDesc sd;
    __shared__ double red[OBS ? 8 : 1][NPART];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    // programmatic dependent launch (graph replays): let the next step launch
    // now; its blocks wait below until this grid has completed
    grid_dependents_go();
    int cur = -1;  // instance whose descriptor sd holds
    // on a grid-stride launch the next tile's entry is read while this tile
    // runs, so that a block's tiles follow each other without a wait
    int4 te_next = blockIdx.x < ntiles ? tiles[blockIdx.x] : make_int4(0, 0, 0, 0);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 te = te_next;
        if (t + (int)gridDim.x < ntiles) te_next = tiles[t + gridDim.x];
        // te.x is the same for the whole block, so the barriers are taken by
        // all of its threads or by none; an observing step also reuses red
        // per tile, so it always synchronises
        if (OBS || te.x != cur) {
            __syncthreads();
            const uint64_t* src = reinterpret_cast<const uint64_t*>(insts + te.x);
            uint64_t* dst = reinterpret_cast<uint64_t*>(&sd);
            for (int k = tid; k < (int)(sizeof(InstDesc) / 8); k += nthreads) dst[k] = src[k];
            __syncthreads();
            cur = te.x;
        }
        // the previous step (if launched as our programmatic prerequisite) has
        // completed and its writes are visible before any population is touched
        grid_dependency_wait();
        const int parity = (sd.parity ^ flip) & 1;
        constexpr bool split = SPLIT && !OBS && sizeof(typename ST::R) == 4;
        if constexpr (split) {
            if (te.y & TILE_EDGE) {
                if (parity) edge_block<ST, 1>(sd, te);
                else edge_block<ST, 0>(sd, te);
                continue;
            }
        }
        A acc[NPART];
#pragma unroll
        for (int k = 0; k < NPART; ++k) acc[k] = A(0);
        if (parity) tile_rows<ST, OBS, 1, A, split>(sd, te, mode, shape, acc);
        else tile_rows<ST, OBS, 0, A, split>(sd, te, mode, shape, acc);
        if (OBS && (mode & OBS_STATS)) {
            warp_block_reduce<A>(acc, red, sd.partials + (int64_t)(te.y & TILE_INDEX) * NPART);
        }
    }
}


// ---------------------------------------------------------------------------
// Dataflow stepping: one cooperative launch advances a tile list by nsteps
// time steps with no grid-wide barrier between steps.  Item (t, s) is tile t
// at step s of the launch.  It reads and writes only slots of the cells of
// tile t and of cells one link away, i.e. slots inside the 3 x 3 tile
// neighbourhood of t, and those slots were last written by step s - 1 of the
// same tiles (the AA pattern touches the same slot set of a cell on both
// parities).  So the block waits until tile t and its eight neighbours (nbr,
// -1 where there is no active tile) report step s - 1 complete, then updates
// the tile and reports step s.
//
// Issue order.  The steps are taken in sweeps of sweep_steps (K) steps; one
// sweep lists the items of its K steps in the order of a wavefront over the
// tile rows ("bands"): at wavefront position j, band j at the sweep's step 0,
// band j - L at step 1, ..., band j - (K-1) L at step K-1 (L >= 2 bands of
// lag, fixed when the list is built).  Item q of the launch is entry
// q mod per_sweep of the list, in sweep q / per_sweep; block b takes items b,
// b + G, b + 2G, ... (G blocks, all co-resident).  Every item waited on comes
// earlier in this order (a band's neighbours at the previous step sit L - 1
// or more wavefront positions back, or in the previous sweep), and the
// earliest unfinished item never waits, so the launch always completes.  With
// K = 1 the order is step by step.  With K > 1 the slots a step writes are
// read by the next step of the sweep a few bands later, while they are still
// in L2, so DRAM sees about one read and one write per slot per sweep.  Every
// wait is bounded: after FLOW_WAIT_LIMIT polls the block raises the launch's
// abort word (which ends every other wait at once) and the sticky status word,
// and the host reports the results as invalid instead of hanging.
//
// flags[0]: sticky status (non-zero after an expired wait; cleared by the
//           host when it reports it);
// flags[1]: abort word of the launch;
// flags[2 + t]: steps of this launch that tile t has completed.
// flags[1..] are zeroed before every launch.

constexpr uint32_t FLOW_WAIT_LIMIT = 1u << 21;

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void flow_wait(const int* done, int target, int* flags) {
    if (ld_acquire_gpu(done) >= target) return;
    for (uint32_t it = 0; it < FLOW_WAIT_LIMIT; ++it) {
        __nanosleep(64);
        if (ld_acquire_gpu(done) >= target) return;
        if (*reinterpret_cast<volatile int*>(flags + 1)) return;
    }
    atomicExch(flags + 1, 1);
    atomicExch(flags, 1);
}

// SPLIT: the same path for every cell as the SPLIT per-step kernel (interior
// pairs in the rows, then the tile's own edge cells)
template <class ST, int MB = 0, bool SPLIT = false>
__global__ void __launch_bounds__(256, MB > 0 ? MB : flow_min_blocks<ST>())
    step_kernel_flow(const InstDesc* __restrict__ insts, const FlowArgs fa, Shape shape) {
    __shared__ __align__(16) InstDesc sd;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    int* const done = fa.flags + 2;
    const int rel = nthreads > 32 ? 32 : 0;
    int held = -1;  // instance whose descriptor sd holds (same in every thread)
    const int64_t nsweeps = (fa.nsteps + fa.sweep_steps - 1) / fa.sweep_steps;
    const int64_t total = nsweeps * fa.per_sweep;
    for (int64_t q = blockIdx.x; q < total; q += gridDim.x) {
        const int64_t w = q / fa.per_sweep;
        const int4 it = fa.items[q - w * fa.per_sweep];
        const int s = (int)w * fa.sweep_steps + (it.x >> 24);
        if (s >= fa.nsteps) continue;  // the last sweep may be shorter
        const int t = it.y & TILE_INDEX;
        const int4 te = make_int4(it.x & 0xFFFFFF, it.y, it.z, it.w);
        if (s > 0 && tid < 9) {
            const int u = tid == 0 ? t : fa.nbr[(int64_t)t * 8 + tid - 1];
            if (u >= 0) flow_wait(done + u, s, fa.flags);
        }
        if (te.x != held) {  // sd is free: the previous item ended with a barrier
            const uint64_t* src = reinterpret_cast<const uint64_t*>(insts + te.x);
            uint64_t* dst = reinterpret_cast<uint64_t*>(&sd);
            for (int k = tid; k < (int)(sizeof(InstDesc) / 8); k += nthreads) dst[k] = src[k];
            held = te.x;
        }
        __syncthreads();
        const int parity = (sd.parity ^ fa.flip ^ s) & 1;
        double acc[NPART];
        constexpr bool split = SPLIT && sizeof(typename ST::R) == 4;
        if (parity) tile_rows<ST, false, 1, double, split>(sd, te, 0, shape, acc);
        else tile_rows<ST, false, 0, double, split>(sd, te, 0, shape, acc);
        if constexpr (split) {
            if (sd.split && (blockDim.x & 31) == 0 && (sd.nx & 1) == 0 && !(te.y & TILE_PURE)) {
                if (parity) tile_edge_cells<ST, 1>(sd, t - sd.tile_base);
                else tile_edge_cells<ST, 0>(sd, t - sd.tile_base);
            }
        }
        __syncthreads();
        // a thread outside warp 0 reports, so that the release overlaps warp
        // 0's polls for the next item
        if (tid == rel && t != fa.stall_tile) st_release_gpu(done + t, s + 1);
    }
}

}  // namespace lbm
