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

#include "lbm_internal.cuh"

// Resident blocks of 256 threads the step kernel is compiled for (register
// budget 65536 / (256 * n)): the two-cell pair path keeps 26 populations and
// the collision temporaries of two cells live.
#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 3
#endif
// the same for the 16-bit storages (which convert on every load and store)
#ifndef LBM_STEP_MIN_BLOCKS_16
#define LBM_STEP_MIN_BLOCKS_16 3
#endif

namespace lbm {

template <class ST>
constexpr int step_min_blocks() {
    return sizeof(typename ST::T) == 2 ? LBM_STEP_MIN_BLOCKS_16 : LBM_STEP_MIN_BLOCKS;
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

template <class R>
__device__ __forceinline__ void warp_block_reduce(double* acc, double (*red)[NPART], double* out) {
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
template <class ST, bool OBS, int PAR>
__device__ __forceinline__ void cell_body(const InstDesc& d, int x, int y,
                                          const typename ST::R* fin, const typename ST::R* gin,
                                          uint8_t m, int mode, double* acc) {
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
    // p = [sum_{i>=1} f_i + S_0(u)] / (4 sigma); the FP32 form multiplies by 0.6
    const E p = sizeof(R) == 8 ? (sum18 + S0) / E(4.0 * K_SIGMA) : (sum18 + S0) * E(0.6);
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
    feq[0] = E(-4.0 * K_SIGMA) * p + S0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const E Si = E(wgt(i)) * (E(3.0) * eu[i] + E(4.5) * eu[i] * eu[i] - E(1.5) * usq);
        feq[i] = (i <= 4 ? E(K_LAMBDA) : E(K_GAMMA)) * p + Si;
    }

    // neighbour types (only next to a boundary)
    uint32_t ntypes = 0, bnd = 0;
    if (m & NEAR_BOUNDARY) {
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const uint32_t tn = d.mask[nb[i]] & TYPE_BITS;
            ntypes |= tn << (4 * (i - 1));
            if (tn > POROUS) bnd |= 1u << i;
        }
    }

    // ---- observables of the pre-collision state -----------------------------
    if (OBS) {
        if (mode & OBS_STATS) {
            acc[P_MASS] += (double)sum18.v;
            // max of |u|^2; the fold takes one square root (sqrt is monotone)
            acc[P_PEAK] = fmax(acc[P_PEAK], (double)usq.v);
            if (type == FLUID) {
                acc[P_SUM_P] += (double)p.v;
                acc[P_N_FLUID] += 1.0;
                if (!isfinite((double)p.v)) acc[P_NAN] += 1.0;
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
                            acc[P_WSS_C] += fabs(-nyw * (sxx * nxw + sxy * nyw) + nxw * (sxy * nxw + syy * nyw));
                            acc[P_N_C] += 1.0;
                        }
                        if (hit_h) {
                            double ax = ah_x, ay = ah_y;
                            if (d.eye_normals) { ax = 0.0; ay = 1.0; }
                            const double r = sqrt(ax * ax + ay * ay);
                            const double nxw = r > 0.0 ? ax / r : 0.0, nyw = r > 0.0 ? ay / r : 0.0;
                            acc[P_WSS_I] += fabs(-nyw * (sxx * nxw + sxy * nyw) + nxw * (sxy * nxw + syy * nyw));
                            acc[P_N_I] += 1.0;
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
                acc[P_RESID] = fmax(acc[P_RESID], dx * dx + dy * dy);
            }
            if (mode & OBS_SNAP) {
                U[c] = ux.v;
                U[np + c] = uy.v;
            }
        }
    }

    // ---- body force, Eqs. 15-17: F_i = (1/2) e_i . F on the axis links --------
    const E gb = E(ph.g_beta) * (Tm - E(ph.T0));
    const E Fx = E(ph.drive_x) - gb * E(ph.gx);
    const E Fy = E(ph.drive_y) - gb * E(ph.gy);
    const E F1 = E(0.5) * Fx, F2 = E(0.5) * Fy;

    // ---- flow collision, Eq. 6 --------------------------------------------
    const E om = E(ph.omega);
    E fs[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fs[i] = f[i] - om * (f[i] - feq[i]);
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
#pragma unroll
    for (int i = 1; i <= 4; ++i) {
        const E teq = Tq * (E(1.0) + E(2.0) * eu[i]);
        gs[i - 1] = g[i - 1] - omT * (g[i - 1] - teq);
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
            if (tn == COLD) v = -gs[i - 1] + E(0.5) * E(ph.T_cold);
            else if (tn == HOT) v = -gs[i - 1] + E(0.5) * E(ph.T_hot);
            else if (tn == INLET) v = -gs[i - 1] + E(0.5) * E(ph.T_in);
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
        acc[P_Q_IN] += q_in;
        acc[P_Q_OUT] += q_out;
    }
}

template <class ST, bool OBS, int PAR>
__device__ __forceinline__ void update_cell(const InstDesc& d, int x, int y, int mode, double* acc) {
    using R = typename ST::R;
    int nb[9];
    neighbours(d, x, y, nb);
    R f[9], g[4];
    uint8_t m;
    load_cell<ST, PAR>(d, nb, f, g, m);
    cell_body<ST, OBS, PAR>(d, x, y, f, g, m, mode, acc);
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
__device__ __forceinline__ void collide_interior(float* f, bool porous, const Phys<float>& ph) {
    const float ux = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const float uy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    const float usq = ux * ux + uy * uy;
    const float S0 = float(K_W0) * (-1.5f * usq);
    const float sum18 = f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    const float p = (sum18 + S0) * 0.6f;
    const float Tm = f[9] + f[10] + f[11] + f[12];
    const float om = ph.omega;
    // equilibrium per opposite pair: common = kappa p + w (4.5 eu^2 - 1.5 usq), odd = 3 w eu
    const float c_ax = float(K_LAMBDA) * p - float(1.5 * K_W1) * usq;
    const float c_dg = float(K_GAMMA) * p - float(1.5 * K_W5) * usq;
    const float e5 = ux + uy, e6 = uy - ux;
    const float q1 = c_ax + float(4.5 * K_W1) * ux * ux, o1 = float(3.0 * K_W1) * ux;
    const float q2 = c_ax + float(4.5 * K_W1) * uy * uy, o2 = float(3.0 * K_W1) * uy;
    const float q5 = c_dg + float(4.5 * K_W5) * e5 * e5, o5 = float(3.0 * K_W5) * e5;
    const float q6 = c_dg + float(4.5 * K_W5) * e6 * e6, o6 = float(3.0 * K_W5) * e6;
    const float feq0 = float(-4.0 * K_SIGMA) * p + S0;
    // body force F = drive - g beta (T - T0) g_hat; F_i = (1/2) e_i . F on the axis links
    const float gb = ph.g_beta * (Tm - ph.T0);
    const float Fx = ph.drive_x - gb * ph.gx;
    const float Fy = ph.drive_y - gb * ph.gy;
    const float F1 = 0.5f * Fx, F2 = 0.5f * Fy;
    f[0] = f[0] - om * (f[0] - feq0);
    f[1] = f[1] - om * (f[1] - (q1 + o1)) + F1;
    f[3] = f[3] - om * (f[3] - (q1 - o1)) - F1;
    f[2] = f[2] - om * (f[2] - (q2 + o2)) + F2;
    f[4] = f[4] - om * (f[4] - (q2 - o2)) - F2;
    f[5] = f[5] - om * (f[5] - (q5 + o5));
    f[7] = f[7] - om * (f[7] - (q5 - o5));
    f[6] = f[6] - om * (f[6] - (q6 + o6));
    f[8] = f[8] - om * (f[8] - (q6 - o6));
    if (porous) {
        const float umx = (ux + 0.5f * Fx) / ph.den;
        const float umy = (uy + 0.5f * Fy) / ph.den;
        const float FDx = -ph.cK * umx, FDy = -ph.cK * umy;
        const float a1 = float(3.0 * K_W1), a5 = float(3.0 * K_W5);
        f[1] += a1 * FDx;
        f[3] -= a1 * FDx;
        f[2] += a1 * FDy;
        f[4] -= a1 * FDy;
        f[5] += a5 * (FDx + FDy);
        f[7] -= a5 * (FDx + FDy);
        f[6] += a5 * (FDy - FDx);
        f[8] -= a5 * (FDy - FDx);
    }
    const float omT = ph.omegaT, Tq = 0.25f * Tm;
    f[9] = f[9] - omT * (f[9] - Tq * (1.0f + 2.0f * ux));
    f[10] = f[10] - omT * (f[10] - Tq * (1.0f + 2.0f * uy));
    f[11] = f[11] - omT * (f[11] - Tq * (1.0f - 2.0f * ux));
    f[12] = f[12] - omT * (f[12] - Tq * (1.0f - 2.0f * uy));
}

// Collision of a cell pair (cells x and x+1, 13 values each) and its AA-pattern
// stores; every lane of the warp takes part (odd steps assemble x-shifted
// links by shuffles).
template <class ST, int PAR>
__device__ __forceinline__ void pair_collide_store(const InstDesc& d, int x, int y, float* a,
                                                   float* b, bool por0, bool por1) {
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
    collide_interior(a, por0, d.pf);
    collide_interior(b, por1, d.pf);

    // ---- store --------------------------------------------------------------
    if (PAR == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) ST::stf2(P + opp(q) * np + row + x, a[q], b[q], d);
#pragma unroll
        for (int i = 1; i <= 4; ++i) ST::stT2(P + (8 + opp(i)) * np + row + x, a[8 + i], b[8 + i], d);
    } else {
        ST::stf2(P + row + x, a[0], b[0], d);
#pragma unroll
        for (int k = 1; k < 13; ++k) {
            const bool heat = k > 8;
            const int i = heat ? k - 8 : k;
            const int pl = heat ? 8 + i : i;           // f*_i(x) goes to slot (x + e_i, i)
            const int dr = ey(i) == 1 ? rowu : (ey(i) == -1 ? rowd : row);
            T* dst = P + pl * np + dr;
            if (ex(i) == 0) {
                if (heat) ST::stT2(dst + x, a[k], b[k], d);
                else ST::stf2(dst + x, a[k], b[k], d);
            } else if (ex(i) == 1) {  // destination columns x+1, x+2
                const float left = __shfl_up_sync(0xffffffffu, b[k], 1);
                if (lane != 0) {
                    if (heat) ST::stT2(dst + x, left, a[k], d);
                    else ST::stf2(dst + x, left, a[k], d);
                } else {
                    if (heat) ST::stT(dst + x + 1, a[k], d);
                    else ST::stf(dst + x + 1, a[k], d);
                }
                if (lane == 31) {
                    if (heat) ST::stT(dst + xr, b[k], d);
                    else ST::stf(dst + xr, b[k], d);
                }
            } else {                  // destination columns x-1, x
                const float right = __shfl_down_sync(0xffffffffu, a[k], 1);
                if (lane != 31) {
                    if (heat) ST::stT2(dst + x, b[k], right, d);
                    else ST::stf2(dst + x, b[k], right, d);
                } else {
                    if (heat) ST::stT(dst + x, b[k], d);
                    else ST::stf(dst + x, b[k], d);
                }
                if (lane == 0) {
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
// two cells are combined in FP32 first (a sum of two values, a maximum, a
// count) and enter the FP64 partials once per pair: GB300's FP64 pipe is
// narrow, and per-cell FP64 updates made this step FP64-bound.
template <class ST>
__device__ __forceinline__ void pair_observe(const InstDesc& d, int x, int y, const float* a,
                                             const float* b, uint32_t m2, int mode, double* acc) {
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
        acc[P_MASS] += (double)mass;
        acc[P_PEAK] = fmax(acc[P_PEAK], (double)pk);
        acc[P_SUM_P] += (double)psum;
        acc[P_N_FLUID] += (double)nfl;
        if (bad) acc[P_NAN] += 1.0;
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
            acc[P_RESID] = fmax(acc[P_RESID], (double)r2);
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

template <class ST, int PAR, bool OBS = false>
__device__ __forceinline__ void update_pair_interior(const InstDesc& d, int x, int y, bool por0,
                                                     bool por1, uint32_t m2 = 0, int mode = 0,
                                                     double* acc = nullptr) {
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

    if constexpr (OBS) pair_observe<ST>(d, x, y, a, b, m2, mode, acc);
    pair_collide_store<ST, PAR>(d, x, y, a, b, por0, por1);
}

template <class ST, bool OBS, int PAR>
__device__ __forceinline__ void tile_rows(const InstDesc& sd, const int4& te, int mode, int rpt,
                                          double* acc) {
    constexpr int V = sizeof(typename ST::R) == 4 ? 2 : 1;
    const int x = te.z + V * threadIdx.x;
    if constexpr (V == 2) {
        // the pair path needs whole warps on one row and even rows; an
        // observing step takes it too when it also writes (the steady-state
        // check), while observe-only reads stay on the per-cell path
        const bool vec_ok = (!OBS || (mode & OBS_WRITE)) && (blockDim.x & 31) == 0 && (sd.nx & 1) == 0;
        // a pure tile (every cell fluid, in the grid, away from boundaries)
        // takes the pair path without reading its mask
        const bool pure = (te.y & TILE_PURE) != 0;
        for (int r = 0; r < rpt; ++r) {
            const int y = te.w + threadIdx.y + r * blockDim.y;
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
                    fast = __all_sync(0xffffffffu, (m2 & 0x0E0Eu) == 0u);
                }
                if (fast)
                    update_pair_interior<ST, PAR, OBS>(sd, x, y, (m2 & 1u) != 0 && sd.tm_model == 0,
                                                       (m2 & 0x100u) != 0 && sd.tm_model == 0, m2, mode,
                                                       acc);
            }
            if (!fast) {
                if (x < sd.nx && y < sd.ny) update_cell<ST, OBS, PAR>(sd, x, y, mode, acc);
                if (x + 1 < sd.nx && y < sd.ny) update_cell<ST, OBS, PAR>(sd, x + 1, y, mode, acc);
            }
        }
    } else {
        for (int r = 0; r < rpt; ++r) {
            const int y = te.w + threadIdx.y + r * blockDim.y;
            if (x < sd.nx && y < sd.ny) update_cell<ST, OBS, PAR>(sd, x, y, mode, acc);
        }
    }
}

// ---------------------------------------------------------------------------
// Staged step of the FP32-arithmetic kernels (selected by launch shapes with
// one row of threads per block).  A block of NT threads walks a strip of
// W = 2 NT cells x H rows, one row at a time.  The 13 population segments each
// row needs (own slots on an even step; on an odd step the source row of each
// plane, widened by a 16-byte halo on both sides for the x-shifted links) are
// copied into shared memory by bulk copies, several rows ahead of the row being
// computed, so no register holds a pending load.  Each thread then updates a
// cell pair from shared memory (interior pairs with collide_interior, every
// other active cell with cell_body) and stores to global memory in the AA
// pattern.  Rows never share a slot (each slot is read and written only by the
// cell that owns it), so staging later rows before this row's stores land is
// exact.  Halo elements that belong to cells of a neighbouring strip are copied
// but never used.  Measured slower than the direct kernel on the eye
// workloads; kept as an autotuner candidate.

// elements per 16-byte chunk, and shared-memory segment length per plane
template <class T>
__host__ __device__ constexpr int chunk_elems() { return 16 / (int)sizeof(T); }
template <class T>
__host__ __device__ constexpr int seg_elems(int W) { return W + 2 * chunk_elems<T>(); }

// source row of plane p for target row y on an odd step: f_i(x) sits in slot
// (x - e_i, opp(i)), i.e. plane p = opp(i) holds it at row y - ey(i) = y + ey(p)
__device__ __forceinline__ constexpr int plane_dir(int p) { return p < 9 ? p : p - 8; }

template <class ST, int PAR>
__device__ __forceinline__ void staged_row(const InstDesc& sd, const typename ST::T* stage, int x0,
                                           int W, int y) {
    using T = typename ST::T;
    using R = float;
    constexpr int CHE = chunk_elems<T>();
    const int SEG = W + 2 * CHE;
    const int nx = sd.nx;
    const int x = x0 + 2 * (int)threadIdx.x;
    if (x >= nx) return;
    const uint32_t m2 = *reinterpret_cast<const uint16_t*>(sd.mask + (int64_t)y * nx + x);
    if ((m2 & 7u) > POROUS && ((m2 >> 8) & 7u) > POROUS) return;  // neither cell is active
    // the pair's wrap-around columns at a periodic edge are not staged: use
    // the direct path there
    if (x == 0 || x + 2 >= nx) {
        update_cell<ST, false, PAR>(sd, x, y, 0, nullptr);
        if (x + 1 < nx) update_cell<ST, false, PAR>(sd, x + 1, y, 0, nullptr);
        return;
    }
    const int j = x - x0 + CHE;  // stage column of cell x
    float a[13], b[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        const bool heat = k > 8;
        const int i = heat ? k - 8 : k;
        const int pl = PAR == 0 ? k : (heat ? 8 + opp(i) : opp(i));
        const int jj = PAR == 0 ? j : j - ex(i);
        const T* src = stage + pl * SEG + jj;
        if (heat) {
            a[k] = ST::sldT(src, sd);
            b[k] = ST::sldT(src + 1, sd);
        } else {
            a[k] = ST::sldf(src, sd);
            b[k] = ST::sldf(src + 1, sd);
        }
    }
    const bool interior = (m2 & 0x0E0Eu) == 0u;
    if (!interior) {
        // at least one cell next to a boundary (or solid): general update of
        // each active cell with the staged populations
        for (int v = 0; v < 2; ++v) {
            const float* c = v == 0 ? a : b;
            R f[9], g[4];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = c[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) g[i] = c[9 + i];
            cell_body<ST, false, PAR>(sd, x + v, y, f, g, (uint8_t)(m2 >> (8 * v)), 0, nullptr);
        }
        return;
    }
    collide_interior(a, (m2 & 1u) != 0 && sd.tm_model == 0, sd.pf);
    collide_interior(b, (m2 & 0x100u) != 0 && sd.tm_model == 0, sd.pf);
    T* const P = static_cast<T*>(sd.pops);
    const int np = (int)sd.npad;
    const int ny = sd.ny;
    const int row = y * nx;
    const int rowu = (y == ny - 1 ? 0 : y + 1) * nx;
    const int rowd = (y == 0 ? ny - 1 : y - 1) * nx;
    if (PAR == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) ST::stf2(P + opp(q) * np + row + x, a[q], b[q], sd);
#pragma unroll
        for (int i = 1; i <= 4; ++i) ST::stT2(P + (8 + opp(i)) * np + row + x, a[8 + i], b[8 + i], sd);
    } else {
        ST::stf2(P + row + x, a[0], b[0], sd);
#pragma unroll
        for (int k = 1; k < 13; ++k) {
            const bool heat = k > 8;
            const int i = heat ? k - 8 : k;
            const int pl = heat ? 8 + i : i;  // f*_i(x) goes to slot (x + e_i, i)
            const int dr = ey(i) == 1 ? rowu : (ey(i) == -1 ? rowd : row);
            T* dst = P + pl * np + dr + x;
            if (ex(i) == 0) {
                if (heat) ST::stT2(dst, a[k], b[k], sd);
                else ST::stf2(dst, a[k], b[k], sd);
            } else {
                const int o = ex(i);
                if (heat) {
                    ST::stT(dst + o, a[k], sd);
                    ST::stT(dst + 1 + o, b[k], sd);
                } else {
                    ST::stf(dst + o, a[k], sd);
                    ST::stf(dst + 1 + o, b[k], sd);
                }
            }
        }
    }
}

// One thread issues the 13 row segments of a row as bulk copies
// (cp.async.bulk) that complete on the row's shared-memory barrier; TSTAGES
// rows are in flight per block.  Every wait on a barrier is
// bounded: if a copy has not landed after TMA_WAIT_LIMIT polls the block sets
// the device status word, waits (again bounded) for the copies it issued and
// leaves, and the host reports the error instead of hanging.

constexpr int TSTAGES = 4;
constexpr uint32_t TMA_WAIT_LIMIT = 1u << 22;

// Non-zero after a staged copy failed to complete; read and cleared by the host
// (take_step_status).  Only the FP32-arithmetic unit instantiates the staged
// kernels, so its copy of this word is the one that is used.
static __device__ int g_step_status = 0;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
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

// Issue row y of a strip (global row sequence g) into stage g % TSTAGES.
// Every copy starts on a 16-byte boundary and moves a multiple of 16 bytes:
// x0 and W are multiples of the 16-byte chunk, so are nx (checked) and the
// plane stride.
template <class ST>
__device__ __forceinline__ void tma_issue(const InstDesc& sd, typename ST::T* buf, uint64_t* bars,
                                          uint32_t g, int x0, int W, int y, int parity) {
    using T = typename ST::T;
    constexpr int CHE = chunk_elems<T>();
    const int SEG = W + 2 * CHE;
    const int s = (int)(g % TSTAGES);
    T* stage = buf + (size_t)s * 13 * SEG;
    const int lo = parity ? max(x0 - CHE, 0) : x0;
    const int hi = parity ? min(x0 + W + CHE, sd.nx) : min(x0 + W, sd.nx);
    const uint32_t bytes = (uint32_t)(hi - lo) * (uint32_t)sizeof(T);
    const T* P = static_cast<const T*>(sd.pops);
    const int np = (int)sd.npad;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(&bars[s], 13u * bytes);
    for (int p = 0; p < 13; ++p) {
        int row = y;
        if (parity) {
            row = y + ey(plane_dir(p));
            if (row < 0) row += sd.ny;
            if (row >= sd.ny) row -= sd.ny;
        }
        bulk_load(stage + p * SEG + (lo - (x0 - CHE)), P + p * np + row * sd.nx + lo, bytes, &bars[s]);
    }
}

template <class ST>
__global__ void __launch_bounds__(128) step_kernel_tma(const InstDesc* __restrict__ insts,
                                                       const int4* __restrict__ tiles, int ntiles,
                                                       int flip, int mode, Shape shape) {
    using T = typename ST::T;
    extern __shared__ __align__(128) unsigned char tma_smem[];
    __shared__ __align__(16) InstDesc sd;
    __shared__ __align__(8) uint64_t bars[TSTAGES];
    T* const buf = reinterpret_cast<T*>(tma_smem);
    const int W = 2 * (int)blockDim.x;
    const int SEG = seg_elems<T>(W);
    const int H = shape.rpt;
    (void)mode;
    if (threadIdx.x == 0) {
        for (int k = 0; k < TSTAGES; ++k) mbar_init(&bars[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    // programmatic dependent launch (graph replays): nothing is read before
    // the previous step has completed
    grid_dependents_go();
    grid_dependency_wait();
    uint32_t seq = 0;  // rows this block has staged so far (same in every thread)
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 te = tiles[t];
        __syncthreads();
        {
            const uint64_t* src = reinterpret_cast<const uint64_t*>(insts + te.x);
            uint64_t* dst = reinterpret_cast<uint64_t*>(&sd);
            for (int k = threadIdx.x; k < (int)(sizeof(InstDesc) / 8); k += blockDim.x) dst[k] = src[k];
        }
        __syncthreads();
        const int parity = (sd.parity ^ flip) & 1;
        const int x0 = te.z, y0 = te.w;
        const int rows = min(H, sd.ny - y0);
        if ((sd.nx % chunk_elems<T>()) != 0) {
            for (int r = 0; r < rows; ++r) {
                const int x = x0 + 2 * (int)threadIdx.x;
                for (int v = 0; v < 2; ++v)
                    if (x + v < sd.nx) {
                        if (parity) update_cell<ST, false, 1>(sd, x + v, y0 + r, 0, nullptr);
                        else update_cell<ST, false, 0>(sd, x + v, y0 + r, 0, nullptr);
                    }
            }
            continue;
        }
        const uint32_t base = seq;
        int issued = 0;  // rows of this strip issued so far (meaningful in thread 0)
        if (threadIdx.x == 0)
            for (; issued < TSTAGES - 1 && issued < rows; ++issued)
                tma_issue<ST>(sd, buf, bars, base + issued, x0, W, y0 + issued, parity);
        for (int r = 0; r < rows; ++r) {
            if (threadIdx.x == 0 && issued < rows && issued < r + TSTAGES) {
                tma_issue<ST>(sd, buf, bars, base + issued, x0, W, y0 + issued, parity);
                ++issued;
            }
            const uint32_t g = base + r;
            const bool ok = mbar_wait_bounded(&bars[g % TSTAGES], (g / TSTAGES) & 1u);
            if (__syncthreads_or(!ok)) {
                // a copy did not land: record it, wait (bounded) for what this
                // block still has in flight, and leave
                if (threadIdx.x == 0) {
                    atomicExch(&g_step_status, 1);
                    for (int q = r; q < issued; ++q) {
                        const uint32_t gq = base + q;
                        (void)mbar_wait_bounded(&bars[gq % TSTAGES], (gq / TSTAGES) & 1u);
                    }
                }
                return;
            }
            const T* stage = buf + (size_t)(g % TSTAGES) * 13 * SEG;
            if (parity) staged_row<ST, 1>(sd, stage, x0, W, y0 + r);
            else staged_row<ST, 0>(sd, stage, x0, W, y0 + r);
            __syncthreads();
        }
        seq += rows;
    }
}

template <class ST, bool OBS>
__global__ void __launch_bounds__(256, OBS ? 2 : step_min_blocks<ST>()) step_kernel(const InstDesc* __restrict__ insts,
                                                    const int4* __restrict__ tiles, int ntiles,
                                                    int flip, int mode, Shape shape) {
    __shared__ __align__(16) InstDesc sd;
    __shared__ double red[OBS ? 8 : 1][NPART];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    // programmatic dependent launch (graph replays): let the next step launch
    // now; its blocks wait below until this grid has completed
    grid_dependents_go();
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 te = tiles[t];
        __syncthreads();
        {
            const uint64_t* src = reinterpret_cast<const uint64_t*>(insts + te.x);
            uint64_t* dst = reinterpret_cast<uint64_t*>(&sd);
            for (int k = tid; k < (int)(sizeof(InstDesc) / 8); k += nthreads) dst[k] = src[k];
        }
        __syncthreads();
        // the previous step (if launched as our programmatic prerequisite) has
        // completed and its writes are visible before any population is touched
        grid_dependency_wait();
        const int parity = (sd.parity ^ flip) & 1;
        double acc[NPART];
#pragma unroll
        for (int k = 0; k < NPART; ++k) acc[k] = 0.0;
        if (parity) tile_rows<ST, OBS, 1>(sd, te, mode, shape.rpt, acc);
        else tile_rows<ST, OBS, 0>(sd, te, mode, shape.rpt, acc);
        if (OBS && (mode & OBS_STATS)) {
            warp_block_reduce<double>(acc, red, sd.partials + (int64_t)(te.y & TILE_INDEX) * NPART);
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

template <class ST>
__global__ void __launch_bounds__(256, step_min_blocks<ST>())
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
        if (parity) tile_rows<ST, false, 1>(sd, te, 0, shape.rpt, acc);
        else tile_rows<ST, false, 0>(sd, te, 0, shape.rpt, acc);
        __syncthreads();
        // a thread outside warp 0 reports, so that the release overlaps warp
        // 0's polls for the next item
        if (tid == rel && t != fa.stall_tile) st_release_gpu(done + t, s + 1);
    }
}

}  // namespace lbm
