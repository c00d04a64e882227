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

namespace lbm {

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

template <class R>
__device__ __forceinline__ R pressure_from(R sum18, R S0) {
    // Eq. 9: p = [sum_{i>=1} f_i + S_0(u)] / (4 sigma)
    if constexpr (sizeof(R) == 8) return (sum18 + S0) / R(4.0 * K_SIGMA);
    else return (sum18 + S0) * R(0.6);
}

template <class R>
__device__ __forceinline__ void warp_block_reduce(double* acc, double (*red)[NPART], double* out) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NPART; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            double o = __shfl_down_sync(0xffffffffu, v, off);
            v = k < NSUM ? v + o : fmax(v, o);
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
                double o = __shfl_down_sync(0xffffffffu, v, off);
                v = k < NSUM ? v + o : fmax(v, o);
            }
            if (lane == 0) out[k] = v;
        }
    }
}

template <class ST, bool OBS, int PAR>
__device__ __forceinline__ void update_cell(const InstDesc& d, int x, int y, int mode,
                                            double* acc) {
    using T = typename ST::T;
    using R = typename ST::R;
    const int nx = d.nx, ny = d.ny;
    const int c = y * nx + x;

    // neighbour indices (wrap-around only ever triggers on periodic edges:
    // a non-periodic edge holds no active cell)
    const int xl = x == 0 ? nx - 1 : x - 1;
    const int xr = x == nx - 1 ? 0 : x + 1;
    const int yd = (y == 0 ? ny - 1 : y - 1) * nx;
    const int yu = (y == ny - 1 ? 0 : y + 1) * nx;
    const int yc = y * nx;
    int nb[9];
    nb[0] = c;
    nb[1] = yc + xr;
    nb[2] = yu + x;
    nb[3] = yc + xl;
    nb[4] = yd + x;
    nb[5] = yu + xr;
    nb[6] = yu + xl;
    nb[7] = yd + xl;
    nb[8] = yd + xr;

    T* const P = static_cast<T*>(d.pops);
    const int np = (int)d.npad;  // 13 * npad < 2^31 (checked at creation)
    const Phys<R>& ph = phys<R>(d);

    // ---- load (AA read pattern) -------------------------------------------
    // The mask and all 13 populations are requested together (every slot
    // index is in range for any cell of the grid), so an active cell pays one
    // memory round trip; a solid cell inside a launched tile discards them.
    const uint8_t m = d.mask[c];
    R f[9], g[4];
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
    const int type = m & TYPE_BITS;
    if (type > POROUS) return;

    // ---- moments, Eq. 9 and Eq. 13 ------------------------------------------
    const R ux = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const R uy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    const R usq = ux * ux + uy * uy;
    const R S0 = R(K_W0) * (R(-1.5) * usq);
    const R sum18 = f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    const R p = pressure_from<R>(sum18, S0);
    const R Tm = g[0] + g[1] + g[2] + g[3];

    // e_i . u for i = 0..8
    R eu[9];
    eu[0] = R(0);
    eu[1] = ux;
    eu[2] = uy;
    eu[3] = -ux;
    eu[4] = -uy;
    eu[5] = ux + uy;
    eu[6] = -ux + uy;
    eu[7] = -ux - uy;
    eu[8] = ux - uy;

    // equilibrium, Eqs. 7-8
    R feq[9];
    feq[0] = R(-4.0 * K_SIGMA) * p + S0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const R Si = R(wgt(i)) * (R(3.0) * eu[i] + R(4.5) * eu[i] * eu[i] - R(1.5) * usq);
        feq[i] = (i <= 4 ? R(K_LAMBDA) : R(K_GAMMA)) * p + Si;
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
            acc[P_MASS] += (double)sum18;
            const double sp = sqrt((double)usq);
            acc[P_PEAK] = fmax(acc[P_PEAK], sp);
            if (type == FLUID) {
                acc[P_SUM_P] += (double)p;
                acc[P_N_FLUID] += 1.0;
                if (!isfinite((double)p)) acc[P_NAN] += 1.0;
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
                        const double d1 = (double)(f[1] - feq[1]), d2 = (double)(f[2] - feq[2]);
                        const double d3 = (double)(f[3] - feq[3]), d4 = (double)(f[4] - feq[4]);
                        const double d5 = (double)(f[5] - feq[5]), d6 = (double)(f[6] - feq[6]);
                        const double d7 = (double)(f[7] - feq[7]), d8 = (double)(f[8] - feq[8]);
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
                const double dx = (double)ux - (double)U[c];
                const double dy = (double)uy - (double)U[np + c];
                acc[P_RESID] = fmax(acc[P_RESID], sqrt(dx * dx + dy * dy));
            }
            if (mode & OBS_SNAP) {
                U[c] = ux;
                U[np + c] = uy;
            }
        }
    }

    // ---- body force, Eqs. 15-17: F_i = (1/2) e_i . F on the axis links --------
    const R gb = ph.g_beta * (Tm - ph.T0);
    const R Fx = ph.drive_x - gb * ph.gx;
    const R Fy = ph.drive_y - gb * ph.gy;
    const R F1 = R(0.5) * Fx, F2 = R(0.5) * Fy;

    // ---- flow collision, Eq. 6 --------------------------------------------
    const R om = ph.omega;
    R fs[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fs[i] = f[i] - om * (f[i] - feq[i]);
    fs[1] = fs[1] + F1;
    fs[2] = fs[2] + F2;
    fs[3] = fs[3] + (-F1);
    fs[4] = fs[4] + (-F2);

    // ---- Darcy drag in porous cells, Eq. 4 at the mid-step velocity ---------
    if (type == POROUS) {
        const R den = ph.den, cK = ph.cK;
        const R umx = (ux + R(0.5) * Fx) / den;
        const R umy = (uy + R(0.5) * Fy) / den;
        const R FDx = -cK * umx;
        const R FDy = -cK * umy;
        const R a1 = R(3.0 * K_W1), a5 = R(3.0 * K_W5);
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
    const R omT = ph.omegaT;
    const R Tq = R(0.25) * Tm;
    R gs[4];
#pragma unroll
    for (int i = 1; i <= 4; ++i) {
        const R teq = Tq * (R(1.0) + R(2.0) * eu[i]);
        gs[i - 1] = g[i - 1] - omT * (g[i - 1] - teq);
    }

    const bool write = !OBS || (mode & OBS_WRITE);

    // ---- stream (AA write pattern) with link-wise boundary rules ----------
    if (write) ST::stf(P + c, fs[0], d);
    double q_in = 0.0, q_out = 0.0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const bool is_bnd = (bnd >> i) & 1u;
        R v = fs[i];
        if (is_bnd) {
            const uint32_t tn = (ntypes >> (4 * (i - 1))) & 15u;
            if (tn == INLET) {
                // moving-wall bounce-back; 6 w_i e_i.u is the odd part of feq
                const int xn = ex(i) == 1 ? xr : (ex(i) == -1 ? xl : x);
                const int ynb = ey(i) == 1 ? (y == ny - 1 ? 0 : y + 1)
                                           : (ey(i) == -1 ? (y == 0 ? ny - 1 : y - 1) : y);
                R shape = R(1.0);
                if (d.inlet_profile == 1) {
                    const int cg = d.inlet_dir_x == 0 ? xn : ynb;
                    const R s = (R(cg - d.inlet_lo) + R(0.5)) / R(d.inlet_width);
                    shape = R(4.0) * s * (R(1.0) - s);
                }
                const R uin = ph.u_in_max * shape;
                const R uix = uin * R(d.inlet_dir_x), uiy = uin * R(d.inlet_dir_y);
                v = fs[i] - R(6.0 * wgt(i)) * (R(ex(i)) * uix + R(ey(i)) * uiy);
                if (OBS) q_in += (double)(v - fs[i]);
            } else if (tn == OUTLET) {
                // pressure anti-bounce-back: minus f* plus the even part of feq(p_out, u)
                const R kap = i <= 4 ? R(K_LAMBDA) : R(K_GAMMA);
                v = -fs[i] + R(2.0) * (kap * ph.p_out +
                                       R(wgt(i)) * (R(4.5) * eu[i] * eu[i] - R(1.5) * usq));
                if (OBS) q_out += (double)(fs[i] - v);
            }
            // any wall: halfway bounce-back, v = f*_i
        }
        if (write) {
            const bool to_own = (PAR == 0) != is_bnd;  // even+stream or odd+boundary
            if (to_own) ST::stf(P + opp(i) * np + c, v, d);
            else ST::stf(P + i * np + nb[i], v, d);
        }
    }
#pragma unroll
    for (int i = 1; i <= 4; ++i) {
        const bool is_bnd = (bnd >> i) & 1u;
        R v = gs[i - 1];
        if (is_bnd) {
            const uint32_t tn = (ntypes >> (4 * (i - 1))) & 15u;
            if (tn == COLD) v = -gs[i - 1] + R(0.5) * ph.T_cold;
            else if (tn == HOT) v = -gs[i - 1] + R(0.5) * ph.T_hot;
            else if (tn == INLET) v = -gs[i - 1] + R(0.5) * ph.T_in;
            else if (tn == OUTLET) v = -gs[i - 1] + R(0.5) * Tm;
            // adiabatic: bounce-back, zero heat flux
        }
        if (write) {
            const bool to_own = (PAR == 0) != is_bnd;
            if (to_own) ST::stT(P + (8 + opp(i)) * np + c, v, d);
            else ST::stT(P + (8 + i) * np + nb[i], v, d);
        }
    }
    if (OBS && (mode & OBS_STATS)) {
        acc[P_Q_IN] += q_in;
        acc[P_Q_OUT] += q_out;
    }
}

template <class ST, bool OBS>
__global__ void __launch_bounds__(256, (OBS || sizeof(typename ST::R) == 8) ? 2 : (sizeof(typename ST::T) == 2 ? 3 : 4)) step_kernel(const InstDesc* __restrict__ insts,
                                                    const int4* __restrict__ tiles, int ntiles,
                                                    int flip, int mode, Shape shape) {
    __shared__ __align__(16) InstDesc sd;
    __shared__ double red[OBS ? 8 : 1][NPART];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 te = tiles[t];
        __syncthreads();
        {
            const uint64_t* src = reinterpret_cast<const uint64_t*>(insts + te.x);
            uint64_t* dst = reinterpret_cast<uint64_t*>(&sd);
            for (int k = tid; k < (int)(sizeof(InstDesc) / 8); k += nthreads) dst[k] = src[k];
        }
        __syncthreads();
        const int parity = (sd.parity ^ flip) & 1;
        double acc[NPART];
#pragma unroll
        for (int k = 0; k < NPART; ++k) acc[k] = 0.0;
        const int x = te.z + threadIdx.x;
        for (int r = 0; r < shape.rpt; ++r) {
            const int y = te.w + threadIdx.y + r * blockDim.y;
            if (x < sd.nx && y < sd.ny) {
                if (parity) update_cell<ST, OBS, 1>(sd, x, y, mode, acc);
                else update_cell<ST, OBS, 0>(sd, x, y, mode, acc);
            }
        }
        if (OBS && (mode & OBS_STATS)) {
            warp_block_reduce<double>(acc, red, sd.partials + (int64_t)te.y * NPART);
        }
    }
}

}  // namespace lbm
