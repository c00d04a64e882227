// Vortex measures of a velocity field on a domain's grid (Eq. 18, Tab. 3):
// the vortex intensity I = 2 * integral of omega_z over the chamber, with
// omega_z = (1/2)(du_y/dx - du_x/dy), signed and in absolute value, and the
// vortex centres as the extrema of the stream function psi (u_x = dpsi/dy).
//
// Discretisation (the same definitions as the test oracle, written apart):
// at a fluid cell each derivative is the difference of the two axis
// neighbours' values over their distance; an active neighbour contributes its
// velocity at distance 1, any other one the no-slip wall value 0 halfway
// along the link (distance 1/2).  psi is the midpoint sum of u_x up each
// column from y = 0 (u_x = 0 at non-active cells).  Extrema ties go to the
// lowest flat index y*nx + x.
//
// One thread walks one column (psi is a running sum along y); the block's
// partial sums and extrema are folded in a fixed order, so the result does
// not depend on scheduling.  Compiled with -fmad=false: the per-cell values
// are those of a plain sequential evaluation.
#include <cstdio>

#include "lbm.h"
#include "lbm_internal.cuh"

namespace lbm {

// internal accessors of lbm_api.cu
lbm_status set_error(lbm_status s, const char* msg);
bool domain_vortex_parts(const lbm_domain* d, const uint8_t** mask, int* nx, int* ny,
                         int* periodic_x, int* periodic_y, double** scratch,
                         int64_t* scratch_doubles, double* dx_m, double* dt_s,
                         cudaStream_t* stream);

constexpr int VX_THREADS = 128;
// per-block partial: I, |I|, n_fluid, psi_max, index of psi_max, psi_min, index of psi_min
constexpr int VX_PART = 7;

__device__ __forceinline__ bool vx_active(uint8_t m) { return (m & TYPE_BITS) <= POROUS; }

__device__ __forceinline__ double vx_axis(const uint8_t* mask, const double* comp, int nx, int ny,
                                          int px, int py, int x, int y, int dx, int dy,
                                          double* dist) {
    int xn = x + dx, yn = y + dy;
    if (px) xn = (xn + nx) % nx;
    if (py) yn = (yn + ny) % ny;
    if (xn < 0 || xn >= nx || yn < 0 || yn >= ny || !vx_active(mask[(int64_t)yn * nx + xn])) {
        *dist = 0.5;
        return 0.0;
    }
    *dist = 1.0;
    return comp[(int64_t)yn * nx + xn];
}

// better extremum: larger (sign +1) or smaller (sign -1) value, then lower index
__device__ __forceinline__ bool vx_better(double v, double i, double bv, double bi, double sign) {
    if (bi < 0.0) return i >= 0.0;
    if (i < 0.0) return false;
    if (v * sign > bv * sign) return true;
    return v == bv && i < bi;
}

__global__ void __launch_bounds__(VX_THREADS) vortex_columns_kernel(
    const uint8_t* __restrict__ mask, const double* __restrict__ u, int nx, int ny, int px,
    int py, double* __restrict__ part) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)nx * ny;
    const double* ux = u;
    const double* uy = u + N;
    double I = 0.0, Ia = 0.0, n = 0.0;
    double pmax = 0.0, imax = -1.0, pmin = 0.0, imin = -1.0;
    if (x < nx) {
        double S = 0.0;
        for (int y = 0; y < ny; ++y) {
            const int64_t c = (int64_t)y * nx + x;
            const uint8_t m = mask[c];
            const double v = vx_active(m) ? ux[c] : 0.0;
            const double psi = S + 0.5 * v;
            S = S + v;
            if ((m & TYPE_BITS) != FLUID) continue;
            double hr, hl, hu, hd;
            const double vr = vx_axis(mask, uy, nx, ny, px, py, x, y, 1, 0, &hr);
            const double vl = vx_axis(mask, uy, nx, ny, px, py, x, y, -1, 0, &hl);
            const double vu = vx_axis(mask, ux, nx, ny, px, py, x, y, 0, 1, &hu);
            const double vd = vx_axis(mask, ux, nx, ny, px, py, x, y, 0, -1, &hd);
            const double duy_dx = (vr - vl) / (hr + hl);
            const double dux_dy = (vu - vd) / (hu + hd);
            const double omega = 0.5 * (duy_dx - dux_dy);
            I += 2.0 * omega;
            Ia += 2.0 * fabs(omega);
            n += 1.0;
            if (imax < 0.0 || psi > pmax) { pmax = psi; imax = (double)c; }
            if (imin < 0.0 || psi < pmin) { pmin = psi; imin = (double)c; }
        }
    }
    __shared__ double sh[VX_PART][VX_THREADS];
    const int t = threadIdx.x;
    sh[0][t] = I; sh[1][t] = Ia; sh[2][t] = n;
    sh[3][t] = pmax; sh[4][t] = imax; sh[5][t] = pmin; sh[6][t] = imin;
    __syncthreads();
    for (int s = VX_THREADS / 2; s > 0; s >>= 1) {
        if (t < s) {
            for (int k = 0; k < 3; ++k) sh[k][t] += sh[k][t + s];
            if (vx_better(sh[3][t + s], sh[4][t + s], sh[3][t], sh[4][t], 1.0)) {
                sh[3][t] = sh[3][t + s];
                sh[4][t] = sh[4][t + s];
            }
            if (vx_better(sh[5][t + s], sh[6][t + s], sh[5][t], sh[6][t], -1.0)) {
                sh[5][t] = sh[5][t + s];
                sh[6][t] = sh[6][t + s];
            }
        }
        __syncthreads();
    }
    if (t == 0)
        for (int k = 0; k < VX_PART; ++k) part[(int64_t)blockIdx.x * VX_PART + k] = sh[k][0];
}

// block partials in block order -> out[VX_PART]
__global__ void vortex_fold_kernel(const double* __restrict__ part, int nblocks,
                                   double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a[VX_PART] = {0.0, 0.0, 0.0, 0.0, -1.0, 0.0, -1.0};
    for (int b = 0; b < nblocks; ++b) {
        const double* p = part + (int64_t)b * VX_PART;
        a[0] += p[0];
        a[1] += p[1];
        a[2] += p[2];
        if (vx_better(p[3], p[4], a[3], a[4], 1.0)) { a[3] = p[3]; a[4] = p[4]; }
        if (vx_better(p[5], p[6], a[5], a[6], -1.0)) { a[5] = p[5]; a[6] = p[6]; }
    }
    for (int k = 0; k < VX_PART; ++k) out[k] = a[k];
}

}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_vortex(lbm_domain* dom, const double* dev_u, lbm_vortex_info* out) {
    if (!out || !dev_u) return set_error(LBM_EINVAL, "null argument");
    const uint8_t* mask = nullptr;
    int nx = 0, ny = 0, px = 0, py = 0;
    double* scratch = nullptr;
    int64_t cap = 0;
    double dx = 0.0, dt = 0.0;
    cudaStream_t s = nullptr;
    if (!domain_vortex_parts(dom, &mask, &nx, &ny, &px, &py, &scratch, &cap, &dx, &dt, &s))
        return LBM_EINVAL;
    const int nblocks = (nx + VX_THREADS - 1) / VX_THREADS;
    if ((int64_t)(nblocks + 1) * VX_PART > cap)
        return set_error(LBM_EINVAL, "grid too small for the vortex reduction scratch");
    double* part = scratch;
    double* res = scratch + (int64_t)nblocks * VX_PART;
    vortex_columns_kernel<<<nblocks, VX_THREADS, 0, s>>>(mask, dev_u, nx, ny, px, py, part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        vortex_fold_kernel<<<1, 32, 0, s>>>(part, nblocks, res);
        e = cudaGetLastError();
    }
    double h[VX_PART];
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        char buf[200];
        snprintf(buf, sizeof(buf), "vortex reduction failed: %s", cudaGetErrorString(e));
        return set_error(LBM_ECUDA, buf);
    }
    lbm_vortex_info o{};
    o.intensity = h[0];
    o.intensity_abs = h[1];
    o.n_fluid = (int64_t)h[2];
    const double area_rate = (dx > 0.0 && dt > 0.0) ? dx * dx / dt : 0.0;
    o.intensity_phys = h[0] * area_rate;
    o.intensity_abs_phys = h[1] * area_rate;
    o.psi_max = h[3];
    o.psi_min = h[5];
    const int64_t imax = h[4] < 0.0 ? -1 : (int64_t)h[4];
    const int64_t imin = h[6] < 0.0 ? -1 : (int64_t)h[6];
    o.max_x = imax < 0 ? -1 : (int32_t)(imax % nx);
    o.max_y = imax < 0 ? -1 : (int32_t)(imax / nx);
    o.min_x = imin < 0 ? -1 : (int32_t)(imin % nx);
    o.min_y = imin < 0 ? -1 : (int32_t)(imin / nx);
    o.max_mm[0] = (o.max_x + 0.5) * dx * 1e3;
    o.max_mm[1] = (o.max_y + 0.5) * dx * 1e3;
    o.min_mm[0] = (o.min_x + 0.5) * dx * 1e3;
    o.min_mm[1] = (o.min_y + 0.5) * dx * 1e3;
    *out = o;
    return LBM_OK;
}
