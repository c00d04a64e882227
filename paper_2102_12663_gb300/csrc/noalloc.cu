// Observables of a domain's current state computed with the library's own
// device scratch instead of the per-tile partials region of the caller's
// domain buffer (lbm_read_observables_noalloc in include/lbm.h).
//
// Why it exists: some host applications hand this library a fixed block of
// device memory at start-up and allow no further device allocation afterwards
// (an embedding simulator with a hard memory budget, a latency-critical
// control loop in which an allocation would stall the device).  Such a caller
// can still read the observables here without reserving reduction scratch of
// its own: the per-row partial sums live in a file-scope device array that is
// part of the library image, so every GPU that loads the library holds it
// until the process exits.
//
// Limits and sharing: at most LBM_NOALLOC_MAX_ROWS grid rows (one partial
// slot per row); every call on a device shares the one array and it keeps the
// contents of the last call, so two calls that overlap on the GPU (different
// streams, no ordering between them) race on it.  Each row slot is fully
// rewritten before it is read, so nothing needs clearing between calls.
#include <cstdio>
#include <mutex>

#include "lbm.h"
#include "kernel_body.cuh"

namespace lbm {

// internal accessors of lbm_api.cu
lbm_status set_error(lbm_status s, const char* msg);
bool domain_parts(const lbm_domain* d, const InstDesc** desc, int* precision, int* ny,
                  int* parity, int* snap_valid, cudaStream_t* stream, int* device);
void fill_observables(const lbm_domain* d, const double* o, lbm_observables* out);

// One NPART-double partial per grid row, then the NOBS finalised values.
static __device__ __align__(256) double g_noalloc_scratch[(LBM_NOALLOC_MAX_ROWS + 1) * NPART];
static_assert((int)NOBS <= (int)NPART, "final observables must fit one slot");

template <class ST>
__global__ void __launch_bounds__(256) noalloc_rows_kernel(const InstDesc* __restrict__ insts,
                                                           int parity, int mode,
                                                           double* __restrict__ scratch) {
    __shared__ __align__(16) InstDesc sd;
    __shared__ double red[8][NPART];
    const int tid = threadIdx.x;
    {
        const uint64_t* src = reinterpret_cast<const uint64_t*>(insts);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&sd);
        for (int k = tid; k < (int)(sizeof(InstDesc) / 8); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    const int y = blockIdx.x;
    double acc[NPART];
#pragma unroll
    for (int k = 0; k < NPART; ++k) acc[k] = 0.0;
    for (int x = tid; x < sd.nx; x += blockDim.x) {
        if (parity) update_cell<ST, true, 1>(sd, x, y, mode, acc);
        else update_cell<ST, true, 0>(sd, x, y, mode, acc);
    }
    warp_block_reduce<double>(acc, red, scratch + (int64_t)y * NPART);
}

// Fixed-order fold of the row partials (thread-strided, then a binary tree).
__global__ void __launch_bounds__(256) noalloc_fold_kernel(const InstDesc* __restrict__ insts,
                                                           int ny, double* __restrict__ scratch) {
    __shared__ double sm[256][NPART];
    double acc[NPART];
    for (int k = 0; k < NPART; ++k) acc[k] = 0.0;
    for (int r = threadIdx.x; r < ny; r += blockDim.x) {
        const double* q = scratch + (int64_t)r * NPART;
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
    if (threadIdx.x == 0) {
        const double* a = sm[0];
        double* o = scratch + (int64_t)LBM_NOALLOC_MAX_ROWS * NPART;
        o[O_IOP] = a[P_N_FLUID] > 0.0 ? a[P_SUM_P] / a[P_N_FLUID] : 0.0;
        o[O_Q_IN] = a[P_Q_IN];
        o[O_Q_OUT] = a[P_Q_OUT];
        o[O_MASS] = a[P_MASS];
        o[O_PEAK] = sqrt(a[P_PEAK]);  // the partials hold max |u|^2
        o[O_WSS_C] = a[P_N_C] > 0.0 ? a[P_WSS_C] / a[P_N_C] : 0.0;
        o[O_WSS_I] = a[P_N_I] > 0.0 ? a[P_WSS_I] / a[P_N_I] : 0.0;
        o[O_RESID] = insts->snap_valid ? sqrt(a[P_RESID]) : -1.0;
        o[O_N_FLUID] = a[P_N_FLUID];
        o[O_N_C] = a[P_N_C];
        o[O_N_I] = a[P_N_I];
        o[O_NAN] = (a[P_NAN] > 0.0 || !isfinite(a[P_SUM_P]) || !isfinite(a[P_MASS])) ? 1.0 : 0.0;
    }
}

// Device address of the scratch array, looked up once per device with that
// device current (the host-side name of a __device__ variable is only a
// stand-in and must never be handed to a kernel).
static constexpr int MAX_DEVICES = 64;
static double* g_scratch_ptr[MAX_DEVICES];
static std::mutex g_scratch_mu;

static cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace lbm

using namespace lbm;

static lbm_status cuda_fail(const char* what, cudaError_t e) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s failed: %s", what, cudaGetErrorString(e));
    return set_error(LBM_ECUDA, buf);
}

extern "C" lbm_status lbm_read_observables_noalloc(lbm_domain* dom, lbm_observables* out) {
    const InstDesc* desc = nullptr;
    int prec = 0, ny = 0, parity = 0, snap_valid = 0, device = 0, current = 0;
    cudaStream_t s = nullptr;
    if (!out) return set_error(LBM_EINVAL, "null output");
    if (!domain_parts(dom, &desc, &prec, &ny, &parity, &snap_valid, &s, &device)) return LBM_EINVAL;
    // the scratch address below is the current device's: it must be the
    // domain's (a device switch since lbm_create_domain would hand the kernels
    // another device's address)
    cudaError_t e = cudaGetDevice(&current);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    if (current != device) {
        char buf[160];
        snprintf(buf, sizeof(buf),
                 "the current device is %d but the domain was created on device %d; make it "
                 "current before lbm_read_observables_noalloc", current, device);
        return set_error(LBM_EINVAL, buf);
    }
    if (ny > LBM_NOALLOC_MAX_ROWS) {
        char buf[160];
        snprintf(buf, sizeof(buf),
                 "grid has %d rows; lbm_read_observables_noalloc supports at most %d "
                 "(use lbm_read_observables)", ny, LBM_NOALLOC_MAX_ROWS);
        return set_error(LBM_EINVAL, buf);
    }
    double* scratch = nullptr;
    e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return cuda_fail("cudaGetSymbolAddress of the scratch array", e);
    const int mode = OBS_STATS | (snap_valid ? OBS_RESID : 0);
    switch (prec) {
    case LBM_F64: noalloc_rows_kernel<StF64><<<ny, 256, 0, s>>>(desc, parity, mode, scratch); break;
    case LBM_F32: noalloc_rows_kernel<StF32><<<ny, 256, 0, s>>>(desc, parity, mode, scratch); break;
    case LBM_F16DEV: noalloc_rows_kernel<StF16><<<ny, 256, 0, s>>>(desc, parity, mode, scratch); break;
    default: noalloc_rows_kernel<StBF16><<<ny, 256, 0, s>>>(desc, parity, mode, scratch); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("row reduction launch", e);
    noalloc_fold_kernel<<<1, 256, 0, s>>>(desc, ny, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail("fold launch", e);
    double o[NOBS];
    if ((e = cudaMemcpyAsync(o, scratch + (int64_t)LBM_NOALLOC_MAX_ROWS * NPART, sizeof(o),
                             cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail("observables copy", e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail("stream synchronize", e);
    fill_observables(dom, o, out);
    return LBM_OK;
}
