// FP32-arithmetic instantiations of the fused step: FP32 storage and the two
// 16-bit deviation storages (FP16 scaled, BF16).
#include "kernel_body.cuh"

namespace lbm {

template <class ST>
static cudaError_t launch_t(const InstDesc* insts, const int4* tiles, int ntiles, int flip, int mode,
                            Shape shape, int grid, cudaStream_t s) {
    dim3 block(shape.tw, shape.bh);
    if (mode == 0) step_kernel<ST, false><<<grid, block, 0, s>>>(insts, tiles, ntiles, flip, 0, shape);
    else step_kernel<ST, true><<<grid, block, 0, s>>>(insts, tiles, ntiles, flip, mode, shape);
    return cudaGetLastError();
}

cudaError_t launch_step_lp(int precision, const InstDesc* insts, const int4* tiles, int ntiles,
                           int flip, int mode, Shape shape, int grid, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    switch (precision) {
    case 1: return launch_t<StF32>(insts, tiles, ntiles, flip, mode, shape, grid, s);
    case 2: return launch_t<StF16>(insts, tiles, ntiles, flip, mode, shape, grid, s);
    case 3: return launch_t<StBF16>(insts, tiles, ntiles, flip, mode, shape, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

const void* step_kernel_ptr_lp(int precision, bool obs) {
    switch (precision) {
    case 1: return obs ? (const void*)&step_kernel<StF32, true> : (const void*)&step_kernel<StF32, false>;
    case 2: return obs ? (const void*)&step_kernel<StF16, true> : (const void*)&step_kernel<StF16, false>;
    case 3: return obs ? (const void*)&step_kernel<StBF16, true> : (const void*)&step_kernel<StBF16, false>;
    default: return nullptr;
    }
}

}  // namespace lbm
