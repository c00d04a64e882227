// FP64 instantiation of the fused step.  Compiled with -fmad=false so that no
// multiply-add is contracted: the arithmetic then matches a sequential FP64
// evaluation of the model operation for operation.
#include "kernel_body.cuh"

namespace lbm {

cudaError_t launch_step_f64(const InstDesc* insts, const int4* tiles, int ntiles, int flip,
                            int mode, Shape shape, int grid, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    dim3 block(shape.tw, shape.bh);
    if (mode == 0) step_kernel<StF64, false><<<grid, block, 0, s>>>(insts, tiles, ntiles, flip, 0, shape);
    else step_kernel<StF64, true><<<grid, block, 0, s>>>(insts, tiles, ntiles, flip, mode, shape);
    return cudaGetLastError();
}

const void* step_kernel_ptr_f64(bool obs) {
    return obs ? reinterpret_cast<const void*>(&step_kernel<StF64, true>)
               : reinterpret_cast<const void*>(&step_kernel<StF64, false>);
}

}  // namespace lbm
