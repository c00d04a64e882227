// FP64 instantiation of the fused step.  Compiled with -fmad=false so that no
// multiply-add is contracted: the arithmetic then matches a sequential FP64
// evaluation of the model operation for operation.
#include "kernel_body.cuh"

namespace lbm {

StepPlan step_plan_f64(int mode, Shape shape) {
    StepPlan p;
    p.func = mode != 0 ? reinterpret_cast<const void*>(&step_kernel<StF64, true>)
                 : reinterpret_cast<const void*>(&step_kernel<StF64, false>);
    p.block = dim3(shape.tw, shape.bh);
    p.smem = 0;
    return p;
}

StepPlan flow_plan_f64(Shape shape, bool keep) {
    StepPlan p;
    p.func = keep ? reinterpret_cast<const void*>(&step_kernel_flow<StF64T<ST_KEEP>>)
                  : reinterpret_cast<const void*>(&step_kernel_flow<StF64>);
    p.block = dim3(shape.tw, shape.bh);
    p.smem = 0;
    return p;
}

}  // namespace lbm
