// FP32-arithmetic instantiations of the fused step: FP32 storage and the two
// 16-bit deviation storages (FP16 scaled, BF16).  Plain steps of launch shapes
// with one row of threads per block and tiles at least 64 cells wide take the
// staged kernel (persistent: its grid is capped at the blocks the device
// holds at once); observing steps and other shapes take the direct kernel.
#include <algorithm>

#include "kernel_body.cuh"

namespace lbm {

// precision code of a storage trait (1 f32, 2 f16-dev, 3 bf16-dev)
template <class ST>
static constexpr int storage_precision() {
    return sizeof(typename ST::T) == 4 ? 1 : (std::is_same<typename ST::T, __half>::value ? 2 : 3);
}

template <class ST>
static StepPlan plan_t(int mode, Shape shape) {
    const bool obs = mode != 0;
    StepPlan p;
    if (!obs && shape.bh == 1 && shape.tw >= WS_SEG) {
        const void* f = reinterpret_cast<const void*>(&step_kernel_ws<ST>);
        p.func = f;
        p.block = dim3(WS_THREADS);
        p.smem = (size_t)ws_smem_bytes<typename ST::T>();
        // co-resident blocks, per device (set once per device and storage)
        static int cap[64] = {};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
        if (cap[dev] == 0) {
            int per_sm = 0, sms = 0;
            if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) ==
                    cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, WS_THREADS, p.smem) == cudaSuccess &&
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
                cap[dev] = std::max(per_sm, 1) * std::max(sms, 1);
            else
                cap[dev] = -1;
        }
        p.max_grid = cap[dev] > 0 ? cap[dev] : 1;
    } else {
        // the steady-state check step (observe and write) folds its partials
        // in FP32 per warp; observe-only reads keep FP64 partials
        // 16-bit storages: the eight-cell vector path (256-wide tiles) keeps 13
        // planes of four packed words live and is built for 2 blocks of 256
        // threads (128 registers); the other shapes for 3 (85 registers: more
        // warps to hide memory latency)
        // Plain steps: the 16-bit storages always with edge-cell chunks (their
        // vector rows would otherwise send up to 256 cells to the per-cell
        // update for one boundary cell); FP32 as the host chose for the grid
        const void* plain = nullptr;
        bool split = true;
        if constexpr (sizeof(typename ST::T) == 2) {
            plain = shape.tw == 256 ? reinterpret_cast<const void*>(&step_kernel<ST, false, double, 2, true>)
                                    : reinterpret_cast<const void*>(&step_kernel<ST, false, double, 3, true>);
        } else {
            split = shape.split != 0;
            plain = split ? reinterpret_cast<const void*>(&step_kernel<ST, false, double, 0, true>)
                          : reinterpret_cast<const void*>(&step_kernel<ST, false>);
        }
        p.func = !obs ? plain
                 : (mode & OBS_WRITE) ? reinterpret_cast<const void*>(&step_kernel<ST, true, typename ST::A>)
                                      : reinterpret_cast<const void*>(&step_kernel<ST, true>);
        p.block = dim3(shape.tw / cells_per_thread(storage_precision<ST>(), shape.tw), shape.bh);
        p.smem = 0;
        p.edges = !obs && split;  // runs the edge-cell chunks
    }
    return p;
}

StepPlan step_plan_lp(int precision, int mode, Shape shape) {
    switch (precision) {
    case 1: return plan_t<StF32>(mode, shape);
    case 2: return plan_t<StF16>(mode, shape);
    default: return plan_t<StBF16>(mode, shape);
    }
}

template <class ST>
static StepPlan flow_t(Shape shape) {
    StepPlan p;
    // the same choice of paths as the per-step kernels (plan_t)
    if constexpr (sizeof(typename ST::T) == 2) {
        p.func = shape.tw == 256 ? reinterpret_cast<const void*>(&step_kernel_flow<ST, 2, true>)
                                 : reinterpret_cast<const void*>(&step_kernel_flow<ST, 3, true>);
    } else {
        p.func = shape.split ? reinterpret_cast<const void*>(&step_kernel_flow<ST, 0, true>)
                             : reinterpret_cast<const void*>(&step_kernel_flow<ST>);
    }
    p.block = dim3(shape.tw / cells_per_thread(storage_precision<ST>(), shape.tw), shape.bh);
    p.smem = 0;
    return p;
}

StepPlan flow_plan_lp(int precision, Shape shape, bool keep) {
    switch (precision) {
    case 1: return keep ? flow_t<StF32T<ST_KEEP>>(shape) : flow_t<StF32>(shape);
    case 2: return keep ? flow_t<StF16T<ST_KEEP>>(shape) : flow_t<StF16>(shape);
    default: return keep ? flow_t<StBF16T<ST_KEEP>>(shape) : flow_t<StBF16>(shape);
    }
}

}  // namespace lbm

namespace lbm {
// Reads and clears the status word of the staged kernels (0 = fine).
cudaError_t take_step_status(int* status) {
    cudaError_t e = cudaMemcpyFromSymbol(status, g_step_status, sizeof(int));
    if (e != cudaSuccess || *status == 0) return e;
    const int zero = 0;
    return cudaMemcpyToSymbol(g_step_status, &zero, sizeof(int));
}
}  // namespace lbm
