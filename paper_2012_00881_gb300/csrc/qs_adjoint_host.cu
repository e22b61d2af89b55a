// Host side of the adjoint engine: occupancy and the cooperative launch.
// The kernels are compiled in their own translation units (one per form).
#include <cuda_runtime.h>

#include "qs_internal.cuh"

const void *qs_kernel_adjoint(int precision) {
    return precision == QS_FP32_REFINED ? qs_kernel_adjoint_fp32r() : qs_kernel_adjoint_fp64();
}

int qs_adjoint_max_blocks(int device, int precision, size_t smem_bytes, int *blocks) {
    const void *fn = qs_kernel_adjoint(precision);
    int per_sm = 0, sms = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) !=
        cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, QS_ENGINE_THREADS,
                                                      smem_bytes) != cudaSuccess)
        return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return -1;
    *blocks = per_sm * sms;
    return 0;
}

cudaError_t qs_launch_adjoint(cudaStream_t st, const EngineArgs &a, const AdjArgs &d,
                              int grid_blocks, size_t smem_bytes) {
    EngineArgs ca = a;
    AdjArgs cd = d;
    void *args[] = {&ca, &cd};
    const void *fn = qs_kernel_adjoint(a.precision);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(fn, dim3(grid_blocks), dim3(QS_ENGINE_THREADS), args,
                                       smem_bytes, st);
}
