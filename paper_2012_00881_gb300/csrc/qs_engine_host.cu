// Host side of the slice engine: occupancy, shared-memory sizing and the
// cooperative launches.  The kernels themselves are compiled in their own
// translation units (one per form), which hand out their launch handles.
#include <cuda_runtime.h>

#include "qs_cluster.cuh"
#include "qs_tile.cuh"

const void *qs_kernel_engine(int precision) {
    return precision == QS_FP32_REFINED ? qs_kernel_engine_fp32r() : qs_kernel_engine_fp64();
}

const void *qs_kernel_engine_batched(int precision) {
    return precision == QS_FP32_REFINED ? qs_kernel_engine_batched_fp32r()
                                        : qs_kernel_engine_batched_fp64();
}

int qs_engine_max_blocks(int device, int precision, size_t smem_bytes, int *blocks, int cluster) {
    const void *fn = qs_kernel_engine(precision);
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
    if (cluster > 1) {  // co-resident whole clusters (they must fit in the GPCs)
        if (cluster > 8 &&
            cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess)
            return -1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(sms - sms % cluster));
        cfg.blockDim = dim3(QS_ENGINE_THREADS);
        cfg.dynamicSmemBytes = smem_bytes;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) return -1;
        if (nc * cluster < *blocks) *blocks = nc * cluster;
    }
    return 0;
}

size_t qs_cluster_smem_bytes(const int *lev_n, int nlev, int cluster, int tsize) {
    return qsclu::cluster_layout(lev_n, nlev, cluster, tsize).total;
}

size_t qs_engine_smem_bytes(const int *lev_n, int nlev, int block_level_n, int precision,
                            int tile_x, int tile_y, int nu, int nu2, size_t *block_offset,
                            size_t *tile_offset) {
    int lg = 0;
    while (lg < nlev - 1 && lev_n[lg] > block_level_n) ++lg;
    const size_t inv = (qsmg::coarse_inv_bytes(lev_n, nlev) + 255) & ~(size_t)255;
    size_t b = precision == QS_FP32_REFINED ? qsmg::block_smem_bytes<float>(lev_n, nlev, lg, 2)
                                            : qsmg::block_smem_bytes<double>(lev_n, nlev, lg, 2);
    b = (b + 255) & ~(size_t)255;
    if (block_offset) *block_offset = inv;
    if (tile_offset) *tile_offset = b;  // relative to the block part
    size_t total = inv + b;
    if (precision == QS_FP32_REFINED && tile_x > 0)
        total += qstile::tile_smem_bytes(tile_x, tile_y, nu, nu2);
    else if (tile_x > 0)  // the float64 form's staged legs: six float64 arrays a region
        total += qstile::tile64_smem_bytes(tile_x, tile_y, nu, nu2);
    return total + 256;
}

cudaError_t qs_launch_engine_batched(cudaStream_t st, const EngineArgs *list, int n_inst,
                                     int precision, int team, int teams, BatchState *bs,
                                     size_t smem_bytes) {
    void *args[] = {(void *)&list, &n_inst, &team, &bs};
    const void *fn = qs_kernel_engine_batched(precision);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) !=
        cudaSuccess)
        return cudaGetLastError();
    return cudaLaunchCooperativeKernel(fn, dim3(team * teams), dim3(QS_ENGINE_THREADS), args,
                                       smem_bytes, st);
}

int qs_engine_batched_max_blocks(int device, int precision, size_t smem_bytes, int *blocks) {
    const void *fn = qs_kernel_engine_batched(precision);
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

cudaError_t qs_launch_engine(cudaStream_t st, const EngineArgs &a, int grid_blocks,
                             size_t smem_bytes) {
    EngineArgs copy = a;
    void *args[] = {&copy};
    const void *fn = qs_kernel_engine(a.precision);
    // the limit is a property of the kernel, shared by every context: set it
    // for this launch (another context may have set a smaller one)
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    if (a.cl_size <= 1)
        return cudaLaunchCooperativeKernel(fn, dim3(grid_blocks), dim3(QS_ENGINE_THREADS), args,
                                           smem_bytes, st);
    // cooperative (every block resident: the grid barrier) and clustered
    if (a.cl_size > 8) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid_blocks);
    cfg.blockDim = dim3(QS_ENGINE_THREADS);
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = (unsigned)a.cl_size;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelExC(&cfg, fn, args);
}
