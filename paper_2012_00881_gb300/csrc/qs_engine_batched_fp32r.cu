// The refined form of slice_engine_batched in a translation unit of its own (the
// kernels are large; separate units compile in parallel).
// the batched launch has no thread-block clusters
#define QS_NO_CLUSTER_SOLVES
#include "qs_engine.cuh"

const void *qs_kernel_engine_batched_fp32r() { return (const void *)slice_engine_batched<true>; }
