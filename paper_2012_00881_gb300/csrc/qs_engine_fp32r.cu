// The refined form of slice_engine in a translation unit of its own (the
// kernels are large; separate units compile in parallel).
#include "qs_engine.cuh"

const void *qs_kernel_engine_fp32r() { return (const void *)slice_engine<true>; }
