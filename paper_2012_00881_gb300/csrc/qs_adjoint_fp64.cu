// The float64 form of adjoint_engine in a translation unit of its own (the
// kernels are large; separate units compile in parallel).
#include "qs_adjoint.cuh"

const void *qs_kernel_adjoint_fp64() { return (const void *)adjoint_engine<false>; }
