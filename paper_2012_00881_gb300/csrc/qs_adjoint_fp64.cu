// The float64 form of adjoint_engine in a translation unit of its own (the
// kernels are large; separate units compile in parallel).
// the adjoint launch has no thread-block clusters
#define QS_NO_CLUSTER_SOLVES
#include "qs_adjoint.cuh"

const void *qs_kernel_adjoint_fp64() { return (const void *)adjoint_engine<false>; }
