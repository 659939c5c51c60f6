// npw_fp64.cu -- double-precision instantiation of the kernels (NPW_FP64).  Built with
// --fmad=false so that every product and sum is rounded on its own, in the written order.
#include "npw_kernels.cuh"
#define NPW_R double
#include "npw_instantiate.inc"
