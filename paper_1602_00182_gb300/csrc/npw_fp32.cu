// npw_fp32.cu -- mixed-precision instantiation (NPW_FP32_MIXED): float state, candidates,
// weights, flux and update; shape parameter, switch, ENO choice and smoothness indicators
// in double from the float cell averages.
#include "npw_kernels.cuh"
#define NPW_R float
#include "npw_instantiate.inc"
