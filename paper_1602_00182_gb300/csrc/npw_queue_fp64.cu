// npw_queue_fp64.cu -- the work-queue kernels of the double-precision path (NPW_FP64), built
// like npw_fp64.cu (--fmad=false).
#include "npw_kernels.cuh"
#define NPW_R double
#include "npw_queue.inc"
