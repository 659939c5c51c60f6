// npw_queue_fp32.cu -- the work-queue kernels of the mixed-precision path (NPW_FP32_MIXED),
// built like npw_fp32.cu (--fmad=false: the queue items give the bits of the other kernels).
#include "npw_kernels.cuh"
#define NPW_R float
#include "npw_queue.inc"
