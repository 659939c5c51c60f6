// npw_format.cu -- npw_format_check: the integer float<->double format changes of the
// mixed-precision shape parameter (fast::widen, widen_nz, narrow, seed_f) run next to the
// hardware conversions, so that tests can check them on every float class.
#include <cuda_runtime.h>

#include "npw_fast.cuh"
#include "npw_internal.h"
#include "npweno.h"

namespace npw {
// One element per thread: the library's integer format changes next to the hardware ones.
__global__ void format_check_kernel(const float* __restrict__ f_in, const double* __restrict__ d_in,
                                           int64_t count, double* widen_out, double* widen_nz_out, float* narrow_out,
                                           float* seed_out, int32_t* flags_out, double* hw_widen_out,
                                           float* hw_narrow_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float x = f_in[i];
    const double d = d_in[i];
    const bool nz = fast::zero_or_normal(x);
    widen_out[i] = fast::widen(x);
    widen_nz_out[i] = nz ? fast::widen_nz(x) : 0.0;
    narrow_out[i] = fast::narrow(d);
    float sf;
    const bool ok = fast::seed_f(d, &sf);
    seed_out[i] = sf;
    flags_out[i] = (nz ? 1 : 0) | (ok ? 2 : 0);
    hw_widen_out[i] = (double)x;
    hw_narrow_out[i] = (float)d;
}

static cudaError_t launch_format_check(const float* f_in, const double* d_in, int64_t count, double* widen_out,
                                double* widen_nz_out, float* narrow_out, float* seed_out, int32_t* flags_out,
                                double* hw_widen_out, float* hw_narrow_out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (count + threads - 1) / threads;
    format_check_kernel<<<(unsigned)blocks, threads, 0, st>>>(f_in, d_in, count, widen_out, widen_nz_out, narrow_out,
                                                              seed_out, flags_out, hw_widen_out, hw_narrow_out);
    return cudaGetLastError();
}
}  // namespace npw

extern "C" npw_status npw_format_check(const float* f_in, const double* d_in, int64_t count, double* widen_out,
                                       double* widen_nz_out, float* narrow_out, float* seed_out, int32_t* flags_out,
                                       double* hw_widen_out, float* hw_narrow_out, void* stream) {
    if (count < 0) return npw::set_error(NPW_EINVAL, "npw_format_check: count < 0");
    if (count > ((int64_t)1 << 31) * 255)
        return npw::set_error(NPW_EINVAL, "npw_format_check: count too large for one launch");
    if (count > 0 && (!f_in || !d_in || !widen_out || !widen_nz_out || !narrow_out || !seed_out || !flags_out ||
                      !hw_widen_out || !hw_narrow_out))
        return npw::set_error(NPW_EINVAL, "npw_format_check: null pointer");
    const cudaError_t e = npw::launch_format_check(f_in, d_in, count, widen_out, widen_nz_out, narrow_out, seed_out,
                                                   flags_out, hw_widen_out, hw_narrow_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return npw::set_error(NPW_ECUDA, cudaGetErrorString(e));
    return NPW_OK;
}
