// npw_noalloc.cu -- npweno_rk3_step_noalloc: the TVD-RK3 step of npweno_rk3_step for callers
// that cannot allocate device memory, with its scratch in a fixed array owned by this library.
//
// Some callers hold device pointers to their state but have no way to allocate device memory
// at the point where they call the solver: code inside a host framework that hands out
// pre-placed buffers and reserves the rest of the GPU for its own pool, or callers in a
// memory-capped share of the GPU where an allocation during the run could fail.  For them the
// scratch that npweno_rk3_step takes as `workspace` (two stage buffers, the instance table,
// the control words and the tile table) lives here, in one file-scope device array that every
// GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "npw_internal.h"
#include "npweno.h"

namespace {

// Size of the fixed scratch array: 8 MiB.
constexpr size_t kScratchBytes = size_t(8) << 20;

static __device__ __align__(256) unsigned char g_npw_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The first call on a device
// looks it up with cudaGetSymbolAddress (the array's name in host code is only a host-side
// stand-in, never a device address) and caches it.  The cache is not invalidated by
// cudaDeviceReset (which reloads the module): calls after a reset are not supported.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_npw_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" {

size_t npw_noalloc_scratch_bytes(void) { return kScratchBytes; }

npw_status npweno_rk3_step_noalloc(void* u, int64_t n, int32_t m, double dx, double dt, int32_t flux_kind,
                                   int32_t bc, const npw_params* params, void* stream) {
    if (!params) return npw::set_error(NPW_EINVAL, "params is NULL");
    const size_t need = npw_workspace_size(n, m, params);
    if (need > kScratchBytes)
        return npw::set_error(NPW_EINVAL,
                              "npweno_rk3_step_noalloc: n * m too large for the fixed 8 MiB scratch "
                              "(use npweno_rk3_step with a caller workspace)");
    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return npw::set_error(NPW_ECUDA, cudaGetErrorString(e));
    return npweno_rk3_step(u, n, m, dx, dt, flux_kind, bc, params, scratch, kScratchBytes, nullptr, stream);
}

}  // extern "C"
