// npw_fp32.cu -- mixed-precision instantiation (NPW_FP32_MIXED): float state, candidates,
// weights, flux and update; shape parameter, switch, ENO choice and smoothness indicators
// in double from the float cell averages.
#include "npw_kernels.cuh"
#define NPW_R float
#include "npw_instantiate.inc"

namespace npw {
// per field: u^n, d1 and d2 with their ghost cells
size_t resident_smem_bytes(int64_t n, int m) {
    return (size_t)m * (size_t)(3 * (n + 2 * RES_GHOST)) * sizeof(float);
}

template <int KIND, int K>
static cudaError_t launch_res(const ResidentArgs& a, int64_t max_n, int threads, cudaStream_t s) {
    constexpr int M = kind_m<KIND>();
    const size_t smem = resident_smem_bytes(max_n, M);
    auto kern = solve1d_resident_kernel<KIND, K>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RESIDENT_SMEM_MAX);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    kern<<<a.count, threads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_resident_f32(const ResidentArgs& a, int m, int kind, int64_t max_n, int threads, cudaStream_t s) {
    (void)m;
    if (resident_smem_bytes(max_n, kind == NPW_FLUX_EULER1D ? 3 : 1) > RESIDENT_SMEM_MAX) return cudaErrorInvalidValue;
    switch (kind) {
        case NPW_FLUX_ADVECTION:
            return a.mp.k == 2 ? launch_res<NPW_FLUX_ADVECTION_, 2>(a, max_n, threads, s)
                               : launch_res<NPW_FLUX_ADVECTION_, 3>(a, max_n, threads, s);
        case NPW_FLUX_BURGERS:
            return a.mp.k == 2 ? launch_res<NPW_FLUX_BURGERS_, 2>(a, max_n, threads, s)
                               : launch_res<NPW_FLUX_BURGERS_, 3>(a, max_n, threads, s);
        case NPW_FLUX_EULER1D:
            return a.mp.k == 2 ? launch_res<NPW_FLUX_EULER1D_, 2>(a, max_n, threads, s)
                               : launch_res<NPW_FLUX_EULER1D_, 3>(a, max_n, threads, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace npw

namespace npw {
cudaError_t launch_comp_begin(const float* u, float* s, float* c, const InstDev* inst, const Tile* tiles, int ntiles,
                              int tile, int m, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    comp_copy_kernel<<<ntiles, THREADS_1D, 0, st>>>(s, u, c, inst, tiles, tile, m, nullptr);
    return cudaGetLastError();
}
cudaError_t launch_comp_end(float* u, const float* s, const InstDev* inst, const Tile* tiles, int ntiles, int tile,
                            int m, const Ctl* odd, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    comp_copy_kernel<<<ntiles, THREADS_1D, 0, st>>>(u, s, nullptr, inst, tiles, tile, m, odd);
    return cudaGetLastError();
}
}  // namespace npw
