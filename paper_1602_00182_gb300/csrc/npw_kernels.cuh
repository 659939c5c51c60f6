// npw_kernels.cuh -- CUDA kernels of libnpweno, templated on the state type.  Included by one
// translation unit per precision (npw_fp64.cu, npw_fp32.cu), which instantiate the launchers.
//
// The hot kernel is stage1d_kernel: one CTA per (instance, tile) work item runs one whole
// TVD-RK3 stage of its tile -- halo load with the boundary mapping, the per-face shape
// parameter / switch / candidates / weights (Sec. 2-4), the Lax-Friedrichs flux (Sec. 5.1),
// the flux difference of eq. PDE1 and the Shu-Osher stage combination -- and, in stage 3,
// the block reduction of the next Lax-Friedrichs alpha and the per-instance time control.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "npw_device.cuh"
#include "npw_fast.cuh"
#include "npw_internal.h"

namespace npw {

// value of cell k (any integer) of a line of n cells with stride `stride`; BC by index map
template <typename R>
__device__ __forceinline__ R line_get(const R* u, int64_t n, int64_t stride, int64_t k, int bc, double inflow) {
    if (bc == NPW_BC_PERIODIC) {
        int64_t kk = k % n;
        if (kk < 0) kk += n;
        return u[kk * stride];
    }
    if (k < 0) return (bc == NPW_BC_INFLOW) ? R(inflow) : u[0];
    if (k >= n) return u[(n - 1) * stride];
    return u[k * stride];
}

// Index of cell k of a line of n cells for a tile halo (k in [-3, n + 2], n >= 6), or -1 for
// the inflow state: periodic images, repeated end cells, inflow on the left
__device__ __forceinline__ int64_t halo_idx(int64_t n, int64_t k, int bc) {
    if (bc == NPW_BC_PERIODIC) return k < 0 ? k + n : (k >= n ? k - n : k);
    if (k < 0) return bc == NPW_BC_INFLOW ? -1 : 0;
    return k >= n ? n - 1 : k;
}

template <typename R>
__device__ __forceinline__ bool finite_(R x) {
    return x - x == R(0.0);
}

// Adds this warp's decision counts to the instance's control word (one atomic per nonzero
// counter and warp).  Every lane of the warp must call it; schemes without a shape parameter
// add nothing.
__device__ __forceinline__ void flush_counts(const EtaCount& c, Ctl* ctl, const MethodParams& mp) {
    if (mp.scheme != NPW_RBF_ENO_ && mp.scheme != NPW_RBF_WENO_) return;
    const unsigned sw = __reduce_add_sync(0xffffffffu, c.sw), ev = __reduce_add_sync(0xffffffffu, c.ev);
    const unsigned gd = __reduce_add_sync(0xffffffffu, c.guard), bd = __reduce_add_sync(0xffffffffu, c.bound);
    if ((threadIdx.x & 31) == 0) {
        if (sw) atomicAdd(&ctl->n_switch, (unsigned long long)sw);
        if (ev) atomicAdd(&ctl->n_eval, (unsigned long long)ev);
        if (gd) atomicAdd(&ctl->n_guard, (unsigned long long)gd);
        if (bd) atomicAdd(&ctl->n_bound, (unsigned long long)bd);
    }
}

// A face is counted once per line: by the tile (or warp) whose cells start at it, and the last
// face n by the tile that ends there.  q = local face index (face between local cells q-1 and
// q), cnt = cells of the tile, last = the tile ends the line.
__device__ __forceinline__ bool face_owned(int q, int cnt, bool last) {
    return (q >= 0 && q < cnt) || (q == cnt && last);
}

// Weights of the last Shu-Osher stage, u^{n+1} = w1 u^n + w2 (u2 + dt L(u2)).  They must sum to
// one exactly, or every step scales the conserved sum: in float, RN(1/3) + RN(2/3) = 1 + 3e-8,
// so the float kernels take w2 = RN(2/3) and w1 = 1 - w2 (exact).  Double keeps 1/3 and 2/3
// (their rounded sum differs from one by 1e-17, below the FP64 path's other rounding).
constexpr float kTwoThirdsF = 2.0f / 3.0f;
constexpr float kThirdF = 1.0f - kTwoThirdsF;
template <typename R>
__device__ __forceinline__ R stage3_w1() {
    return sizeof(R) == sizeof(float) ? R(kThirdF) : R(1.0 / 3.0);
}
template <typename R>
__device__ __forceinline__ R stage3_w2() {
    return sizeof(R) == sizeof(float) ? R(kTwoThirdsF) : R(2.0 / 3.0);
}

// max over the block of a non-negative speed; any non-finite input makes the result NaN
__device__ __forceinline__ double block_max_nan(double v, bool bad, double* red, int* redbad) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    unsigned b = __ballot_sync(0xffffffffu, bad);
    if (lane == 0) {
        red[warp] = v;
        redbad[warp] = b != 0u;
    }
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x == 0) {
        int anybad = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            out = red[w] > out ? red[w] : out;
            anybad |= redbad[w];
        }
        if (anybad) out = __longlong_as_double(0x7ff8000000000000ll);
    }
    return out;  // valid in thread 0
}

// The same maximum over float values (exact, so equal to the maximum of their widened
// values), taken with float comparisons; one conversion of the result in thread 0.
__device__ __forceinline__ double block_max_nan_f(float v, bool bad, float* red, int* redbad) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    const unsigned b = __ballot_sync(0xffffffffu, bad);
    if (lane == 0) {
        red[warp] = v;
        redbad[warp] = b != 0u;
    }
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x == 0) {
        float m = 0.0f;
        int anybad = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            m = red[w] > m ? red[w] : m;
            anybad |= redbad[w];
        }
        out = anybad ? __longlong_as_double(0x7ff8000000000000ll) : (double)m;
    }
    return out;  // valid in thread 0
}

// ---------------------------------------------------------------------------------------
// time control, executed by one thread for one instance
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void next_dt(Ctl* c, double rate, double t_end, double cfl) {
    double dt = (rate > 0.0) ? cfl / rate : t_end - c->t;
    int last = 0;
    if (c->t + dt * (1.0 + 1e-10) >= t_end) {
        dt = t_end - c->t;
        last = 1;
    }
    c->dt = dt;
    c->last = last;
}

__device__ __forceinline__ bool take_alpha(Ctl* c, double* ax, double* ay, bool two_d) {
    *ax = __longlong_as_double((long long)c->alpha_next_bits);
    *ay = two_d ? __longlong_as_double((long long)c->alpha_y_next_bits) : 0.0;
    c->alpha_next_bits = 0ull;
    c->alpha_y_next_bits = 0ull;
    bool ok = (*ax - *ax == 0.0) && (*ay - *ay == 0.0);
    if (!ok) {
        c->status = NPW_ENONFINITE;
        c->done = 1;
        return false;
    }
    c->alpha = *ax;
    c->alpha_y = *ay;
    double m = *ax > *ay ? *ax : *ay;
    c->alpha_max = m > c->alpha_max ? m : c->alpha_max;
    return true;
}

// the step limit or a time that no longer advances ends the run (see step_cap)
__device__ __forceinline__ void check_progress(Ctl* c) {
    if (c->steps >= c->step_cap || !(c->t + c->dt > c->t)) {
        c->status = NPW_ETIMEOUT;
        c->done = 1;
    }
}

__device__ __forceinline__ void finalize_1d(Ctl* c, const InstDev& in) {
    c->tiles_done = 0u;
    c->steps += 1;
    c->t = c->last ? in.t_end : c->t + c->dt;
    double ax, ay;
    if (!take_alpha(c, &ax, &ay, false)) return;
    if (c->last) {
        c->done = 1;
        return;
    }
    next_dt(c, ax / in.dx, in.t_end, in.cfl);
    check_progress(c);
}

__device__ __forceinline__ void finalize_2d(Ctl* c, const Inst2D& in) {
    c->tiles_done = 0u;
    c->steps += 1;
    c->t = c->last ? in.t_end : c->t + c->dt;
    double ax, ay;
    if (!take_alpha(c, &ax, &ay, true)) return;
    if (c->last) {
        c->done = 1;
        return;
    }
    next_dt(c, ax / in.dx + ay / in.dy, in.t_end, in.cfl);
    check_progress(c);
}

// ---------------------------------------------------------------------------------------
// npweno_reconstruct: one thread per face, all fields.  The flag byte also carries the
// near-tie bit of every decision at the face (face_near_tie; characteristic: on the projected
// fields), and eta (optional) the shape parameters as used.
// ---------------------------------------------------------------------------------------
template <typename R, typename D, int M, bool CHAR>
__global__ void reconstruct_kernel(const R* __restrict__ u, int64_t n, int bc, MethodParams mp, R* __restrict__ vm,
                                   R* __restrict__ vp, uint8_t* __restrict__ flags, R* __restrict__ eta) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f > n) return;
    R S[6 * M];
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
        for (int k = 0; k < M; ++k) S[j * M + k] = line_get<R>(u + k * n, n, 1, f - 3 + j, bc, mp.inflow[k]);
    R a[M], b[M], e[M];
    uint32_t fl[M];
    bool ok = face_all<R, D, NPW_FLUX_EULER1D_, M, CHAR>(S, mp, a, b, fl, (const D*)nullptr, e);
    if (flags) {
        R line[M][6];
        if constexpr (CHAR) {
            R Rm[3][3], Lm[3][3];
            euler_eig<R>(S + 2 * M, S + 3 * M, mp_val<R>(mp.gamma, mp.gamma_f), Rm, Lm);
#pragma unroll
            for (int q = 0; q < M; ++q)
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    R s = R(0.0);
#pragma unroll
                    for (int k = 0; k < M; ++k) s += Lm[q][k] * S[j * M + k];
                    line[q][j] = s;
                }
        } else {
#pragma unroll
            for (int k = 0; k < M; ++k)
#pragma unroll
                for (int j = 0; j < 6; ++j) line[k][j] = S[j * M + k];
        }
#pragma unroll
        for (int k = 0; k < M; ++k)
            if (face_near_tie<R>(line[k], mp, mp.tie_tol)) fl[k] |= FL_NEAR_TIE;
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        R nan = R(__longlong_as_double(0x7ff8000000000000ll));
        vm[k * (n + 1) + f] = ok ? a[k] : nan;
        vp[k * (n + 1) + f] = ok ? b[k] : nan;
        if (flags) flags[k * (n + 1) + f] = flag_byte(fl[k]);
        if (eta) eta[k * (n + 1) + f] = ok ? e[k] : nan;
    }
}

// npweno_flux: one thread per face
template <typename R, int KIND>
__global__ void flux_kernel(const R* __restrict__ vm, const R* __restrict__ vp, int64_t nf, R alpha, MethodParams mp,
                            R* __restrict__ h) {
    constexpr int M = kind_m<KIND>();
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    R a[M], b[M], o[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
        a[k] = vm[k * nf + f];
        b[k] = vp[k * nf + f];
    }
    lf_flux<R, KIND, M>(a, b, alpha, mp, 0, o);
#pragma unroll
    for (int k = 0; k < M; ++k) h[k * nf + f] = o[k];
}

// alpha^0 = max |f'(u^0)| per instance: every tile adds its maximum by atomicMax on the
// bits of the non-negative double (the bit order of non-negative doubles is their order).
template <typename R, int KIND>
__global__ void __launch_bounds__(THREADS_1D) alpha_init_kernel(const R* __restrict__ u, const InstDev* __restrict__ inst,
                                                                 Ctl* ctl, const Tile* __restrict__ tiles, int tile,
                                                                 MethodParams mp) {
    constexpr int M = kind_m<KIND>();
    __shared__ double red[32];
    __shared__ int redbad[32];
    const Tile td = tiles[blockIdx.x];
    const InstDev in = inst[td.inst];
    const int64_t n = in.n;
    const int c0 = td.start;
    const int cnt = (int)((n - c0) < tile ? (n - c0) : tile);
    const R* base = u + in.off;
    double vmax = 0.0;
    bool bad = false;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        R U[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            U[k] = base[k * n + c0 + q];
            bad |= !finite_(U[k]);
        }
        double s = (double)wave_speed<R, KIND>(U, mp, 0);
        bad |= !finite_(s);
        vmax = s > vmax ? s : vmax;
    }
    double b = block_max_nan(vmax, bad, red, redbad);
    if (threadIdx.x == 0) atomicMax(&ctl[td.inst].alpha_next_bits, (unsigned long long)__double_as_longlong(b));
}

// ---------------------------------------------------------------------------------------
// The fused stage kernel (1D).  Shared memory: su[(tile + 6) * M] cell-major stage input
// with 3 ghost cells per side, sh[(tile + 1) * M] face fluxes.
// ---------------------------------------------------------------------------------------
// One work item (instance td.inst, tile starting at cell td.start) of one stage; the CTA calls
// it together.  smem: (a.tile + 6 + a.tile + 1) * M elements of R.
template <typename R, typename D, int KIND, bool CHAR>
__device__ __forceinline__ void stage1d_body(const Stage1DArgs& a, const Tile td, const InstDev& in, Ctl* ctl,
                                             unsigned char* smem_raw) {
    constexpr int M = kind_m<KIND>();
    __shared__ double red[32];
    __shared__ int redbad[32];
    R* su = reinterpret_cast<R*>(smem_raw);
    R* sh = su + (a.tile + 6) * M;
    if (*(volatile int32_t*)&ctl->done) return;  // uniform over the CTA
    const int64_t n = in.n;
    const int c0 = td.start;
    const int cnt = (int)((n - c0) < a.tile ? (n - c0) : a.tile);
    const R* uin = reinterpret_cast<const R*>(a.uin) + in.off;
    const int span = cnt + 6;

    // halo load: cell c0 - 3 + j, field k; consecutive threads read consecutive cells (the
    // field index is a compile-time constant: an indexed parameter array would live in local
    // memory)
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const double inflow_k = a.mp.inflow[k];
        for (int j = threadIdx.x; j < span; j += blockDim.x)
            su[j * M + k] = line_get<R>(uin + k * n, n, 1, (int64_t)c0 - 3 + j, in.bc, inflow_k);
    }
    const double dt = *(volatile double*)&ctl->dt;
    const R alpha = R(*(volatile double*)&ctl->alpha);
    __syncthreads();

    // faces c0 - 1/2 .. c0 + cnt - 1/2 (local q = 0..cnt): stencil su[q .. q+5]
    EtaCount ec;
    const bool last_tile = c0 + cnt == n;
    for (int q = threadIdx.x; q <= cnt; q += blockDim.x) {
        R vm[M], vp[M], h[M];
        uint32_t fl[M];
        bool ok = face_all<R, D, KIND, M, CHAR>(su + q * M, a.mp, vm, vp, fl);
        lf_flux<R, KIND, M>(vm, vp, alpha, a.mp, 0, h);
#pragma unroll
        for (int k = 0; k < M; ++k) sh[q * M + k] = ok ? h[k] : R(__longlong_as_double(0x7ff8000000000000ll));
        if (face_owned(q, cnt, last_tile))
#pragma unroll
            for (int k = 0; k < M; ++k) ec.face(fl[k], a.mp.k);
    }
    flush_counts(ec, ctl, a.mp);
    __syncthreads();

    // cells: eq. PDE1 and the Shu-Osher combination
    R* uout = reinterpret_cast<R*>(a.uout) + in.off;
    const R* un = reinterpret_cast<const R*>(a.un) + in.off;
    const R dtR = R(dt);
    const R dxR = R(in.dx);
    double vmax = 0.0;
    bool bad = false;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        R U[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const R L = -(sh[(q + 1) * M + k] - sh[q * M + k]) / dxR;
            const R uk = su[(q + 3) * M + k];
            R o;
            if (a.stage == 0) {
                o = uk + dtR * L;
            } else if (a.stage == 1) {
                o = R(0.75) * un[k * n + c0 + q] + R(0.25) * (uk + dtR * L);
            } else {
                o = stage3_w1<R>() * un[k * n + c0 + q] + stage3_w2<R>() * (uk + dtR * L);
            }
            uout[k * n + c0 + q] = o;
            U[k] = o;
            bad |= !finite_(o);
        }
        if (a.stage == 2) {
            double s = (double)wave_speed<R, KIND>(U, a.mp, 0);
            bad |= !finite_(s);
            vmax = s > vmax ? s : vmax;
        }
    }
    if (a.stage == 2 && a.advance) {
        double b = block_max_nan(vmax, bad, red, redbad);
        if (threadIdx.x == 0) {
            atomicMax(&ctl->alpha_next_bits, (unsigned long long)__double_as_longlong(b));
            __threadfence();
            unsigned prev = atomicAdd(&ctl->tiles_done, 1u);
            if (prev == (unsigned)in.ntiles - 1u) {
                __threadfence();
                finalize_1d(ctl, in);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// One warp's pass over the cells [lo, hi) of a line, for one RK stage of the resident kernel
// (the per-stage kernel runs the same arithmetic in phases over its tile): lane l of the chunk
// at base takes
//   face f = base + l: its eta (k = 3, cells f-2..f+1);
//   cell f - 1: its reconstruction (cells f-3..f+1), v^+ at face f - 1 with the eta of face
//     f - 1 (lane l - 1) and v^- at face f with the eta of face f;
//   face f - 1: the Lax-Friedrichs flux from v^- of cell f - 2 (lane l - 1) and v^+ of cell f - 1;
//   cell f - 2: the update, upd(j, flux of face j, flux of face j + 1).
// Lane 0 takes the lane l - 1 values from lane 31 of the previous chunk.  Faces lo..hi, cells
// lo-1..hi and the updates of cells lo..hi-1 are covered by f = lo..hi+1; faces lo and hi are
// also computed by the warps on either side, from the same data, so the copies agree bit for
// bit.  X(k, i) is the stage input of field k at cell i, for i in lo-3..hi+2.
// ---------------------------------------------------------------------------------------
template <int KIND, int K, int M, typename LoadX, typename Upd>
__device__ __forceinline__ void warp_line_pass(int lo, int hi, int n, int lane, const fast::FParams& fp,
                                               const MethodParams& mp, float alpha, LoadX X, Upd upd, EtaCount& ec) {
    float c_eta[M], c_vm[M], c_h[M];
#pragma unroll
    for (int k = 0; k < M; ++k) c_eta[k] = c_vm[k] = c_h[k] = 0.0f;
    for (int base = lo; base <= hi + 1; base += 32) {
        const int f = base + lane, i = f - 1, j = f - 2;
        const bool face_ok = f <= hi, cell_ok = i <= hi;
        float vm[M], vp[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            float c[5], eta = 0.0f;
            vm[k] = vp[k] = 0.0f;
            if (cell_ok) {
#pragma unroll
                for (int q = 0; q < 5; ++q) c[q] = X(k, i - 2 + q);
                if (K == 3 && face_ok) {
                    uint32_t fl = 0;
                    eta = fast::face_eta(c[1], c[2], c[3], c[4], fp, &fl);
                    if (f < hi || f == n) ec.face_k3(fl);
                }
            }
            if constexpr (K == 3) {
                float eprev = __shfl_up_sync(0xffffffffu, eta, 1);
                if (lane == 0) eprev = c_eta[k];
                c_eta[k] = __shfl_sync(0xffffffffu, eta, 31);
                if (cell_ok) fast::cell_recon(c, eta, i >= lo ? eprev : 0.0f, fp, &vm[k], &vp[k]);
            } else {
                if (cell_ok) {
                    // v^- of cell i at face f, v^+ at face f - 1
                    const uint32_t d = fast::cell_recon_k2(c + 1, 0.0, mp, fp, &vm[k], &vp[k]);
                    if (f < hi || f == n) fast::count_k2(ec, d, 0);
                    if (f - 1 >= lo && (f - 1 < hi || f - 1 == n)) fast::count_k2(ec, d, 1);
                }
            }
        }
        // flux of face f - 1
        float A[M], h[M], hl[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            A[k] = __shfl_up_sync(0xffffffffu, vm[k], 1);
            if (lane == 0) A[k] = c_vm[k];
            c_vm[k] = __shfl_sync(0xffffffffu, vm[k], 31);
            h[k] = 0.0f;
        }
        if (i >= lo && i <= hi) lf_flux<float, KIND, M>(A, vp, alpha, mp, 0, h);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            hl[k] = __shfl_up_sync(0xffffffffu, h[k], 1);
            if (lane == 0) hl[k] = c_h[k];
            c_h[k] = __shfl_sync(0xffffffffu, h[k], 31);
        }
        // update of cell j = f - 2 (cells lo..hi-1)
        if (j >= lo && j < hi) upd(j, hl, h);
    }
}

// ---------------------------------------------------------------------------------------
// The mixed-precision fused stage kernel (1D, component-wise).  Phases over the tile with
// three ghost cells per side, extended index e = 0 .. cnt+5 for cell c0 - 3 + e:
//   F: eta (and the switch) once per face, faces between e-1 and e for e = 2 .. cnt+4;
//   C: once per cell e = 2 .. cnt+3: smoothness indicators, weights and the two face values
//      v^-_{e+1/2} (with the eta of face e|e+1) and v^+_{e-1/2} (eta of face e-1|e);
//   U: cells e = 3 .. cnt+2: Lax-Friedrichs fluxes of both faces, eq. PDE1, stage update.
// The stages are kept in increment form so that the float state conserves its sum: with
// du = dt L(u^(k)) (per cell, telescoping over the faces),
//   stage 1: d1 = du0                         (u1 = u^n + d1)
//   stage 2: d2 = (d1 + du1) / 4              (u2 = 3/4 u^n + 1/4 (u1 + du1) = u^n + d2)
//   stage 3: u^{n+1} = u^n + 2/3 (d2 + du2)   (= 1/3 u^n + 2/3 (u2 + du2))
// and the last addition is compensated with a per-cell carry (Kahan): increments smaller than
// half an ulp of u are kept in the carry instead of being rounded away.  Stage 3 writes the new
// state to s (neighbouring tiles still read u^n); the next step's stage 1 reads s and commits it
// to u.  Shared memory (floats): u^(k), eta, v^-, v^+, each (tile + 6) * M.  K = 2: the shape
// parameters belong to the cell (Table k2) and are formed in the reconstruction phase; the eta
// phase is skipped.
// ---------------------------------------------------------------------------------------
template <int KIND, int K>
__device__ __forceinline__ void stage1d_fast_body(const Stage1DArgs& a, const Tile td, const InstDev& in, Ctl* ctl,
                                                  unsigned char* smem_raw) {
    constexpr int M = kind_m<KIND>();
    __shared__ float red[32];
    __shared__ int redbad[32];
    __shared__ float s_lam;
    const int span_max = a.tile + 6;
    float* su = reinterpret_cast<float*>(smem_raw);
    float* se = su + span_max * M;
    float* svm = se + span_max * M;
    float* svp = svm + span_max * M;
    if (*(volatile int32_t*)&ctl->done) return;  // uniform over the CTA
    const int64_t n = in.n;
    const int c0 = td.start;
    const int cnt = (int)((n - c0) < a.tile ? (n - c0) : a.tile);
    const int stage = a.stage;
    float* u = a.u + in.off;
    float* d1 = a.d1 + in.off;
    float* d2 = a.d2 + in.off;
    float* sn = a.s + in.off;
    float* cr = a.c + in.off;
    const int span = cnt + 6;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        for (int j = threadIdx.x; j < span; j += blockDim.x) {
            const int64_t g = halo_idx(n, (int64_t)c0 - 3 + j, in.bc);
            float x;
            if (g < 0)
                x = a.mp.inflow_f[k];
            else if (stage == 0)
                x = sn[k * n + g];
            else
                x = u[k * n + g] + (stage == 1 ? d1[k * n + g] : d2[k * n + g]);
            su[j * M + k] = x;
        }
    }
    if (threadIdx.x == 0) s_lam = (float)(*(volatile double*)&ctl->dt / in.dx);
    const float alpha = (float)*(volatile double*)&ctl->alpha;
    const fast::FParams fp = fast::fparams(a.mp);
    __syncthreads();

    // F: faces between extended cells e-1 and e (local face q = e - 3)
    EtaCount ec;
    const bool last_tile = c0 + cnt == n;
    if constexpr (K == 3) {
        for (int idx = threadIdx.x; idx < (cnt + 3) * M; idx += blockDim.x) {
            const int e = 2 + idx / M, k = idx - (e - 2) * M;
            uint32_t fl = 0;
            se[e * M + k] = fast::face_eta(su[(e - 2) * M + k], su[(e - 1) * M + k], su[e * M + k],
                                           su[(e + 1) * M + k], fp, &fl);
            if (face_owned(e - 3, cnt, last_tile)) ec.face_k3(fl);
        }
        __syncthreads();
    }
    // C: cells
    for (int idx = threadIdx.x; idx < (cnt + 2) * M; idx += blockDim.x) {
        const int e = 2 + idx / M, k = idx - (e - 2) * M;
        float c[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) c[j] = su[(e - 2 + j) * M + k];
        float vm, vp;
        if constexpr (K == 3) {
            fast::cell_recon(c, se[(e + 1) * M + k], se[e * M + k], fp, &vm, &vp);
        } else {
            // v^- at the cell's right face (local face e - 2), v^+ at its left face (e - 3)
            const uint32_t d = fast::cell_recon_k2(c + 1, 0.0, a.mp, fp, &vm, &vp);
            if (face_owned(e - 2, cnt, last_tile)) fast::count_k2(ec, d, 0);
            if (face_owned(e - 3, cnt, last_tile)) fast::count_k2(ec, d, 1);
        }
        svm[e * M + k] = vm;
        svp[e * M + k] = vp;
    }
    flush_counts(ec, ctl, a.mp);
    __syncthreads();
    // U: cells
    const float lam = s_lam;
    float vmaxf = 0.0f;
    bool bad = false;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int e = q + 3;
        const int64_t gi = c0 + q;
        float hl[M], hr[M], U[M];
        lf_flux<float, KIND, M>(svm + (e - 1) * M, svp + e * M, alpha, a.mp, 0, hl);
        lf_flux<float, KIND, M>(svm + e * M, svp + (e + 1) * M, alpha, a.mp, 0, hr);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const float du = lam * (hl[k] - hr[k]);
            const int64_t ix = k * n + gi;
            if (stage == 0) {
                u[ix] = su[e * M + k];  // commit u^n (the state s of the previous step)
                d1[ix] = du;
                bad |= !finite_(du);
            } else if (stage == 1) {
                const float v = 0.25f * (d1[ix] + du);
                d2[ix] = v;
                bad |= !finite_(v);
            } else {
                const float base = u[ix];
                const float y = kTwoThirdsF * (d2[ix] + du) + cr[ix];
                const float t = base + y;
                cr[ix] = y - (t - base);
                sn[ix] = t;
                U[k] = t;
                bad |= !finite_(t);
            }
        }
        if (stage == 2) {
            const float sp = wave_speed<float, KIND>(U, a.mp, 0);
            bad |= !finite_(sp);
            vmaxf = sp > vmaxf ? sp : vmaxf;
        }
    }
    if (stage == 2 && a.advance) {
        const double b = block_max_nan_f(vmaxf, bad, red, redbad);
        if (threadIdx.x == 0) {
            atomicMax(&ctl->alpha_next_bits, (unsigned long long)__double_as_longlong(b));
            __threadfence();
            const unsigned prev = atomicAdd(&ctl->tiles_done, 1u);
            if (prev == (unsigned)in.ntiles - 1u) {
                __threadfence();
                finalize_1d(ctl, in);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// One whole RK3 step of one 1D tile (mixed precision, compensated, component-wise), for
// instances too large for the resident kernel.  The tile loads u^n once with a 9-cell halo
// (three stages, each reaching 3 cells), and computes in shared memory
//   stage 1 on the cells within 6 of the tile: d1 = du(u^n),        x1 = u^n + d1;
//   stage 2 on the cells within 3:              d2 = (d1 + du(x1))/4, x2 = u^n + d2;
//   stage 3 on the tile:  u^{n+1} = u^n + 2/3 (d2 + du(x2)), compensated by the carry c,
// with the arithmetic of the per-stage body cell for cell, so that the results are the same
// bits.  Cells of the halo outside the domain are ghosts: their stage values follow the
// boundary rule from the tile's own stage values (a periodic ghost is the same computation as
// the cell it wraps to).  u^n is read from `uin` and u^{n+1} written to `uout`: the two state
// buffers alternate between steps (neighbouring tiles read the halo of u^n in the same launch).
// Shared memory (floats, span = tile + 18 cells per field): u^n, the stage input, d, eta, v^-,
// v^+.
// ---------------------------------------------------------------------------------------
// the stage values of the ghost cells of [lo, hi) (extended indices; cell e is global cell
// c0 - FUSE_HALO + e) from the boundary rule: transmissive and the right end of an inflow
// line repeat the end cell, the left end of an inflow line holds the inflow state
template <int M>
__device__ __forceinline__ void fused_fill_ghosts(float* x, int lo, int hi, int c0, int64_t n, int bc,
                                                  const MethodParams& mp) {
    const int e0 = FUSE_HALO - c0;                   // extended index of cell 0
    const int64_t e1 = (int64_t)e0 + n - 1;          // of cell n - 1
    for (int e = lo + (int)threadIdx.x; e < hi; e += blockDim.x) {
        if (e >= e0 && e <= e1) continue;
#pragma unroll
        for (int k = 0; k < M; ++k)
            x[e * M + k] = e < e0 ? (bc == NPW_BC_INFLOW ? mp.inflow_f[k] : x[e0 * M + k]) : x[(int)e1 * M + k];
    }
}

template <int KIND, int K>
__device__ __forceinline__ void step1d_fused_body(const Stage1DArgs& a, const Tile td, const InstDev& in, Ctl* ctl,
                                                  unsigned char* smem_raw) {
    constexpr int M = kind_m<KIND>();
    constexpr int H = FUSE_HALO;
    __shared__ float red[32];
    __shared__ int redbad[32];
    __shared__ float s_lam;
    const int span_max = a.tile + 2 * H;
    float* su0 = reinterpret_cast<float*>(smem_raw);  // u^n
    float* sx = su0 + span_max * M;                    // input of the current stage
    float* sd = sx + span_max * M;                     // d1, then d2
    float* se = sd + span_max * M;                     // eta of face e (between e-1 and e)
    float* svm = se + span_max * M;                    // v^- at the right face of cell e
    float* svp = svm + span_max * M;                   // v^+ at the left face of cell e
    if (*(volatile int32_t*)&ctl->done) return;       // uniform over the CTA
    const int64_t n = in.n;
    const int c0 = td.start;
    const int cnt = (int)((n - c0) < a.tile ? (n - c0) : a.tile);
    const int span = cnt + 2 * H;
    const float* uin = reinterpret_cast<const float*>(a.uin) + in.off;
    float* uout = reinterpret_cast<float*>(a.uout) + in.off;
    float* cr = a.c + in.off;
    const bool periodic = in.bc == NPW_BC_PERIODIC;
    // halo load of u^n (a periodic index may wrap more than once on a short line)
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const float inflow_k = a.mp.inflow_f[k];
        for (int j = threadIdx.x; j < span; j += blockDim.x) {
            int64_t g = (int64_t)c0 - H + j;
            float x;
            if (periodic) {
                g %= n;
                if (g < 0) g += n;
                x = uin[k * n + g];
            } else if (g < 0 && in.bc == NPW_BC_INFLOW) {
                x = inflow_k;
            } else {
                g = g < 0 ? 0 : (g >= n ? n - 1 : g);
                x = uin[k * n + g];
            }
            su0[j * M + k] = x;
            sx[j * M + k] = x;
        }
    }
    if (threadIdx.x == 0) s_lam = (float)(*(volatile double*)&ctl->dt / in.dx);
    const float alpha = (float)*(volatile double*)&ctl->alpha;
    const fast::FParams fp = fast::fparams(a.mp);
    const bool last_tile = c0 + cnt == n;
    const int e0 = H - c0;  // extended index of global cell 0
    EtaCount ec;
    float vmaxf = 0.0f;
    bool bad = false;
    __syncthreads();
    const float lam = s_lam;
#pragma unroll 1
    for (int st = 0; st < 3; ++st) {
        const int L = 3 * (st + 1), R = span - 3 * (st + 1);  // cells updated by this stage: [L, R)
        // F: eta of the faces q in [L - 1, R + 2) (face q between cells q - 1 and q)
        if constexpr (K == 3) {
            for (int idx = threadIdx.x; idx < (R - L + 3) * M; idx += blockDim.x) {
                const int q = L - 1 + idx / M, k = idx - (q - L + 1) * M;
                uint32_t fl = 0;
                se[q * M + k] = fast::face_eta(sx[(q - 2) * M + k], sx[(q - 1) * M + k], sx[q * M + k],
                                               sx[(q + 1) * M + k], fp, &fl);
                if (face_owned(q - H, cnt, last_tile)) ec.face_k3(fl);
            }
            __syncthreads();
        }
        // C: cells e in [L - 1, R + 1): v^- at face e + 1, v^+ at face e
        for (int idx = threadIdx.x; idx < (R - L + 2) * M; idx += blockDim.x) {
            const int e = L - 1 + idx / M, k = idx - (e - L + 1) * M;
            float c[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) c[j] = sx[(e - 2 + j) * M + k];
            float vm, vp;
            if constexpr (K == 3) {
                fast::cell_recon(c, se[(e + 1) * M + k], se[e * M + k], fp, &vm, &vp);
            } else {
                const uint32_t d = fast::cell_recon_k2(c + 1, 0.0, a.mp, fp, &vm, &vp);
                if (face_owned(e + 1 - H, cnt, last_tile)) fast::count_k2(ec, d, 0);
                if (face_owned(e - H, cnt, last_tile)) fast::count_k2(ec, d, 1);
            }
            svm[e * M + k] = vm;
            svp[e * M + k] = vp;
        }
        __syncthreads();
        // U: fluxes of both faces, eq. PDE1, the stage in increment form
        for (int e = L + (int)threadIdx.x; e < R; e += blockDim.x) {
            const int64_t g = (int64_t)c0 - H + e;
            if (!periodic && (g < 0 || g >= n)) continue;  // a ghost: filled below
            float hl[M], hr[M];
            lf_flux<float, KIND, M>(svm + (e - 1) * M, svp + e * M, alpha, a.mp, 0, hl);
            lf_flux<float, KIND, M>(svm + e * M, svp + (e + 1) * M, alpha, a.mp, 0, hr);
            if (st < 2) {
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const float du = lam * (hl[k] - hr[k]);
                    const float d = st == 0 ? du : 0.25f * (sd[e * M + k] + du);
                    sd[e * M + k] = d;
                    sx[e * M + k] = su0[e * M + k] + d;
                }
            } else {
                float U[M];
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const float du = lam * (hl[k] - hr[k]);
                    const int64_t ix = k * n + g;
                    const float base = su0[e * M + k];
                    const float y = kTwoThirdsF * (sd[e * M + k] + du) + cr[ix];
                    const float t = base + y;
                    cr[ix] = y - (t - base);
                    uout[ix] = t;
                    U[k] = t;
                    bad |= !finite_(t);
                }
                const float sp = wave_speed<float, KIND>(U, a.mp, 0);
                bad |= !finite_(sp);
                vmaxf = sp > vmaxf ? sp : vmaxf;
            }
        }
        if (st < 2) {
            __syncthreads();
            if (!periodic && (e0 > L || e0 + n < (int64_t)R)) {
                fused_fill_ghosts<M>(sx, L, R, c0, n, in.bc, a.mp);
                __syncthreads();
            }
        }
    }
    flush_counts(ec, ctl, a.mp);
    if (a.advance) {
        const double b = block_max_nan_f(vmaxf, bad, red, redbad);
        if (threadIdx.x == 0) {
            atomicMax(&ctl->alpha_next_bits, (unsigned long long)__double_as_longlong(b));
            __threadfence();
            const unsigned prev = atomicAdd(&ctl->tiles_done, 1u);
            if (prev == (unsigned)in.ntiles - 1u) {
                __threadfence();
                finalize_1d(ctl, in);
            }
        }
    }
}

// s = u and c = 0 over the tiles (before the first step); u = s (after the last; odd: only
// for the instances that took an odd number of fused steps, whose last step wrote s)
static __global__ void comp_copy_kernel(float* dst, const float* src, float* zero, const InstDev* __restrict__ inst,
                                        const Tile* __restrict__ tiles, int tile, int m, const Ctl* odd) {
    const Tile td = tiles[blockIdx.x];
    if (odd && (odd[td.inst].steps & 1) == 0) return;
    const InstDev in = inst[td.inst];
    const int64_t n = in.n;
    const int c0 = td.start;
    const int cnt = (int)((n - c0) < tile ? (n - c0) : tile);
    for (int idx = threadIdx.x; idx < cnt * m; idx += blockDim.x) {
        const int k = idx / cnt, q = idx - k * cnt;
        const int64_t ix = in.off + k * n + c0 + q;
        dst[ix] = src[ix];
        if (zero) zero[ix] = 0.0f;
    }
}

// ---------------------------------------------------------------------------------------
// Resident whole-solve kernel (float state, component-wise).  One CTA owns one instance for
// its whole run: u^n and the two stage values live in shared memory, and thread 0 advances
// t, alpha and dt between steps.  Each warp owns a contiguous range of cells [lo, hi) and
// runs a stage on it in one pass without waiting for the other warps: per chunk of 32 faces,
// each lane forms the eta of its face, reconstructs the cell to its left, computes the flux of
// the face before and updates the cell before that, taking its left neighbour's values by lane
// shuffles.  The faces lo and hi are also computed by the neighbouring warps, from the same
// data, so the copies agree bit for bit.  Warps therefore drift apart within a stage; the only
// CTA-wide barrier is between stages (the next stage reads the neighbours' halo).  Stage values
// are double-buffered (u^n -> uA -> uB -> u^{n+1}) so no warp overwrites a value another still
// reads.  Shared memory per field: u^n, uA, uB, each n cells with RES_GHOST ghost cells per side.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int res_map(int i, int n, int bc) {
    if (bc == NPW_BC_PERIODIC) return i < 0 ? i + n : (i >= n ? i - n : i);
    return i < 0 ? (bc == NPW_BC_INFLOW ? -1 : 0) : (i >= n ? n - 1 : i);
}

// Store v as cell i of a ghosted array p (p[-3..-1] and p[n..n+2] are the ghost cells, n >= 6)
// and refresh the ghost cells that copy it: periodic ghosts are cells n-3..n-1 (left) and
// 0..2 (right); outflow ghosts repeat cells 0 and n-1; the inflow boundary (left) holds
// inflow_ghost (the inflow value in a state, -0 in an increment, so that u^n + d reproduces
// the inflow value bit for bit).
__device__ __forceinline__ void res_store(float* p, int i, int n, int bc, float v, float inflow_ghost) {
    p[i] = v;
    if (i >= RES_GHOST && i < n - RES_GHOST) return;
    if (bc == NPW_BC_PERIODIC) {
        p[i < RES_GHOST ? i + n : i - n] = v;
    } else {
        if (i == 0) {
            const float gl = bc == NPW_BC_INFLOW ? inflow_ghost : v;
#pragma unroll
            for (int j = 1; j <= RES_GHOST; ++j) p[-j] = gl;
        }
        if (i == n - 1) {
#pragma unroll
            for (int j = 0; j < RES_GHOST; ++j) p[n + j] = v;
        }
    }
}

template <int KIND, int K>
__global__ void __launch_bounds__(1024) solve1d_resident_kernel(ResidentArgs a) {
    constexpr int M = kind_m<KIND>();
    extern __shared__ __align__(16) float smf[];
    __shared__ float red[32];
    __shared__ int redbad[32];
    __shared__ float s_alpha, s_lam;
    __shared__ int s_done;
    const int inst_idx = a.list[blockIdx.x];
    const InstDev in = a.inst[inst_idx];
    Ctl* ctl = a.ctl + inst_idx;
    const int n = (int)in.n;
    // u^n, d1 and d2 carry RES_GHOST ghost cells on each side (field k, cell i at k NS + 3 + i),
    // so that the stencils read them without a boundary map: the boundary cells write the
    // ghost copies when they are updated (res_store).
    const int NS = n + 2 * RES_GHOST;
    float* un = smf;                // [M][NS] u^n
    float* uA = un + M * NS;        // [M][NS] d1, then the new state
    float* uB = uA + M * NS;        // [M][NS] d2
    const fast::FParams fp = fast::fparams(a.mp);
    float* g = reinterpret_cast<float*>(a.arena) + in.off;
    float* cr = a.carry + in.off;
    for (int idx = threadIdx.x; idx < M * n; idx += blockDim.x) {
        const int k = idx / n;
        un[idx + k * 2 * RES_GHOST + RES_GHOST] = g[idx];
        cr[idx] = 0.0f;
    }
    float inflow[M];
#pragma unroll
    for (int k = 0; k < M; ++k) inflow[k] = a.mp.inflow_f[k];
    EtaCount ec;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int per = (n + nwarps - 1) / nwarps;
    const int lo = min(n, warp * per), hi = min(n, lo + per);
    __syncthreads();
    // ghost cells of u^n
    if (threadIdx.x < 2 * RES_GHOST * M) {
        const int k = threadIdx.x / (2 * RES_GHOST), q = threadIdx.x - k * 2 * RES_GHOST;
        const int gi = q < RES_GHOST ? q - RES_GHOST : n + q - RES_GHOST;
        const int c = res_map(gi, n, in.bc);
        const float v = c < 0 ? inflow[k] : un[k * NS + RES_GHOST + c];
        un[k * NS + RES_GHOST + gi] = v;
    }
    __syncthreads();

    // alpha^0 and the first dt
    float vmaxf = 0.0f;
    bool bad = false;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float U[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            U[k] = un[k * NS + RES_GHOST + i];
            bad |= !finite_(U[k]);
        }
        const float sp = wave_speed<float, KIND>(U, a.mp, 0);
        bad |= !finite_(sp);
        vmaxf = sp > vmaxf ? sp : vmaxf;
    }
    double t = 0.0, dt = 0.0, alpha = 0.0, alpha_max = 0.0;  // thread 0's copies
    int64_t steps = 0, cap = 0;
    int last = 0, status = 0;
    {
        const double b = block_max_nan_f(vmaxf, bad, red, redbad);
        if (threadIdx.x == 0) {
            if (!(b - b == 0.0)) {
                status = NPW_ENONFINITE;
                s_done = 1;
            } else {
                alpha = alpha_max = b;
                s_done = !(t < in.t_end);
                const double rate = b / in.dx;
                dt = (rate > 0.0) ? in.cfl / rate : in.t_end - t;
                if (t + dt * (1.0 + 1e-10) >= in.t_end) {
                    dt = in.t_end - t;
                    last = 1;
                }
                cap = step_cap(in.t_end - t, dt, a.mp.max_steps);
            }
            s_lam = (float)(dt / in.dx);
            s_alpha = (float)alpha;
        }
        __syncthreads();
    }

    while (!s_done) {
        const float lam = s_lam;
        const float alphaf = s_alpha;
        vmaxf = 0.0f;
        bad = false;
#pragma unroll
        for (int stage = 0; stage < 3; ++stage) {
            // stage input u^(k) = u^n + d_k, formed on the fly (increment form, see
            // stage1d_fast_kernel); stage 3 writes the new state into uA
            const float* D = stage == 1 ? uA : uB;
#define NPW_X(idx) (stage == 0 ? un[(idx)] : un[(idx)] + D[(idx)])
            if (lo < hi) {
                auto X = [&](int k, int i) { return NPW_X(k * NS + RES_GHOST + i); };
                auto upd = [&](int j, const float* hl, const float* hr) {
                    float U[M];
#pragma unroll
                    for (int k = 0; k < M; ++k) {
                        const float du = lam * (hl[k] - hr[k]);
                        const int ix = k * NS + RES_GHOST + j;
                        if (stage == 0) {
                            res_store(uA + k * NS + RES_GHOST, j, n, in.bc, du, -0.0f);
                            U[k] = du;
                        } else if (stage == 1) {
                            const float v = 0.25f * (uA[ix] + du);
                            res_store(uB + k * NS + RES_GHOST, j, n, in.bc, v, -0.0f);
                            U[k] = v;
                        } else {
                            const int gx = k * n + j;
                            const float base_u = un[ix];
                            const float y = kTwoThirdsF * (uB[ix] + du) + cr[gx];
                            const float t = base_u + y;
                            cr[gx] = y - (t - base_u);
                            res_store(uA + k * NS + RES_GHOST, j, n, in.bc, t, inflow[k]);
                            U[k] = t;
                        }
                        bad |= !finite_(U[k]);
                    }
                    if (stage == 2) {
                        const float sp = wave_speed<float, KIND>(U, a.mp, 0);
                        bad |= !finite_(sp);
                        vmaxf = sp > vmaxf ? sp : vmaxf;
                    }
                };
                warp_line_pass<KIND, K, M>(lo, hi, n, lane, fp, a.mp, alphaf, X, upd, ec);
            }
            __syncthreads();
#undef NPW_X
        }
        {  // the new state (in uA) becomes u^n
            float* tmp = un;
            un = uA;
            uA = tmp;
        }
        const double b = block_max_nan_f(vmaxf, bad, red, redbad);
        if (threadIdx.x == 0) {
            steps += 1;
            t = last ? in.t_end : t + dt;
            if (!(b - b == 0.0)) {
                status = NPW_ENONFINITE;
                s_done = 1;
            } else {
                alpha = b;
                alpha_max = b > alpha_max ? b : alpha_max;
                if (last) {
                    s_done = 1;
                } else {
                    const double rate = b / in.dx;
                    dt = (rate > 0.0) ? in.cfl / rate : in.t_end - t;
                    if (t + dt * (1.0 + 1e-10) >= in.t_end) {
                        dt = in.t_end - t;
                        last = 1;
                    }
                    if (steps >= cap || !(t + dt > t)) {  // step limit, or time stopped advancing
                        status = NPW_ETIMEOUT;
                        s_done = 1;
                    }
                    s_lam = (float)(dt / in.dx);
                    s_alpha = (float)alpha;
                }
            }
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < M * n; idx += blockDim.x) g[idx] = un[idx + (idx / n) * 2 * RES_GHOST + RES_GHOST];
    flush_counts(ec, ctl, a.mp);
    if (threadIdx.x == 0) {
        ctl->t = t;
        ctl->dt = dt;
        ctl->alpha = alpha;
        ctl->alpha_max = alpha_max;
        ctl->steps = steps;
        ctl->status = status;
        ctl->done = 1;
    }
}

// ---------------------------------------------------------------------------------------
// 2D dimension-by-dimension stage kernel (component-wise).  Tile TX x TY cells; shared
// memory holds the (TX + 6) x (TY + 6) input block, the x-face fluxes (TX + 1) x TY and
// the y-face fluxes TX x (TY + 1).
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R grid_get(const R* u, const Inst2D& in, int64_t i, int64_t j, double inflow) {
    // columns (i) follow the instance boundary condition bc, rows (j) bc_y; an inflow side
    // (left for bc, bottom for bc_y) gives the inflow state, whatever the other index
    const int64_t nx = in.nx, ny = in.ny;
    if (in.bc_y == NPW_BC_INFLOW && j < 0) return R(inflow);
    if (in.bc == NPW_BC_INFLOW && i < 0) return R(inflow);
    if (in.bc == NPW_BC_PERIODIC) {
        i %= nx;
        if (i < 0) i += nx;
    } else {
        i = i < 0 ? 0 : (i >= nx ? nx - 1 : i);
    }
    if (in.bc_y == NPW_BC_PERIODIC) {
        j %= ny;
        if (j < 0) j += ny;
    } else {
        j = j < 0 ? 0 : (j >= ny ? ny - 1 : j);
    }
    return u[j * nx + i];
}

// grid_get for a tile halo: i in [-3, nx + 2] and j in [-3, ny + 2] (nx, ny >= 6), so one
// comparison per side replaces the general map of grid_get (and its 64-bit remainders)
__device__ __forceinline__ float halo_get(const float* u, const Inst2D& in, int i, int j, float inflow) {
    const int nx = (int)in.nx, ny = (int)in.ny;
    if (in.bc_y == NPW_BC_INFLOW && j < 0) return inflow;
    if (in.bc == NPW_BC_INFLOW && i < 0) return inflow;
    if (in.bc == NPW_BC_PERIODIC)
        i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
    else
        i = i < 0 ? 0 : (i >= nx ? nx - 1 : i);
    if (in.bc_y == NPW_BC_PERIODIC)
        j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
    else
        j = j < 0 ? 0 : (j >= ny ? ny - 1 : j);
    return u[(int64_t)j * in.nx + i];
}

// ---------------------------------------------------------------------------------------
// 2D stage kernel of the mixed path (float state, component-wise) in phases, each a balanced
// loop over independent work items:
//   E  (k = 3) eta of every (face, field) of both directions (FP64 quotient, switch)
//   C  reconstruction of every (cell, field) of both directions: v^- at its right / upper face
//      and v^+ at its left / lower face, one set of smoothness indicators for both (k = 2: the
//      cell's own switch and shape parameters, with the transverse term of the 5-cell cross)
//   F  Lax-Friedrichs flux of every face (all fields)
//   U  flux difference and Shu-Osher stage combination of every cell
// Every face value gets the arithmetic of fast::face_field, so the result is the same as the
// face-by-face kernel's; the phases avoid reconstructing a cell once per face and the uneven
// per-thread face counts of that kernel.
// ---------------------------------------------------------------------------------------
// shared memory (floats) of the 2D fast body: the (TX+6) x (TY+6) block and three face arrays
template <int M>
__host__ __device__ constexpr int stage2d_fast_smem_floats() {
    return ((TY_2D + 6) * (TX_2D + 6) + 3 * ((TX_2D + 1) * TY_2D + TX_2D * (TY_2D + 1))) * M;
}

// One tile (index `tile` of the instance's tiles_x x tiles_y tiles) of one stage.
template <int KIND, int K>
__device__ __forceinline__ void stage2d_fast_body(const Stage2DArgs& a, const Inst2D& in, Ctl* ctl, int tile,
                                                  float* smem) {
    constexpr int M = kind_m<KIND>();
    constexpr int BX = TX_2D + 6, BY = TY_2D + 6;
    constexpr int NFX = (TX_2D + 1) * TY_2D;  // x faces: (qx, qy), qx = 0..TX between cells qx-1, qx
    constexpr int NFY = TX_2D * (TY_2D + 1);  // y faces: (qx, qy), qy = 0..TY
    constexpr int NF = NFX + NFY;
    // field-major layout: su[k][by][bx], and ef, vmf, vpf [k][face] (x faces, then y faces), so
    // that consecutive threads (consecutive cells or faces of one field) hit consecutive banks
    float* su = smem;                          // [BY * BX * M]
    float* ef = su + BY * BX * M;              // [M][NF] eta per (field, face); then the fluxes
    float* vmf = ef + NF * M;                  // v^- per (field, face)
    float* vpf = vmf + NF * M;                 // v^+ per (field, face)
    __shared__ float red[32];
    __shared__ int redbad[32];
    __shared__ float red2[32];
    __shared__ int redbad2[32];
    __shared__ float s_par[5];               // alpha_x, alpha_y, dt, dx, dy in float
    if (*(volatile int32_t*)&ctl->done) return;
    const int tx0 = (tile % in.tiles_x) * TX_2D;
    const int ty0 = (tile / in.tiles_x) * TY_2D;
    const int64_t nx = in.nx, ny = in.ny, cells = nx * ny;
    const float* uin = reinterpret_cast<const float*>(a.uin) + in.off;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const fast::FParams fp = fast::fparams(a.mp);
    const bool cross = K == 2 && a.mp.cross_2d && (a.mp.scheme == NPW_RBF_ENO_ || a.mp.scheme == NPW_RBF_WENO_);
    // the field index is a compile-time constant in each loop (an indexed parameter array would
    // put the stage arguments in local memory)
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const float inflow_k = a.mp.inflow_f[k];
        for (int rem = tid; rem < BX * BY; rem += nthr) {
            const int by = rem / BX, bx = rem - by * BX;
            // the corners are read only by the 5-cell cross (transverse differences of halo cells)
            const bool corner = (bx < 3 || bx >= TX_2D + 3) && (by < 3 || by >= TY_2D + 3);
            su[(k * BY + by) * BX + bx] =
                (corner && !cross) ? 0.0f : halo_get(uin + k * cells, in, tx0 - 3 + bx, ty0 - 3 + by, inflow_k);
        }
    }
    if (tid == 0) {
        s_par[0] = (float)(*(volatile double*)&ctl->alpha);
        s_par[1] = (float)(*(volatile double*)&ctl->alpha_y);
        s_par[2] = (float)(*(volatile double*)&ctl->dt);
        s_par[3] = (float)in.dx;
        s_par[4] = (float)in.dy;
    }
    __syncthreads();
    const float ax = s_par[0], ay = s_par[1];
    // counted faces: x face (qx, qy) of grid row ty0 + qy, y face of grid column tx0 + qx
    EtaCount ec;
    const int cols_in = (int)min((int64_t)TX_2D, nx - tx0), rows_in = (int)min((int64_t)TY_2D, ny - ty0);
    const bool last_x = tx0 + TX_2D >= nx, last_y = ty0 + TY_2D >= ny;
    auto own_x = [=](int qx, int qy) { return qy < rows_in && face_owned(qx, cols_in, last_x); };
    auto own_y = [=](int qx, int qy) { return qx < cols_in && face_owned(qy, rows_in, last_y); };
#define NPW_SU(bx, by, k) su[((k) * BY + (by)) * BX + (bx)]
    // E: item = (face, field); x face (qx, qy) has the eta stencil su[qy+3][qx+1 .. qx+4],
    // y face (qx, qy) su[qy+1 .. qy+4][qx+3]
    for (int it = tid; K == 3 && it < NF * M; it += nthr) {
        const int k = it / NF, f = it - k * NF;
        float w0, w1, w2, w3;
        bool own;
        if (f < NFX) {
            const int qy = f / (TX_2D + 1), qx = f - qy * (TX_2D + 1);
            w0 = NPW_SU(qx + 1, qy + 3, k);
            w1 = NPW_SU(qx + 2, qy + 3, k);
            w2 = NPW_SU(qx + 3, qy + 3, k);
            w3 = NPW_SU(qx + 4, qy + 3, k);
            own = own_x(qx, qy);
        } else {
            const int g = f - NFX;
            const int qy = g / TX_2D, qx = g - qy * TX_2D;
            w0 = NPW_SU(qx + 3, qy + 1, k);
            w1 = NPW_SU(qx + 3, qy + 2, k);
            w2 = NPW_SU(qx + 3, qy + 3, k);
            w3 = NPW_SU(qx + 3, qy + 4, k);
            own = own_y(qx, qy);
        }
        uint32_t fl = 0;
        ef[k * NF + f] = fast::face_eta(w0, w1, w2, w3, fp, &fl);
        if (own) ec.face_k3(fl);
    }
    __syncthreads();
    // C: item = (cell, field); x: cells cx = -1..TX of each row (TX + 2 per row), y: cells
    // cy = -1..TY of each column.  Cell -1 only gives v^- at face 0, cell TX (TY) only v^+ at the
    // last face.
    constexpr int NCX = (TX_2D + 2) * TY_2D, NCY = TX_2D * (TY_2D + 2);
    for (int it = tid; it < (NCX + NCY) * M; it += nthr) {
        const int k = it / (NCX + NCY), c = it - k * (NCX + NCY);
        float cc[5];
        double trans = 0.0;  // k = 2 cross: transverse second difference of the cell
        int fl_idx, fr_idx;  // faces left / right of the cell (-1 when outside the tile)
        bool own_l, own_r;   // those faces are counted by this tile
        if (c < NCX) {
            const int qy = c / (TX_2D + 2), cx = c - qy * (TX_2D + 2) - 1;
#pragma unroll
            for (int j = 0; j < 5; ++j) cc[j] = NPW_SU(cx + 1 + j, qy + 3, k);
            fl_idx = cx >= 0 ? qy * (TX_2D + 1) + cx : -1;
            fr_idx = cx < TX_2D ? qy * (TX_2D + 1) + cx + 1 : -1;
            own_l = cx >= 0 && own_x(cx, qy);
            own_r = cx < TX_2D && own_x(cx + 1, qy);
            if (cross)
                trans = (fast::widen(NPW_SU(cx + 3, qy + 2, k)) - 2.0 * fast::widen(NPW_SU(cx + 3, qy + 3, k))) +
                        fast::widen(NPW_SU(cx + 3, qy + 4, k));
        } else {
            // consecutive threads take consecutive columns of one row (no shared-memory bank
            // conflicts on the column stencil or on the face arrays)
            const int g = c - NCX;
            const int cy = g / TX_2D - 1, qx = g - (cy + 1) * TX_2D;
#pragma unroll
            for (int j = 0; j < 5; ++j) cc[j] = NPW_SU(qx + 3, cy + 1 + j, k);
            fl_idx = cy >= 0 ? NFX + cy * TX_2D + qx : -1;
            fr_idx = cy < TY_2D ? NFX + (cy + 1) * TX_2D + qx : -1;
            own_l = cy >= 0 && own_y(qx, cy);
            own_r = cy < TY_2D && own_y(qx, cy + 1);
            if (cross)
                trans = (fast::widen(NPW_SU(qx + 2, cy + 3, k)) - 2.0 * fast::widen(NPW_SU(qx + 3, cy + 3, k))) +
                        fast::widen(NPW_SU(qx + 4, cy + 3, k));
        }
        float vm, vp;
        if constexpr (K == 3) {
            const float er = fr_idx >= 0 ? ef[k * NF + fr_idx] : 0.0f;
            const float el = fl_idx >= 0 ? ef[k * NF + fl_idx] : 0.0f;
            fast::cell_recon(cc, er, el, fp, &vm, &vp);
        } else {
            const uint32_t d = fast::cell_recon_k2(cc + 1, trans, a.mp, fp, &vm, &vp);
            if (own_r) fast::count_k2(ec, d, 0);
            if (own_l) fast::count_k2(ec, d, 1);
        }
        if (fr_idx >= 0) vmf[k * NF + fr_idx] = vm;
        if (fl_idx >= 0) vpf[k * NF + fl_idx] = vp;
    }
    flush_counts(ec, ctl, a.mp);
    __syncthreads();
    // F: item = face (all fields); the fluxes overwrite the eta array
    for (int f = tid; f < NFX + NFY; f += nthr) {
        float vm[M], vp[M], h[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            vm[k] = vmf[k * NF + f];
            vp[k] = vpf[k * NF + f];
        }
        if (f < NFX)
            lf_flux<float, KIND, M>(vm, vp, ax, a.mp, 0, h);
        else
            lf_flux<float, KIND, M>(vm, vp, ay, a.mp, 1, h);
#pragma unroll
        for (int k = 0; k < M; ++k) ef[k * NF + f] = h[k];
    }
    __syncthreads();
#undef NPW_SU
    // U: one cell per thread (the same arithmetic as stage2d_kernel)
    float* uout = reinterpret_cast<float*>(a.uout) + in.off;
    const float* un = reinterpret_cast<const float*>(a.un) + in.off;
    // the flux differences are scaled by 1/dx and 1/dy (two multiplies per field and cell in
    // place of two correctly rounded divisions: 3% of this kernel's time on 2D Euler)
    const float dtR = s_par[2], idxR = 1.0f / s_par[3], idyR = 1.0f / s_par[4];
    float vmx = 0.0f, vmy = 0.0f;
    bool bad = false;
    for (int cidx = tid; cidx < TX_2D * TY_2D; cidx += nthr) {
        const int qy = cidx / TX_2D, qx = cidx - qy * TX_2D;
        const int64_t gi = tx0 + qx, gj = ty0 + qy;
        if (gi >= nx || gj >= ny) continue;
        float U[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const float* hx = ef + k * NF;
            const float* hy = hx + NFX;
            float L = -((hx[qy * (TX_2D + 1) + qx + 1] - hx[qy * (TX_2D + 1) + qx]) * idxR);
            L = L - (hy[(qy + 1) * TX_2D + qx] - hy[qy * TX_2D + qx]) * idyR;
            const float uk = su[(k * BY + qy + 3) * BX + qx + 3];
            const int64_t gidx = k * cells + gj * nx + gi;
            float o;
            if (a.stage == 0) {
                o = uk + dtR * L;
            } else if (a.stage == 1) {
                o = 0.75f * un[gidx] + 0.25f * (uk + dtR * L);
            } else {
                o = stage3_w1<float>() * un[gidx] + stage3_w2<float>() * (uk + dtR * L);
            }
            uout[gidx] = o;
            U[k] = o;
            bad |= !finite_(o);
        }
        if (a.stage == 2) {
            const float sx = wave_speed<float, KIND>(U, a.mp, 0);
            const float sy = wave_speed<float, KIND>(U, a.mp, 1);
            bad |= !finite_(sx) || !finite_(sy);
            vmx = sx > vmx ? sx : vmx;
            vmy = sy > vmy ? sy : vmy;
        }
    }
    if (a.stage == 2 && a.advance) {
        const double bx = block_max_nan_f(vmx, bad, red, redbad);
        const double by = block_max_nan_f(vmy, bad, red2, redbad2);
        if (tid == 0) {
            atomicMax(&ctl->alpha_next_bits, (unsigned long long)__double_as_longlong(bx));
            atomicMax(&ctl->alpha_y_next_bits, (unsigned long long)__double_as_longlong(by));
            __threadfence();
            const unsigned prev = atomicAdd(&ctl->tiles_done, 1u);
            if (prev == (unsigned)(in.tiles_x * in.tiles_y) - 1u) {
                __threadfence();
                finalize_2d(ctl, in);
            }
        }
    }
}

// shared memory (elements of R) of the 2D plain body: the block and the two face-flux arrays
template <int M>
__host__ __device__ constexpr int stage2d_smem_elems() {
    return ((TY_2D + 6) * (TX_2D + 6) + TY_2D * (TX_2D + 1) + (TY_2D + 1) * TX_2D) * M;
}

// One face of a 2D tile with the two-point Gauss rule (Sec. 7, k = 2 on the cross of Sec. 6):
// the face values at -+ 1/(2 sqrt 3) cell widths from the midpoint, their Lax-Friedrichs fluxes
// and h = (h(-) + h(+)) / 2.  S: the 6-cell stencil along the normal ([j * M + k]); su: the
// tile's cells with halo ([(by * BX + bx) * M + k]); (bx, by): the cell behind v^-, the cell
// behind v^+ one step of `along` further; `across`: the step across the line.  Each point
// counts as a face evaluation.
template <typename R, typename D, int KIND, int M>
__device__ __forceinline__ void gauss_face(const R* S, const R* su, int BX, int bx, int by, int along, int across,
                                           R alpha, const MethodParams& mp, int dir, R* h, R* h1, EtaCount& ec,
                                           bool counted) {
    constexpr D G = D(0.28867513459481288225);  // 1 / (2 sqrt 3)
    const int cl = by * BX + bx, cr = cl + along;
    R vm0[M], vp0[M], vm1[M], vp1[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
        auto at = [&](int c, int t) { return D(su[(c + t * across) * M + k]); };
        const CrossSide<D> l = cross_side<D>(at(cl, -1), at(cl, 0), at(cl, 1), at(cr, -1), at(cr, 0), at(cr, 1));
        const CrossSide<D> r = cross_side<D>(at(cr, -1), at(cr, 0), at(cr, 1), at(cl, -1), at(cl, 0), at(cl, 1));
        R w[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) w[j] = S[j * M + k];
        const uint32_t f0 = face_point_k2<R, D>(w, mp, &vm0[k], &vp0[k], l, r, -G);
        const uint32_t f1 = face_point_k2<R, D>(w, mp, &vm1[k], &vp1[k], l, r, G);
        if (counted) {
            ec.face(f0, 2);
            ec.face(f1, 2);
        }
    }
    lf_flux<R, KIND, M>(vm0, vp0, alpha, mp, dir, h1);
    lf_flux<R, KIND, M>(vm1, vp1, alpha, mp, dir, h);
#pragma unroll
    for (int k = 0; k < M; ++k) h[k] = R(0.5) * (h1[k] + h[k]);
}

template <typename R, typename D, int KIND>
__device__ __forceinline__ void stage2d_body(const Stage2DArgs& a, const Inst2D& in, Ctl* ctl, int tile,
                                             unsigned char* smem_raw) {
    constexpr int M = kind_m<KIND>();
    constexpr int BX = TX_2D + 6, BY = TY_2D + 6;
    R* su = reinterpret_cast<R*>(smem_raw);   // [BY * BX * M]
    R* hx = su + BY * BX * M;                 // [TY * (TX + 1) * M]
    R* hy = hx + TY_2D * (TX_2D + 1) * M;     // [(TY + 1) * TX * M]
    __shared__ double red[32];
    __shared__ int redbad[32];
    __shared__ double red2[32];
    __shared__ int redbad2[32];
    if (*(volatile int32_t*)&ctl->done) return;
    const int tx0 = (tile % in.tiles_x) * TX_2D;
    const int ty0 = (tile / in.tiles_x) * TY_2D;
    const int64_t nx = in.nx, ny = in.ny, cells = nx * ny;
    const R* uin = reinterpret_cast<const R*>(a.uin) + in.off;
    const int tid = threadIdx.x;
    const bool gauss = a.mp.k == 2 && a.mp.gauss_2d;
    const bool cross = gauss || (a.mp.k == 2 && a.mp.cross_2d &&
                                 (a.mp.scheme == NPW_RBF_ENO_ || a.mp.scheme == NPW_RBF_WENO_));
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const double inflow_k = a.mp.inflow[k];
        for (int rem = tid; rem < BX * BY; rem += blockDim.x) {
            const int by = rem / BX, bx = rem - by * BX;
            // the corners are read only by the 5-cell cross of k = 2 (transverse differences of
            // the halo cells next to the tile)
            const bool corner = (bx < 3 || bx >= TX_2D + 3) && (by < 3 || by >= TY_2D + 3);
            su[(by * BX + bx) * M + k] =
                (corner && !cross) ? R(0.0)
                                   : grid_get<R>(uin + k * cells, in, (int64_t)tx0 - 3 + bx, (int64_t)ty0 - 3 + by,
                                                 inflow_k);
        }
    }
    const double dt = *(volatile double*)&ctl->dt;
    const R ax = R(*(volatile double*)&ctl->alpha);
    const R ay = R(*(volatile double*)&ctl->alpha_y);
    EtaCount ec;
    const int cnt_x = (int)min((int64_t)TX_2D, nx - tx0), cnt_y = (int)min((int64_t)TY_2D, ny - ty0);
    const bool last_x = tx0 + TX_2D >= nx, last_y = ty0 + TY_2D >= ny;
    __syncthreads();
    // x faces: (qx, qy), qx = 0..TX, qy = 0..TY-1, stencil su[qy+3][qx .. qx+5]
    for (int f = tid; f < (TX_2D + 1) * TY_2D; f += blockDim.x) {
        const int qy = f / (TX_2D + 1), qx = f - qy * (TX_2D + 1);
        R S[6 * M], vm[M], vp[M], h[M];
        uint32_t fl[M];
#pragma unroll
        for (int j = 0; j < 6; ++j)
#pragma unroll
            for (int k = 0; k < M; ++k) S[j * M + k] = su[((qy + 3) * BX + qx + j) * M + k];
        if (gauss) {
            // two Gauss points (Sec. 7): the cross reconstruction at y_j -+ dy / (2 sqrt 3), the
            // mean of the two Lax-Friedrichs fluxes; transverse data of the cells qx-1 (v^-) and qx
            // (v^+) from rows qy-1..qy+1, each with the other as the cell across the face
            R h1[M];
            gauss_face<R, D, KIND, M>(S, su, BX, qx + 2, qy + 3, 1, BX, ax, a.mp, 0, h, h1, ec,
                                      qy < cnt_y && face_owned(qx, cnt_x, last_x));
#pragma unroll
            for (int k = 0; k < M; ++k) hx[(qy * (TX_2D + 1) + qx) * M + k] = h[k];
            continue;
        }
        if (cross) {
            // transverse (y) second differences of the cells qx-1 and qx of row qy
            D T[2 * M];
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const int bx = qx + 2 + c;
                    T[c * M + k] = (D(su[((qy + 2) * BX + bx) * M + k]) - D(2.0) * D(su[((qy + 3) * BX + bx) * M + k])) +
                                   D(su[((qy + 4) * BX + bx) * M + k]);
                }
            face_all<R, D, KIND, M, false>(S, a.mp, vm, vp, fl, T);
        } else {
            face_all<R, D, KIND, M, false>(S, a.mp, vm, vp, fl);
        }
        lf_flux<R, KIND, M>(vm, vp, ax, a.mp, 0, h);
#pragma unroll
        for (int k = 0; k < M; ++k) hx[(qy * (TX_2D + 1) + qx) * M + k] = h[k];
        if (qy < cnt_y && face_owned(qx, cnt_x, last_x))
#pragma unroll
            for (int k = 0; k < M; ++k) ec.face(fl[k], a.mp.k);
    }
    // y faces: (qx, qy), qx = 0..TX-1, qy = 0..TY, stencil su[qy .. qy+5][qx+3]
    for (int f = tid; f < TX_2D * (TY_2D + 1); f += blockDim.x) {
        const int qy = f / TX_2D, qx = f - qy * TX_2D;
        R S[6 * M], vm[M], vp[M], h[M];
        uint32_t fl[M];
#pragma unroll
        for (int j = 0; j < 6; ++j)
#pragma unroll
            for (int k = 0; k < M; ++k) S[j * M + k] = su[((qy + j) * BX + qx + 3) * M + k];
        if (gauss) {
            R h1[M];
            gauss_face<R, D, KIND, M>(S, su, BX, qx + 3, qy + 2, BX, 1, ay, a.mp, 1, h, h1, ec,
                                      qx < cnt_x && face_owned(qy, cnt_y, last_y));
#pragma unroll
            for (int k = 0; k < M; ++k) hy[(qy * TX_2D + qx) * M + k] = h[k];
            continue;
        }
        if (cross) {
            // transverse (x) second differences of the cells qy-1 and qy of column qx
            D T[2 * M];
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const int by = qy + 2 + c;
                    T[c * M + k] = (D(su[(by * BX + qx + 2) * M + k]) - D(2.0) * D(su[(by * BX + qx + 3) * M + k])) +
                                   D(su[(by * BX + qx + 4) * M + k]);
                }
            face_all<R, D, KIND, M, false>(S, a.mp, vm, vp, fl, T);
        } else {
            face_all<R, D, KIND, M, false>(S, a.mp, vm, vp, fl);
        }
        lf_flux<R, KIND, M>(vm, vp, ay, a.mp, 1, h);
#pragma unroll
        for (int k = 0; k < M; ++k) hy[(qy * TX_2D + qx) * M + k] = h[k];
        if (qx < cnt_x && face_owned(qy, cnt_y, last_y))
#pragma unroll
            for (int k = 0; k < M; ++k) ec.face(fl[k], a.mp.k);
    }
    flush_counts(ec, ctl, a.mp);
    __syncthreads();
    R* uout = reinterpret_cast<R*>(a.uout) + in.off;
    const R* un = reinterpret_cast<const R*>(a.un) + in.off;
    const R dtR = R(dt), dxR = R(in.dx), dyR = R(in.dy);
    double vmx = 0.0, vmy = 0.0;
    bool bad = false;
    {
        const int qy = tid / TX_2D, qx = tid - qy * TX_2D;
        const int64_t gi = tx0 + qx, gj = ty0 + qy;
        if (gi < nx && gj < ny) {
            R U[M];
#pragma unroll
            for (int k = 0; k < M; ++k) {
                R L = -((hx[(qy * (TX_2D + 1) + qx + 1) * M + k] - hx[(qy * (TX_2D + 1) + qx) * M + k]) / dxR);
                L = L - (hy[((qy + 1) * TX_2D + qx) * M + k] - hy[(qy * TX_2D + qx) * M + k]) / dyR;
                const R uk = su[((qy + 3) * BX + qx + 3) * M + k];
                const int64_t gidx = k * cells + gj * nx + gi;
                R o;
                if (a.stage == 0) {
                    o = uk + dtR * L;
                } else if (a.stage == 1) {
                    o = R(0.75) * un[gidx] + R(0.25) * (uk + dtR * L);
                } else {
                    o = stage3_w1<R>() * un[gidx] + stage3_w2<R>() * (uk + dtR * L);
                }
                uout[gidx] = o;
                U[k] = o;
                bad |= !finite_(o);
            }
            if (a.stage == 2) {
                double sx = (double)wave_speed<R, KIND>(U, a.mp, 0);
                double sy = (double)wave_speed<R, KIND>(U, a.mp, 1);
                bad |= !finite_(sx) || !finite_(sy);
                vmx = sx;
                vmy = sy;
            }
        }
    }
    if (a.stage == 2 && a.advance) {
        double bx = block_max_nan(vmx, bad, red, redbad);
        double by = block_max_nan(vmy, bad, red2, redbad2);
        if (tid == 0) {
            atomicMax(&ctl->alpha_next_bits, (unsigned long long)__double_as_longlong(bx));
            atomicMax(&ctl->alpha_y_next_bits, (unsigned long long)__double_as_longlong(by));
            __threadfence();
            unsigned prev = atomicAdd(&ctl->tiles_done, 1u);
            if (prev == (unsigned)(in.tiles_x * in.tiles_y) - 1u) {
                __threadfence();
                finalize_2d(ctl, in);
            }
        }
    }
}

template <typename R, int KIND>
__global__ void __launch_bounds__(TX_2D * TY_2D) alpha_init_2d_kernel(const R* __restrict__ u, const Inst2D* inst,
                                                                       Ctl* ctl, MethodParams mp) {
    constexpr int M = kind_m<KIND>();
    __shared__ double red[32];
    __shared__ int redbad[32];
    __shared__ double red2[32];
    __shared__ int redbad2[32];
    const Inst2D in = *inst;
    const int tx0 = (blockIdx.x % in.tiles_x) * TX_2D;
    const int ty0 = (blockIdx.x / in.tiles_x) * TY_2D;
    const int64_t cells = in.nx * in.ny;
    const int qy = threadIdx.x / TX_2D, qx = threadIdx.x - qy * TX_2D;
    const int64_t gi = tx0 + qx, gj = ty0 + qy;
    double sx = 0.0, sy = 0.0;
    bool bad = false;
    if (gi < in.nx && gj < in.ny) {
        R U[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            U[k] = u[in.off + k * cells + gj * in.nx + gi];
            bad |= !finite_(U[k]);
        }
        sx = (double)wave_speed<R, KIND>(U, mp, 0);
        sy = (double)wave_speed<R, KIND>(U, mp, 1);
        bad |= !finite_(sx) || !finite_(sy);
    }
    double bx = block_max_nan(sx, bad, red, redbad);
    double by = block_max_nan(sy, bad, red2, redbad2);
    if (threadIdx.x == 0) {
        atomicMax(&ctl->alpha_next_bits, (unsigned long long)__double_as_longlong(bx));
        atomicMax(&ctl->alpha_y_next_bits, (unsigned long long)__double_as_longlong(by));
    }
}

// ---------------------------------------------------------------------------------------
// One CTA per work item: the per-stage kernels of the 1D runtime (tile table) and of a single
// 2D instance (blockIdx.x = tile index).
// ---------------------------------------------------------------------------------------
template <typename R, typename D, int KIND, bool CHAR>
__global__ void __launch_bounds__(THREADS_1D) stage1d_kernel(Stage1DArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Tile td = a.tiles[blockIdx.x];
    stage1d_body<R, D, KIND, CHAR>(a, td, a.inst[td.inst], a.ctl + td.inst, smem_raw);
}

template <int KIND, int K>
__global__ void __launch_bounds__(THREADS_1D) stage1d_fast_kernel(Stage1DArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Tile td = a.tiles[blockIdx.x];
    stage1d_fast_body<KIND, K>(a, td, a.inst[td.inst], a.ctl + td.inst, smem_raw);
}

template <int KIND, int K>
__global__ void __launch_bounds__(TX_2D * TY_2D) stage2d_fast_kernel(Stage2DArgs a) {
    extern __shared__ __align__(16) float smem_f[];
    stage2d_fast_body<KIND, K>(a, *a.inst, a.ctl, blockIdx.x, smem_f);
}

template <typename R, typename D, int KIND>
__global__ void __launch_bounds__(TX_2D * TY_2D) stage2d_kernel(Stage2DArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    stage2d_body<R, D, KIND>(a, *a.inst, a.ctl, blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------------------------------
// Persistent work-queue kernel (QueueArgs): one launch per stage for every instance of a batch,
// 1D and 2D together.  Each CTA takes the next item from q.head[0] until the list is exhausted
// and runs the per-item body of the instance's kind: for the float state the compensated 1D
// body (or the face-based characteristic body) and the phased 2D body, for the double state the
// face-based bodies.  The bodies are those of the one-CTA-per-item kernels, so the results are
// the same bits.  The last CTA to finish resets the counters for the next launch (the next
// launch is ordered after this one on the stream).
// ---------------------------------------------------------------------------------------
template <typename R, int K, bool CHAR, int KIND>
__device__ __forceinline__ void queue_item_1d(const Stage1DArgs& a1, const Tile w, const InstDev& in, Ctl* ctl,
                                              unsigned char* smem) {
    if constexpr (sizeof(R) == sizeof(float) && !CHAR) {
        if (a1.stage == QUEUE_FUSED_STEP)
            step1d_fused_body<KIND, K>(a1, w, in, ctl, smem);
        else
            stage1d_fast_body<KIND, K>(a1, w, in, ctl, smem);
    } else
        stage1d_body<R, double, KIND, CHAR && KIND == NPW_FLUX_EULER1D_>(a1, w, in, ctl, smem);
}
template <typename R, int K, int KIND>
__device__ __forceinline__ void queue_item_2d(const Stage2DArgs& a2, const Inst2D& in, Ctl* ctl, int tile,
                                              unsigned char* smem) {
    if constexpr (sizeof(R) == sizeof(float))
        stage2d_fast_body<KIND, K>(a2, in, ctl, tile, reinterpret_cast<float*>(smem));
    else
        stage2d_body<R, double, KIND>(a2, in, ctl, tile, smem);
}

// CTAs per SM the register allocation aims for: 5 for the specialised mixed-precision k = 3
// kernels (48 registers a thread; their shared memory allows at least as many), else no bound
template <typename R, int K, bool CHAR, int SHAPE>
constexpr int queue_min_blocks() {
    return (sizeof(R) == sizeof(float) && K == 3 && !CHAR && SHAPE != QS_ANY && SHAPE != QS_2D_ADV) ? 5 : 1;
}

template <typename R, int K, bool CHAR, int SHAPE>
__device__ __forceinline__ void queue_stage_body(const QueueArgs& q) {
    static_assert(THREADS_1D == TX_2D * TY_2D, "1D and 2D items share the CTA shape");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    // stage input and output: u -> u1 -> u2 -> u (selects, not an indexed local array); the
    // fused 1D step reads the state buffer of this step's parity and writes the other
    const bool fused = q.stage == QUEUE_FUSED_STEP;
    const void* sin = fused ? (q.parity ? (const void*)q.s : q.u) : (q.stage == 0 ? q.u : (q.stage == 1 ? q.u1 : q.u2));
    void* sout = fused ? (q.parity ? q.u : (void*)q.s) : (q.stage == 0 ? q.u1 : (q.stage == 1 ? q.u2 : q.u));
    Stage1DArgs a1{};
    a1.uin = sin;
    a1.un = q.u;
    a1.uout = sout;
    a1.u = reinterpret_cast<float*>(q.u);
    a1.d1 = reinterpret_cast<float*>(q.u1);
    a1.d2 = reinterpret_cast<float*>(q.u2);
    a1.s = q.s;
    a1.c = q.c;
    a1.stage = q.stage;
    a1.advance = q.advance;
    a1.tile = q.tile;
    a1.mp = q.mp;
    Stage2DArgs a2{};
    a2.uin = sin;
    a2.un = q.u;
    a2.uout = sout;
    a2.stage = q.stage;
    a2.advance = q.advance;
    a2.mp = q.mp;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&q.head[0], 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= q.nitems) break;  // uniform over the CTA
        const Tile w = q.items[it];
        Ctl* ctl = q.ctl + w.inst;
        if constexpr (SHAPE == QS_1D_ADV) {
            queue_item_1d<R, K, CHAR, NPW_FLUX_ADVECTION_>(a1, w, q.inst1[w.inst], ctl, smem_raw);
        } else if constexpr (SHAPE == QS_1D_BURG) {
            queue_item_1d<R, K, CHAR, NPW_FLUX_BURGERS_>(a1, w, q.inst1[w.inst], ctl, smem_raw);
        } else if constexpr (SHAPE == QS_1D_EULER) {
            queue_item_1d<R, K, CHAR, NPW_FLUX_EULER1D_>(a1, w, q.inst1[w.inst], ctl, smem_raw);
        } else if constexpr (SHAPE == QS_2D_ADV) {
            queue_item_2d<R, K, NPW_FLUX_ADVECTION_>(a2, q.inst2[w.inst], ctl, w.start, smem_raw);
        } else if constexpr (SHAPE == QS_2D_BURG) {
            queue_item_2d<R, K, NPW_FLUX_BURGERS_>(a2, q.inst2[w.inst], ctl, w.start, smem_raw);
        } else if constexpr (SHAPE == QS_2D_EULER) {
            queue_item_2d<R, K, NPW_FLUX_EULER2D_>(a2, q.inst2[w.inst], ctl, w.start, smem_raw);
        } else if (q.is2d[w.inst]) {
            const int kind = q.kind[w.inst];
            const Inst2D& in = q.inst2[w.inst];
            if (kind == NPW_FLUX_EULER2D_)
                queue_item_2d<R, K, NPW_FLUX_EULER2D_>(a2, in, ctl, w.start, smem_raw);
            else if (kind == NPW_FLUX_BURGERS_)
                queue_item_2d<R, K, NPW_FLUX_BURGERS_>(a2, in, ctl, w.start, smem_raw);
            else
                queue_item_2d<R, K, NPW_FLUX_ADVECTION_>(a2, in, ctl, w.start, smem_raw);
        } else {
            const int kind = q.kind[w.inst];
            const InstDev& in = q.inst1[w.inst];
            if (kind == NPW_FLUX_EULER1D_)
                queue_item_1d<R, K, CHAR, NPW_FLUX_EULER1D_>(a1, w, in, ctl, smem_raw);
            else if (kind == NPW_FLUX_BURGERS_)
                queue_item_1d<R, K, CHAR, NPW_FLUX_BURGERS_>(a1, w, in, ctl, smem_raw);
            else
                queue_item_1d<R, K, CHAR, NPW_FLUX_ADVECTION_>(a1, w, in, ctl, smem_raw);
        }
        __syncthreads();  // shared memory and s_item are reused by the next item
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&q.head[1], 1u) == gridDim.x - 1u) {  // every CTA has left the loop
            q.head[0] = 0u;
            q.head[1] = 0u;
        }
    }
}


// the kernels: one without a register bound, one bounded at 5 CTAs per SM (see queue_min_blocks)
template <typename R, int K, bool CHAR, int SHAPE>
__global__ void __launch_bounds__(THREADS_1D) queue_stage_kernel(QueueArgs q) {
    queue_stage_body<R, K, CHAR, SHAPE>(q);
}
template <typename R, int K, bool CHAR, int SHAPE>
__global__ void __launch_bounds__(THREADS_1D, 5) queue_stage_kernel_b5(QueueArgs q) {
    queue_stage_body<R, K, CHAR, SHAPE>(q);
}

// alpha^0 of every instance of a queue batch: one CTA per item, the wave speeds of its cells
// (2D: both directions) into the instance's running maxima
template <typename R, int KIND>
__device__ __forceinline__ void queue_speed_cell(const R* base, int64_t stride, int64_t i, const MethodParams& mp,
                                                 bool two_d, double* sx, double* sy, bool* bad) {
    constexpr int M = kind_m<KIND>();
    R U[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
        U[k] = base[k * stride + i];
        *bad |= !finite_(U[k]);
    }
    const double x = (double)wave_speed<R, KIND>(U, mp, 0);
    const double y = two_d ? (double)wave_speed<R, KIND>(U, mp, 1) : 0.0;
    *bad |= !finite_(x) || !finite_(y);
    *sx = x > *sx ? x : *sx;
    *sy = y > *sy ? y : *sy;
}

template <typename R>
__global__ void __launch_bounds__(THREADS_1D) queue_alpha_kernel(QueueArgs q) {
    __shared__ double red[32];
    __shared__ int redbad[32];
    __shared__ double red2[32];
    __shared__ int redbad2[32];
    const Tile w = q.items[blockIdx.x];
    const bool two_d = q.is2d[w.inst] != 0;
    const int kind = q.kind[w.inst];
    const R* u = reinterpret_cast<const R*>(q.u);
    double sx = 0.0, sy = 0.0;
    bool bad = false;
    if (two_d) {
        const Inst2D in = q.inst2[w.inst];
        const int64_t cells = in.nx * in.ny;
        const int tx0 = (w.start % in.tiles_x) * TX_2D, ty0 = (w.start / in.tiles_x) * TY_2D;
        const int qy = threadIdx.x / TX_2D, qx = threadIdx.x - qy * TX_2D;
        const int64_t gi = tx0 + qx, gj = ty0 + qy;
        if (gi < in.nx && gj < in.ny) {
            const R* base = u + in.off;
            const int64_t i = gj * in.nx + gi;
            if (kind == NPW_FLUX_EULER2D_)
                queue_speed_cell<R, NPW_FLUX_EULER2D_>(base, cells, i, q.mp, true, &sx, &sy, &bad);
            else if (kind == NPW_FLUX_BURGERS_)
                queue_speed_cell<R, NPW_FLUX_BURGERS_>(base, cells, i, q.mp, true, &sx, &sy, &bad);
            else
                queue_speed_cell<R, NPW_FLUX_ADVECTION_>(base, cells, i, q.mp, true, &sx, &sy, &bad);
        }
    } else {
        const InstDev in = q.inst1[w.inst];
        const int cnt = (int)((in.n - w.start) < q.tile ? (in.n - w.start) : q.tile);
        const R* base = u + in.off;
        for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
            const int64_t i = w.start + c;
            if (kind == NPW_FLUX_EULER1D_)
                queue_speed_cell<R, NPW_FLUX_EULER1D_>(base, in.n, i, q.mp, false, &sx, &sy, &bad);
            else if (kind == NPW_FLUX_BURGERS_)
                queue_speed_cell<R, NPW_FLUX_BURGERS_>(base, in.n, i, q.mp, false, &sx, &sy, &bad);
            else
                queue_speed_cell<R, NPW_FLUX_ADVECTION_>(base, in.n, i, q.mp, false, &sx, &sy, &bad);
        }
    }
    const double bx = block_max_nan(sx, bad, red, redbad);
    const double by = block_max_nan(sy, bad, red2, redbad2);
    if (threadIdx.x == 0) {
        Ctl* ctl = q.ctl + w.inst;
        atomicMax(&ctl->alpha_next_bits, (unsigned long long)__double_as_longlong(bx));
        if (two_d) atomicMax(&ctl->alpha_y_next_bits, (unsigned long long)__double_as_longlong(by));
    }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
// smooth data for the tile autotuner: m = 1: 1 + 0.5 sin(16 pi x); m = 3: a quiet Euler state
// (rho = 1 + 0.2 sin(16 pi x), u = 0, p = 1, gamma = 1.4)
template <typename R>
__global__ void tune_init_kernel(R* u, int64_t n, int m) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = ((double)i + 0.5) / (double)n;
    const double s = sin(16.0 * 3.141592653589793 * x);
    if (m == 1) {
        u[i] = R(1.0 + 0.5 * s);
    } else {
        u[i] = R(1.0 + 0.2 * s);
        for (int k = 1; k < m; ++k) u[k * n + i] = R(k == m - 1 ? 2.5 : 0.0);
    }
}

template <typename R, typename D>
struct Launchers {
    static cudaError_t reconstruct(const R* u, int64_t n, int m, int bc, const MethodParams& mp, R* vm, R* vp,
                                   uint8_t* flags, R* eta, cudaStream_t s) {
        const int threads = 128;
        const unsigned blocks = (unsigned)((n + 1 + threads - 1) / threads);
        if (m == 1)
            reconstruct_kernel<R, D, 1, false><<<blocks, threads, 0, s>>>(u, n, bc, mp, vm, vp, flags, eta);
        else if (m == 3 && mp.characteristic)
            reconstruct_kernel<R, D, 3, true><<<blocks, threads, 0, s>>>(u, n, bc, mp, vm, vp, flags, eta);
        else if (m == 3)
            reconstruct_kernel<R, D, 3, false><<<blocks, threads, 0, s>>>(u, n, bc, mp, vm, vp, flags, eta);
        else if (m == 4)
            reconstruct_kernel<R, D, 4, false><<<blocks, threads, 0, s>>>(u, n, bc, mp, vm, vp, flags, eta);
        else
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    }

    static cudaError_t flux(const R* vm, const R* vp, int64_t nf, int kind, double alpha, const MethodParams& mp, R* h,
                            cudaStream_t s) {
        const int threads = 128;
        const unsigned blocks = (unsigned)((nf + threads - 1) / threads);
        switch (kind) {
            case NPW_FLUX_ADVECTION:
                flux_kernel<R, NPW_FLUX_ADVECTION_><<<blocks, threads, 0, s>>>(vm, vp, nf, R(alpha), mp, h);
                break;
            case NPW_FLUX_BURGERS:
                flux_kernel<R, NPW_FLUX_BURGERS_><<<blocks, threads, 0, s>>>(vm, vp, nf, R(alpha), mp, h);
                break;
            case NPW_FLUX_EULER1D:
                flux_kernel<R, NPW_FLUX_EULER1D_><<<blocks, threads, 0, s>>>(vm, vp, nf, R(alpha), mp, h);
                break;
            default:
                return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }

    static cudaError_t alpha_init(const void* u, const InstDev* inst, Ctl* ctl, const Tile* tiles, int ntiles, int tile,
                                  int kind, const MethodParams& mp, cudaStream_t s) {
        const R* uu = reinterpret_cast<const R*>(u);
        switch (kind) {
            case NPW_FLUX_ADVECTION:
                alpha_init_kernel<R, NPW_FLUX_ADVECTION_><<<ntiles, THREADS_1D, 0, s>>>(uu, inst, ctl, tiles, tile, mp);
                break;
            case NPW_FLUX_BURGERS:
                alpha_init_kernel<R, NPW_FLUX_BURGERS_><<<ntiles, THREADS_1D, 0, s>>>(uu, inst, ctl, tiles, tile, mp);
                break;
            case NPW_FLUX_EULER1D:
                alpha_init_kernel<R, NPW_FLUX_EULER1D_><<<ntiles, THREADS_1D, 0, s>>>(uu, inst, ctl, tiles, tile, mp);
                break;
            default:
                return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }

    template <int KIND, bool CHAR>
    static cudaError_t stage_k(const Stage1DArgs& a, cudaStream_t s) {
        constexpr int M = kind_m<KIND>();
        const size_t smem = (size_t)((a.tile + 6) + (a.tile + 1)) * M * sizeof(R);
        auto kern = stage1d_kernel<R, D, KIND, CHAR>;
        static bool attr_set = false;
        if (!attr_set) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            if (e != cudaSuccess) return e;
            attr_set = true;
        }
        kern<<<a.ntiles, THREADS_1D, smem, s>>>(a);
        return cudaGetLastError();
    }

    template <int KIND, int K>
    static cudaError_t stage_fast(const Stage1DArgs& a, cudaStream_t s) {
        constexpr int M = kind_m<KIND>();
        const size_t smem = (size_t)(a.tile + 6) * 4 * M * sizeof(float);
        auto kern = stage1d_fast_kernel<KIND, K>;
        static bool attr_set = false;
        if (!attr_set) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            if (e != cudaSuccess) return e;
            attr_set = true;
        }
        kern<<<a.ntiles, THREADS_1D, smem, s>>>(a);
        return cudaGetLastError();
    }

    static cudaError_t stage1d(const Stage1DArgs& a, int kind, cudaStream_t s) {
        if constexpr (sizeof(R) == sizeof(float)) {
            if (!a.mp.characteristic) {
                const bool k2 = a.mp.k == 2;
                switch (kind) {
                    case NPW_FLUX_ADVECTION:
                        return k2 ? stage_fast<NPW_FLUX_ADVECTION_, 2>(a, s) : stage_fast<NPW_FLUX_ADVECTION_, 3>(a, s);
                    case NPW_FLUX_BURGERS:
                        return k2 ? stage_fast<NPW_FLUX_BURGERS_, 2>(a, s) : stage_fast<NPW_FLUX_BURGERS_, 3>(a, s);
                    case NPW_FLUX_EULER1D:
                        return k2 ? stage_fast<NPW_FLUX_EULER1D_, 2>(a, s) : stage_fast<NPW_FLUX_EULER1D_, 3>(a, s);
                    default: return cudaErrorInvalidValue;
                }
            }
        }
        switch (kind) {
            case NPW_FLUX_ADVECTION: return stage_k<NPW_FLUX_ADVECTION_, false>(a, s);
            case NPW_FLUX_BURGERS: return stage_k<NPW_FLUX_BURGERS_, false>(a, s);
            case NPW_FLUX_EULER1D:
                return a.mp.characteristic ? stage_k<NPW_FLUX_EULER1D_, true>(a, s)
                                           : stage_k<NPW_FLUX_EULER1D_, false>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }

    static cudaError_t alpha_init_2d(const void* u, const Inst2D* inst, int tiles, Ctl* ctl, int kind,
                                     const MethodParams& mp, cudaStream_t s) {
        const R* uu = reinterpret_cast<const R*>(u);
        switch (kind) {
            case NPW_FLUX_ADVECTION:
                alpha_init_2d_kernel<R, NPW_FLUX_ADVECTION_><<<tiles, TX_2D * TY_2D, 0, s>>>(uu, inst, ctl, mp);
                break;
            case NPW_FLUX_BURGERS:
                alpha_init_2d_kernel<R, NPW_FLUX_BURGERS_><<<tiles, TX_2D * TY_2D, 0, s>>>(uu, inst, ctl, mp);
                break;
            case NPW_FLUX_EULER2D:
                alpha_init_2d_kernel<R, NPW_FLUX_EULER2D_><<<tiles, TX_2D * TY_2D, 0, s>>>(uu, inst, ctl, mp);
                break;
            default:
                return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }

    static cudaError_t stage2d(const Stage2DArgs& a, int tiles, int kind, cudaStream_t s) {
        if constexpr (sizeof(R) == sizeof(float)) {
            if (a.mp.gauss_2d) {
                // the two-point Gauss rule with a float state: the face-based body, shape
                // parameters, ENO choices, switch and smoothness indicators in double from the
                // float cell averages, candidates, weights, flux and update in float
                switch (kind) {
                    case NPW_FLUX_ADVECTION:
                        stage2d_kernel<float, double, NPW_FLUX_ADVECTION_><<<tiles, TX_2D * TY_2D, stage2d_smem_elems<1>() * sizeof(float), s>>>(a);
                        break;
                    case NPW_FLUX_BURGERS:
                        stage2d_kernel<float, double, NPW_FLUX_BURGERS_><<<tiles, TX_2D * TY_2D, stage2d_smem_elems<1>() * sizeof(float), s>>>(a);
                        break;
                    case NPW_FLUX_EULER2D:
                        stage2d_kernel<float, double, NPW_FLUX_EULER2D_><<<tiles, TX_2D * TY_2D, stage2d_smem_elems<4>() * sizeof(float), s>>>(a);
                        break;
                    default:
                        return cudaErrorInvalidValue;
                }
                return cudaGetLastError();
            }
            // the mixed path: the phased kernel, k = 3 or k = 2
            switch (kind * 4 + a.mp.k) {
                case NPW_FLUX_ADVECTION * 4 + 3:
                    stage2d_fast_kernel<NPW_FLUX_ADVECTION_, 3><<<tiles, TX_2D * TY_2D, stage2d_fast_smem_floats<1>() * sizeof(float), s>>>(a);
                    break;
                case NPW_FLUX_BURGERS * 4 + 3:
                    stage2d_fast_kernel<NPW_FLUX_BURGERS_, 3><<<tiles, TX_2D * TY_2D, stage2d_fast_smem_floats<1>() * sizeof(float), s>>>(a);
                    break;
                case NPW_FLUX_EULER2D * 4 + 3:
                    stage2d_fast_kernel<NPW_FLUX_EULER2D_, 3><<<tiles, TX_2D * TY_2D, stage2d_fast_smem_floats<4>() * sizeof(float), s>>>(a);
                    break;
                case NPW_FLUX_ADVECTION * 4 + 2:
                    stage2d_fast_kernel<NPW_FLUX_ADVECTION_, 2><<<tiles, TX_2D * TY_2D, stage2d_fast_smem_floats<1>() * sizeof(float), s>>>(a);
                    break;
                case NPW_FLUX_BURGERS * 4 + 2:
                    stage2d_fast_kernel<NPW_FLUX_BURGERS_, 2><<<tiles, TX_2D * TY_2D, stage2d_fast_smem_floats<1>() * sizeof(float), s>>>(a);
                    break;
                case NPW_FLUX_EULER2D * 4 + 2:
                    stage2d_fast_kernel<NPW_FLUX_EULER2D_, 2><<<tiles, TX_2D * TY_2D, stage2d_fast_smem_floats<4>() * sizeof(float), s>>>(a);
                    break;
                default:
                    return cudaErrorInvalidValue;
            }
            return cudaGetLastError();
        }
        switch (kind) {
            case NPW_FLUX_ADVECTION:
                stage2d_kernel<R, D, NPW_FLUX_ADVECTION_><<<tiles, TX_2D * TY_2D, stage2d_smem_elems<1>() * sizeof(R), s>>>(a);
                break;
            case NPW_FLUX_BURGERS:
                stage2d_kernel<R, D, NPW_FLUX_BURGERS_><<<tiles, TX_2D * TY_2D, stage2d_smem_elems<1>() * sizeof(R), s>>>(a);
                break;
            case NPW_FLUX_EULER2D:
                stage2d_kernel<R, D, NPW_FLUX_EULER2D_><<<tiles, TX_2D * TY_2D, stage2d_smem_elems<4>() * sizeof(R), s>>>(a);
                break;
            default:
                return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
};

}  // namespace npw
