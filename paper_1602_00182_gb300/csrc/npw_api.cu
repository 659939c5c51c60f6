// npw_api.cu -- host runtime of libnpweno: argument checks, workspace layout, device-side
// time control kernels, the solve loops and the C ABI of include/npweno.h.
#include <cuda_runtime.h>

#include <time.h>

#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <deque>
#include <string>
#include <array>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "npw_internal.h"

namespace {

thread_local std::string g_err;

npw_status fail(npw_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
npw_status fail(npw_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

npw_status cuda_fail(cudaError_t e, const char* where) {
    return fail(NPW_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define NPW_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int flux_m(int kind) { return kind == NPW_FLUX_EULER1D ? 3 : (kind == NPW_FLUX_EULER2D ? 4 : 1); }

size_t elem_size(const npw_params* p) { return p->precision == NPW_FP32_MIXED ? sizeof(float) : sizeof(double); }

npw_status check_params(const npw_params* p) {
    if (!p) return fail(NPW_EINVAL, "params is NULL");
    if (p->k != 2 && p->k != 3) return fail(NPW_EINVAL, "k must be 2 (ENO2 / WENO3) or 3 (ENO3 / WENO5), got %d", p->k);
    if (p->scheme < NPW_ENO || p->scheme > NPW_RBF_WENO) return fail(NPW_EINVAL, "bad scheme %d", p->scheme);
    if (p->rbf != NPW_RBF_MQ && p->rbf != NPW_RBF_GA) return fail(NPW_EINVAL, "bad rbf %d", p->rbf);
    if (p->switch_variant < 0 || p->switch_variant > 1) return fail(NPW_EINVAL, "bad switch_variant");
    if (p->precision != NPW_FP64 && p->precision != NPW_FP32_MIXED) return fail(NPW_EINVAL, "bad precision");
    if (p->eta_eval < 0 || p->eta_eval > 1) return fail(NPW_EINVAL, "bad eta_eval %d", p->eta_eval);
    if (p->batch_mode < 0 || p->batch_mode > 1) return fail(NPW_EINVAL, "bad batch_mode %d", p->batch_mode);
    if (p->cross_2d < 0 || p->cross_2d > 1) return fail(NPW_EINVAL, "bad cross_2d %d", p->cross_2d);
    if (p->gauss_2d < 0 || p->gauss_2d > 1) return fail(NPW_EINVAL, "bad gauss_2d %d", p->gauss_2d);
    if (p->tile_1d != 0 && p->tile_1d != 256 && p->tile_1d != 512 && p->tile_1d != 1024 && p->tile_1d != 2048)
        return fail(NPW_EINVAL, "tile_1d must be 0, 256, 512, 1024 or 2048, got %d", p->tile_1d);
    if (!(p->eps_weno > 0.0)) return fail(NPW_EINVAL, "eps_weno must be > 0");
    if (!(p->gamma > 1.0)) return fail(NPW_EINVAL, "gamma must be > 1");
    return NPW_OK;
}

// the two-point Gauss rule of the 2D entry points: k = 2, the cross form for the RBF schemes;
// both precisions in npweno_rk3_step_2d / npweno_solve_2d, the FP64 path in the work queue
npw_status check_gauss(const npw_params* p, bool queue = false) {
    if (!p->gauss_2d) return NPW_OK;
    if (p->k != 2) return fail(NPW_EINVAL, "gauss_2d needs k = 2 (the point reconstruction of Sec. 6)");
    if ((p->scheme == NPW_RBF_ENO || p->scheme == NPW_RBF_WENO) && !p->cross_2d)
        return fail(NPW_EINVAL, "gauss_2d with an RBF scheme needs cross_2d = 1");
    if (queue && p->precision != NPW_FP64)
        return fail(NPW_EINVAL, "the work queue runs gauss_2d in NPW_FP64 (NPW_FP32_MIXED: npweno_solve_2d)");
    return NPW_OK;
}

npw::MethodParams method(const npw_params* p) {
    npw::MethodParams mp{};
    mp.scheme = p->scheme;
    mp.rbf = p->rbf;
    mp.monotone_switch = p->monotone_switch ? 1 : 0;
    mp.switch_variant = p->switch_variant;
    mp.characteristic = p->characteristic ? 1 : 0;
    mp.eta_eval = p->eta_eval;
    mp.k = p->k;
    mp.cross_2d = p->cross_2d ? 1 : 0;
    mp.gauss_2d = p->gauss_2d ? 1 : 0;
    mp.eps_M = p->eps_M;
    mp.eps_weno = p->eps_weno;
    mp.gamma = p->gamma;
    mp.adv_speed = p->adv_speed;
    mp.adv_speed_y = p->adv_speed_y;
    for (int k = 0; k < 4; ++k) mp.inflow[k] = p->inflow[k];
    // automatic guard: none for the double state (the paper's eps_M alone), eight units of
    // float round-off for the float state, whose noise a fixed eps_M = 1e-12 does not cover
    if (p->eta_guard > 0.0)
        mp.eta_guard = p->eta_guard;
    else if (p->eta_guard == 0.0 && p->precision == NPW_FP32_MIXED)
        mp.eta_guard = 8.0 * 5.9604644775390625e-08;
    else
        mp.eta_guard = 0.0;
    // the shape parameter exactly as printed unless a bound is asked for
    mp.eta_max = p->eta_max > 0.0 ? p->eta_max : 0.0;
    mp.tie_tol = p->tie_tol > 0.0 ? p->tie_tol : 1e-10;
    mp.max_steps = p->max_steps > 0 ? p->max_steps : 0;
    mp.eps_weno_f = (float)mp.eps_weno;
    mp.eps_M_f = (float)mp.eps_M;
    mp.eps_M_lo_f = (float)(mp.eps_M - (double)mp.eps_M_f);
    mp.eta_guard_f = (float)mp.eta_guard;
    mp.eta_max_f = (float)mp.eta_max;
    mp.gamma_f = (float)mp.gamma;
    mp.adv_speed_f = (float)mp.adv_speed;
    mp.adv_speed_y_f = (float)mp.adv_speed_y;
    for (int k = 0; k < 4; ++k) mp.inflow_f[k] = (float)mp.inflow[k];
    return mp;
}

npw_status check_kind_1d(int kind, int m, const npw_params* p) {
    if (kind != NPW_FLUX_ADVECTION && kind != NPW_FLUX_BURGERS && kind != NPW_FLUX_EULER1D)
        return fail(NPW_EINVAL, "flux kind %d is not a 1D flux", kind);
    if (m != flux_m(kind)) return fail(NPW_EINVAL, "m = %d does not match flux kind %d", m, kind);
    if (p->characteristic && kind != NPW_FLUX_EULER1D)
        return fail(NPW_EINVAL, "characteristic reconstruction needs the 1D Euler flux");
    return NPW_OK;
}

npw_status check_bc(int bc) {
    if (bc < NPW_BC_PERIODIC || bc > NPW_BC_INFLOW) return fail(NPW_EINVAL, "bad boundary condition %d", bc);
    return NPW_OK;
}

// ---------------------------------------------------------------------------------------
// Workspace layout of the 1D runtime: two stage buffers (u1, u2) of the arena size, the
// instance table, the per-instance control words, the tile table and the poll words.
// ---------------------------------------------------------------------------------------
struct Layout1D {
    size_t u1, u2, inst, ctl, tiles, poll, list, sbuf, cbuf, total;
};

Layout1D layout_1d(int64_t arena_elems, int count, int64_t ntiles, size_t esz) {
    Layout1D L{};
    size_t o = 0;
    L.list = o;
    o = align256(o + sizeof(int32_t) * (size_t)count);
    L.u1 = o;
    o = align256(o + (size_t)arena_elems * esz);
    L.u2 = o;
    o = align256(o + (size_t)arena_elems * esz);
    // compensated float path: next state s and carry c (float, arena-shaped)
    L.sbuf = o;
    o = align256(o + (esz == sizeof(float) ? (size_t)arena_elems * sizeof(float) : 0));
    L.cbuf = o;
    o = align256(o + (esz == sizeof(float) ? (size_t)arena_elems * sizeof(float) : 0));
    L.inst = o;
    o = align256(o + sizeof(npw::InstDev) * (size_t)count);
    L.ctl = o;
    o = align256(o + sizeof(npw::Ctl) * (size_t)count);
    L.tiles = o;
    o = align256(o + sizeof(npw::Tile) * (size_t)ntiles);
    L.poll = o;
    o = align256(o + 4 * sizeof(long long));
    L.total = o;
    return L;
}

// tiles of an instance; the default (the smallest tile a run may use) sizes the tile tables
int64_t tiles_of(int64_t n, int tile = npw::TILE_1D_MIN) { return (n + tile - 1) / tile; }

double wait_timeout_s() {
    const char* e = getenv("NPW_WAIT_TIMEOUT_S");
    double v = e ? atof(e) : 0.0;
    return v > 0.0 ? v : 1800.0;
}

// Wait for the stream with a deadline (polling; never an unbounded block).
npw_status bounded_sync(cudaStream_t s) {
    cudaEvent_t ev;
    NPW_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, s);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev);
        return cuda_fail(e, "cudaEventRecord");
    }
    auto t0 = std::chrono::steady_clock::now();
    const double limit = wait_timeout_s();
    while (true) {
        e = cudaEventQuery(ev);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) {
            cudaEventDestroy(ev);
            return cuda_fail(e, "cudaEventQuery");
        }
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > limit) {
            cudaEventDestroy(ev);
            return fail(NPW_ETIMEOUT, "stream did not complete within %.0f s", limit);
        }
        if (el > 1e-3) {
            struct timespec ts = {0, 20000};
            nanosleep(&ts, nullptr);
        }
    }
    cudaEventDestroy(ev);
    return NPW_OK;
}

// ---------------------------------------------------------------------------------------
// Profiling: launch counters and event-bracketed stage kernels
// ---------------------------------------------------------------------------------------
struct Profiler {
    std::mutex mu;
    bool on = false;
    int64_t launches = 0, stage_launches = 0, timed = 0;
    double stage_ms = 0.0;
    int64_t res_launches[4] = {0, 0, 0, 0};
    double res_ms[4] = {0.0, 0.0, 0.0, 0.0};
    // pending event pairs with the slot they add to: -1 = stage kernel, 0..3 = resident class
    std::vector<std::pair<std::pair<cudaEvent_t, cudaEvent_t>, int>> pending;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
};
Profiler& prof() {
    static Profiler p;
    return p;
}
void count_launch(int64_t k = 1) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.launches += k;
}
// set while a step sequence is captured into a CUDA graph: launches are counted, and timed,
// when the graph is replayed instead
thread_local bool t_capturing = false;

// returns the event pair to bracket a stage launch, or a replay of nlaunch captured stage
// launches (null events when profiling is off)
std::pair<cudaEvent_t, cudaEvent_t> stage_begin(cudaStream_t s, int slot = -1, int64_t nlaunch = 1) {
    if (t_capturing) return {nullptr, nullptr};
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.launches += nlaunch;
    if (slot < 0)
        p.stage_launches += nlaunch;
    else
        p.res_launches[slot] += nlaunch;
    if (!p.on) return {nullptr, nullptr};
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (!p.pool.empty()) {
        ev = p.pool.back();
        p.pool.pop_back();
    } else if (cudaEventCreate(&ev.first) != cudaSuccess || cudaEventCreate(&ev.second) != cudaSuccess) {
        return {nullptr, nullptr};
    }
    cudaEventRecord(ev.first, s);
    return ev;
}
void stage_end(std::pair<cudaEvent_t, cudaEvent_t> ev, cudaStream_t s, int slot = -1) {
    if (!ev.first) return;
    cudaEventRecord(ev.second, s);
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.pending.push_back({ev, slot});
}
// after the stream has been waited for: sum the elapsed times of completed pairs
void profile_collect() {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    std::vector<std::pair<std::pair<cudaEvent_t, cudaEvent_t>, int>> still;
    for (auto& item : p.pending) {
        auto& ev = item.first;
        if (cudaEventQuery(ev.second) == cudaSuccess) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) {
                if (item.second < 0) {
                    p.stage_ms += ms;
                    p.timed += 1;
                } else {
                    p.res_ms[item.second] += ms;
                }
            }
            p.pool.push_back(ev);
        } else {
            still.push_back(item);
        }
    }
    p.pending.swap(still);
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Device-side time control helpers (precision independent)
// ---------------------------------------------------------------------------------------
namespace npw {

// mode 0: reset; mode 1: start a solve (dt from alpha^0); mode 2: one step with fixed dt
__global__ void ctl_start_kernel(Ctl* ctl, const InstDev* inst, int count, int mode, double dt_fixed,
                                 int64_t max_steps) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    Ctl* c = ctl + i;
    if (mode == 0) {
        memset(c, 0, sizeof(Ctl));
        return;
    }
    double a = __longlong_as_double((long long)c->alpha_next_bits);
    c->alpha_next_bits = 0ull;
    c->tiles_done = 0u;
    if (!(a - a == 0.0)) {
        c->status = NPW_ENONFINITE;
        c->done = 1;
        return;
    }
    c->alpha = a;
    c->alpha_max = a;
    if (mode == 2) {
        c->dt = dt_fixed;
        c->last = 0;
        c->done = 0;
        return;
    }
    const InstDev in = inst[i];
    c->t = 0.0;
    if (!(c->t < in.t_end) || in.ntiles == 0) {  // finished, or solved by the resident kernel
        c->done = 1;
        return;
    }
    double rate = a / in.dx;
    double dt = (rate > 0.0) ? in.cfl / rate : in.t_end - c->t;
    int last = 0;
    if (c->t + dt * (1.0 + 1e-10) >= in.t_end) {
        dt = in.t_end - c->t;
        last = 1;
    }
    c->dt = dt;
    c->last = last;
    c->step_cap = step_cap(in.t_end - c->t, dt, max_steps);
}

__global__ void ctl_start_2d_kernel(Ctl* c, const Inst2D* inst, int mode, double dt_fixed, int64_t max_steps) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (mode == 0) {
        memset(c, 0, sizeof(Ctl));
        return;
    }
    double ax = __longlong_as_double((long long)c->alpha_next_bits);
    double ay = __longlong_as_double((long long)c->alpha_y_next_bits);
    c->alpha_next_bits = 0ull;
    c->alpha_y_next_bits = 0ull;
    c->tiles_done = 0u;
    if (!(ax - ax == 0.0) || !(ay - ay == 0.0)) {
        c->status = NPW_ENONFINITE;
        c->done = 1;
        return;
    }
    c->alpha = ax;
    c->alpha_y = ay;
    c->alpha_max = ax > ay ? ax : ay;
    if (mode == 2) {
        c->dt = dt_fixed;
        c->last = 0;
        c->done = 0;
        return;
    }
    const Inst2D in = *inst;
    c->t = 0.0;
    if (!(c->t < in.t_end)) {
        c->done = 1;
        return;
    }
    double rate = ax / in.dx + ay / in.dy;
    double dt = (rate > 0.0) ? in.cfl / rate : in.t_end - c->t;
    int last = 0;
    if (c->t + dt * (1.0 + 1e-10) >= in.t_end) {
        dt = in.t_end - c->t;
        last = 1;
    }
    c->dt = dt;
    c->last = last;
    c->step_cap = step_cap(in.t_end - c->t, dt, max_steps);
}

// poll[0] = active instances, poll[1] = largest remaining step estimate
__global__ void count_active_kernel(const Ctl* ctl, const InstDev* inst, int count, const Inst2D* inst2d,
                                    long long* poll) {
    __shared__ long long s_act[256], s_rem[256];
    long long act = 0, rem = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const Ctl& c = ctl[i];
        if (!c.done) {
            ++act;
            double t_end = inst ? inst[i].t_end : inst2d->t_end;
            double r = (c.dt > 0.0) ? (t_end - c.t) / c.dt : 1.0;
            long long ri = (long long)(r < 1e9 ? r : 1e9) + 1;
            rem = ri > rem ? ri : rem;
        }
    }
    s_act[threadIdx.x] = act;
    s_rem[threadIdx.x] = rem;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_act[threadIdx.x] += s_act[threadIdx.x + o];
            s_rem[threadIdx.x] = s_rem[threadIdx.x + o] > s_rem[threadIdx.x] ? s_rem[threadIdx.x + o] : s_rem[threadIdx.x];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        poll[0] = s_act[0];
        poll[1] = s_rem[0];
    }
}

// Server slots: mode 0 zeroes the control words of the listed slots; mode 1 starts them
// (alpha^0 from the running max bits, first dt).
__global__ void ctl_slots_kernel(Ctl* ctl, const InstDev* inst, const int32_t* list, int count, int mode,
                                 int64_t max_steps) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int i = list[k];
    Ctl* c = ctl + i;
    if (mode == 0) {
        memset(c, 0, sizeof(Ctl));
        return;
    }
    const double a = __longlong_as_double((long long)c->alpha_next_bits);
    c->alpha_next_bits = 0ull;
    c->tiles_done = 0u;
    if (!(a - a == 0.0)) {
        c->status = NPW_ENONFINITE;
        c->done = 1;
        return;
    }
    c->alpha = a;
    c->alpha_max = a;
    const InstDev in = inst[i];
    c->t = 0.0;
    if (!(c->t < in.t_end)) {
        c->done = 1;
        return;
    }
    const double rate = a / in.dx;
    double dt = (rate > 0.0) ? in.cfl / rate : in.t_end - c->t;
    int last = 0;
    if (c->t + dt * (1.0 + 1e-10) >= in.t_end) {
        dt = in.t_end - c->t;
        last = 1;
    }
    c->dt = dt;
    c->last = last;
    c->step_cap = step_cap(in.t_end - c->t, dt, max_steps);
}

}  // namespace npw

namespace {

// ---------------------------------------------------------------------------------------
// The 1D runtime shared by rk3_step, solve and batch_solve.
// ---------------------------------------------------------------------------------------
struct Run1D {
    void* arena;
    int count;
    int m;
    int kind;
    npw::MethodParams mp;
    bool fp32;
    unsigned char* ws;
    Layout1D L;
    int64_t ntiles;
    cudaStream_t s;
    int tile = npw::TILE_1D;     // cells per CTA of the per-stage kernels
    bool comp = false;           // compensated float per-stage kernels (float, component-wise)
    std::vector<char> resident;  // per instance: solved by the resident kernel
    std::vector<cudaEvent_t> joins;  // side-stream work the caller's stream waits for at the end
};

// ---------------------------------------------------------------------------------------
// Tile sizes chosen by npw_autotune_1d, per device and (flux kind, m, k, precision,
// characteristic).  A run with params->tile_1d = 0 takes the chosen size, else the default.
// ---------------------------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::array<int, 6>, int> g_tune;

std::array<int, 6> tune_key(const npw_params* p, int kind, int m) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    return {dev, kind, m, p->k, p->precision, p->characteristic ? 1 : 0};
}

int resolve_tile(const npw_params* p, int kind, int m) {
    if (p->tile_1d > 0) return p->tile_1d;
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(tune_key(p, kind, m));
    return it == g_tune.end() ? npw::TILE_1D : it->second;
}

// the compensated float kernels (stage1d_fast_kernel, the resident kernel) cover float,
// component-wise (k = 3 and k = 2); FP64 and characteristic runs take the face-based stage kernel
bool compensated(const npw_params* p) {
    return p->precision == NPW_FP32_MIXED && !p->characteristic;
}

// instances the resident kernel can take: compensated float path, fits in shared memory
bool resident_ok(const npw_params* p, int m, int64_t n) {
    return compensated(p) && p->batch_mode == 0 && npw::resident_smem_bytes(n, m) <= npw::RESIDENT_SMEM_MAX;
}

int64_t tiles_for(const Run1D& r, const npw_instance* inst, int count) {
    int64_t nt = 0;
    for (int i = 0; i < count; ++i)
        if (r.resident.empty() || !r.resident[i]) nt += tiles_of(inst[i].n, r.tile);
    return nt;
}

template <typename R>
npw_status run_step_kernels(const Run1D& r, int advance) {
    if (r.ntiles == 0) return NPW_OK;
    npw::Stage1DArgs a{};
    a.inst = reinterpret_cast<const npw::InstDev*>(r.ws + r.L.inst);
    a.ctl = reinterpret_cast<npw::Ctl*>(r.ws + r.L.ctl);
    a.tiles = reinterpret_cast<const npw::Tile*>(r.ws + r.L.tiles);
    a.ntiles = (int)r.ntiles;
    a.advance = advance;
    a.tile = r.tile;
    a.mp = r.mp;
    void* u = r.arena;
    void* u1 = r.ws + r.L.u1;
    void* u2 = r.ws + r.L.u2;
    a.u = reinterpret_cast<float*>(u);
    a.d1 = reinterpret_cast<float*>(u1);
    a.d2 = reinterpret_cast<float*>(u2);
    a.s = reinterpret_cast<float*>(r.ws + r.L.sbuf);
    a.c = reinterpret_cast<float*>(r.ws + r.L.cbuf);
    // stage 1: u -> u1; stage 2: (u1, u) -> u2; stage 3: (u2, u) -> u (in place: each cell reads
    // its own u^n before writing it, and the halo of stage 3 comes from u2).  The compensated
    // float kernels use u, d1, d2, s and c instead (see stage1d_fast_kernel).
    const void* in_[3] = {u, u1, u2};
    void* out_[3] = {u1, u2, u};
    for (int st = 0; st < 3; ++st) {
        a.uin = in_[st];
        a.un = u;
        a.uout = out_[st];
        a.stage = st;
        auto ev = stage_begin(r.s);
        cudaError_t e = npw::launch_stage1d<R>(a, r.m, r.kind, r.s);
        stage_end(ev, r.s);
        if (e != cudaSuccess) return cuda_fail(e, "stage kernel launch");
    }
    return NPW_OK;
}

npw_status step_kernels(const Run1D& r, int advance) {
    return r.fp32 ? run_step_kernels<float>(r, advance) : run_step_kernels<double>(r, advance);
}

npw_status setup_1d(Run1D& r, const npw_instance* inst, int count, double dt_fixed, int mode) {
    std::vector<npw::InstDev> hi(count);
    std::vector<npw::Tile> ht;
    ht.reserve((size_t)r.ntiles);
    for (int i = 0; i < count; ++i) {
        hi[i].off = inst[i].offset;
        hi[i].n = inst[i].n;
        hi[i].dx = inst[i].dx;
        hi[i].t_end = inst[i].t_end;
        hi[i].cfl = inst[i].cfl;
        hi[i].bc = inst[i].bc;
        const bool res = !r.resident.empty() && r.resident[i];
        hi[i].ntiles = res ? 0 : (int32_t)tiles_of(inst[i].n, r.tile);
        for (int64_t t = 0; t < hi[i].ntiles; ++t) ht.push_back(npw::Tile{i, (int32_t)(t * r.tile)});
    }
    // pageable source: each call returns once the data is staged
    NPW_CUDA(cudaMemcpyAsync(r.ws + r.L.inst, hi.data(), sizeof(npw::InstDev) * count, cudaMemcpyHostToDevice, r.s));
    if (!ht.empty())
        NPW_CUDA(cudaMemcpyAsync(r.ws + r.L.tiles, ht.data(), sizeof(npw::Tile) * ht.size(), cudaMemcpyHostToDevice, r.s));
    npw::Ctl* ctl = reinterpret_cast<npw::Ctl*>(r.ws + r.L.ctl);
    const npw::InstDev* di = reinterpret_cast<const npw::InstDev*>(r.ws + r.L.inst);
    const unsigned blocks = (unsigned)((count + 127) / 128);
    npw::ctl_start_kernel<<<blocks, 128, 0, r.s>>>(ctl, di, count, 0, 0.0, 0);
    NPW_CUDA(cudaGetLastError());
    cudaError_t e = r.ntiles == 0 ? cudaSuccess
                  : r.fp32 ? npw::launch_alpha_init<float>(r.arena, di, ctl,
                                                           reinterpret_cast<const npw::Tile*>(r.ws + r.L.tiles),
                                                           (int)r.ntiles, r.tile, r.m, r.kind, r.mp, r.s)
                           : npw::launch_alpha_init<double>(r.arena, di, ctl,
                                                            reinterpret_cast<const npw::Tile*>(r.ws + r.L.tiles),
                                                            (int)r.ntiles, r.tile, r.m, r.kind, r.mp, r.s);
    if (e != cudaSuccess) return cuda_fail(e, "alpha kernel launch");
    npw::ctl_start_kernel<<<blocks, 128, 0, r.s>>>(ctl, di, count, mode, dt_fixed, r.mp.max_steps);
    NPW_CUDA(cudaGetLastError());
    count_launch(3);
    if (r.comp && r.ntiles > 0) {
        NPW_CUDA(npw::launch_comp_begin(reinterpret_cast<const float*>(r.arena), reinterpret_cast<float*>(r.ws + r.L.sbuf),
                                        reinterpret_cast<float*>(r.ws + r.L.cbuf), di,
                                        reinterpret_cast<const npw::Tile*>(r.ws + r.L.tiles), (int)r.ntiles, r.tile,
                                        r.m, r.s));
        count_launch();
    }
    return NPW_OK;
}

npw_status poll(const Run1D& r, long long* act, long long* rem, const npw::Inst2D* inst2d = nullptr) {
    long long* dpoll = reinterpret_cast<long long*>(r.ws + r.L.poll);
    npw::count_active_kernel<<<1, 256, 0, r.s>>>(reinterpret_cast<const npw::Ctl*>(r.ws + r.L.ctl),
                                                 inst2d ? nullptr : reinterpret_cast<const npw::InstDev*>(r.ws + r.L.inst),
                                                 r.count, inst2d, dpoll);
    NPW_CUDA(cudaGetLastError());
    count_launch();
    // wait (bounded) before the copy: a copy into pageable host memory returns only when the
    // stream has drained, so issued first it would be an unbounded wait
    npw_status st = bounded_sync(r.s);
    if (st) return st;
    long long h[2] = {0, 0};
    NPW_CUDA(cudaMemcpyAsync(h, dpoll, sizeof h, cudaMemcpyDeviceToHost, r.s));
    profile_collect();
    *act = h[0];
    *rem = h[1];
    return NPW_OK;
}

void fill_stats(const npw::Ctl& c, npw_solve_stats* o) {
    o->steps = c.steps;
    o->t = c.t;
    o->alpha_max = c.alpha_max;
    o->status = c.status;
    o->eta_switch = (int64_t)c.n_switch;
    o->eta_eval = (int64_t)c.n_eval;
    o->eta_guard = (int64_t)c.n_guard;
    o->eta_bound = (int64_t)c.n_bound;
}

npw_status collect_stats(const Run1D& r, npw_solve_stats* out) {
    std::vector<npw::Ctl> hc(r.count);
    npw_status st = bounded_sync(r.s);  // before the (blocking) copy into pageable memory
    if (st) return st;
    NPW_CUDA(cudaMemcpyAsync(hc.data(), r.ws + r.L.ctl, sizeof(npw::Ctl) * r.count, cudaMemcpyDeviceToHost, r.s));
    profile_collect();
    npw_status first = NPW_OK;
    for (int i = 0; i < r.count; ++i) {
        if (out) fill_stats(hc[i], &out[i]);
        if (hc[i].status != NPW_OK && first == NPW_OK) first = (npw_status)hc[i].status;
    }
    if (first == NPW_ENONFINITE) return fail(first, "an instance became non-finite");
    if (first != NPW_OK) return fail(first, "an instance reached its step limit or stopped advancing");
    return NPW_OK;
}

// Library-owned side streams (created once per device) for the resident launches.
struct SideStreams {
    cudaStream_t st[4];
    cudaEvent_t fork;
    bool ok = false;
};
std::mutex g_side_mu;
SideStreams g_side[64];

npw_status side_streams(SideStreams** out) {
    int dev = 0;
    NPW_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(NPW_ECUDA, "device index out of range");
    std::lock_guard<std::mutex> g(g_side_mu);
    SideStreams& s = g_side[dev];
    if (!s.ok) {
        for (int k = 0; k < 4; ++k) {
            NPW_CUDA(cudaStreamCreateWithFlags(&s.st[k], cudaStreamNonBlocking));
        }
        NPW_CUDA(cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming));
        s.ok = true;
    }
    *out = &s;
    return NPW_OK;
}

// Launch resident instances (all of one flux kind) in four size classes (largest first within
// a class), each on its own side stream after the set-up on the caller's stream.  ids: the
// instances (indices into inst / ctl), n_of / cost_of: their cells and expected work; dlist:
// device scratch for the index list.  The join events are appended to joins.
struct ResidentLaunch {
    void* arena;
    float* carry;
    const npw::InstDev* inst;
    npw::Ctl* ctl;
    int32_t* dlist;
    int m;
    int kind;
    npw::MethodParams mp;
};
npw_status launch_resident_set(const ResidentLaunch& rl, const std::vector<int32_t>& ids,
                               const std::vector<int64_t>& n_of, const std::vector<double>& cost_of,
                               SideStreams* ss, cudaStream_t s, std::vector<cudaEvent_t>& joins) {
    std::vector<int32_t> cls[4];
    for (int32_t i : ids) {
        const int64_t n = n_of[i];
        cls[n > 4096 ? 0 : (n > 2048 ? 1 : (n > 1024 ? 2 : 3))].push_back(i);
    }
    // two 512-thread CTAs per SM for the largest class (64 registers per thread fill the register
    // file either way) measured 10% faster than one 1024-thread CTA
    static const int threads[4] = {512, 512, 256, 128};
    std::vector<int32_t> all;
    size_t offs[5] = {0, 0, 0, 0, 0};
    for (int c = 0; c < 4; ++c) {
        auto& v = cls[c];
        std::sort(v.begin(), v.end(), [&](int a, int b) { return cost_of[a] > cost_of[b]; });  // longest first
        offs[c] = all.size();
        all.insert(all.end(), v.begin(), v.end());
    }
    offs[4] = all.size();
    if (all.empty()) return NPW_OK;
    NPW_CUDA(cudaMemcpyAsync(rl.dlist, all.data(), sizeof(int32_t) * all.size(), cudaMemcpyHostToDevice, s));
    NPW_CUDA(cudaEventRecord(ss->fork, s));
    for (int c = 0; c < 4; ++c) {
        const int cnt = (int)(offs[c + 1] - offs[c]);
        if (cnt == 0) continue;
        int64_t max_n = 0;
        for (size_t k = offs[c]; k < offs[c + 1]; ++k) max_n = n_of[all[k]] > max_n ? n_of[all[k]] : max_n;
        NPW_CUDA(cudaStreamWaitEvent(ss->st[c], ss->fork, 0));
        npw::ResidentArgs a{};
        a.arena = rl.arena;
        a.carry = rl.carry;
        a.inst = rl.inst;
        a.ctl = rl.ctl;
        a.list = rl.dlist + offs[c];
        a.count = cnt;
        a.mp = rl.mp;
        auto ev = stage_begin(ss->st[c], c);
        cudaError_t e = npw::launch_resident_f32(a, rl.m, rl.kind, max_n, threads[c], ss->st[c]);
        stage_end(ev, ss->st[c], c);
        if (e != cudaSuccess) return cuda_fail(e, "resident kernel launch");
        // one event per launch: a later launch set on the same side stream records its own
        cudaEvent_t je = nullptr;
        NPW_CUDA(cudaEventCreateWithFlags(&je, cudaEventDisableTiming));
        NPW_CUDA(cudaEventRecord(je, ss->st[c]));
        joins.push_back(je);
    }
    return NPW_OK;
}

// the 1D batch runtime's resident instances (one flux kind)
npw_status launch_resident(Run1D& r, const npw_instance* inst, SideStreams* ss, int* joined) {
    std::vector<int32_t> ids;
    std::vector<int64_t> n_of(r.count);
    std::vector<double> cost(r.count);
    for (int i = 0; i < r.count; ++i) {
        n_of[i] = inst[i].n;
        cost[i] = (double)inst[i].n * inst[i].t_end / (inst[i].cfl * inst[i].dx);  // ~ n * steps
        if (r.resident[i]) ids.push_back(i);
    }
    ResidentLaunch rl{r.arena, reinterpret_cast<float*>(r.ws + r.L.cbuf), reinterpret_cast<const npw::InstDev*>(r.ws + r.L.inst),
                      reinterpret_cast<npw::Ctl*>(r.ws + r.L.ctl), reinterpret_cast<int32_t*>(r.ws + r.L.list), r.m,
                      r.kind, r.mp};
    const size_t before = r.joins.size();
    npw_status st = launch_resident_set(rl, ids, n_of, cost, ss, r.s, r.joins);
    *joined = (int)(r.joins.size() - before);
    return st;
}

// compensated float path: the final states are in s; copy them back into the arena
npw_status comp_end(const Run1D& r) {
    if (!r.comp || r.ntiles == 0) return NPW_OK;
    NPW_CUDA(npw::launch_comp_end(reinterpret_cast<float*>(r.arena), reinterpret_cast<const float*>(r.ws + r.L.sbuf),
                                  reinterpret_cast<const npw::InstDev*>(r.ws + r.L.inst),
                                  reinterpret_cast<const npw::Tile*>(r.ws + r.L.tiles), (int)r.ntiles, r.tile, r.m,
                                  nullptr, r.s));
    count_launch();
    return NPW_OK;
}

// Run steps until every instance is done: launch as many steps as the largest remaining
// estimate (capped), then poll.
// ---------------------------------------------------------------------------------------
// CUDA graph of GRAPH_STEPS whole steps (3 stage launches each) for the per-stage path.  The
// stage kernels read t, dt, alpha and the done flag of every instance from its control word,
// so one captured launch sequence serves every replay, and steps past an instance's end time
// are no-ops for it (its CTAs return at once).  Capture uses a private stream; the graph is
// launched on the caller's stream.
// ---------------------------------------------------------------------------------------
constexpr int GRAPH_STEPS = 8;

struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    StepGraph() = default;
    StepGraph(const StepGraph&) = delete;
    StepGraph& operator=(const StepGraph&) = delete;
    ~StepGraph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
    // after a wait ran out the graph may still have launches queued: it is not destroyed
    // (a small leak on that error path instead of destroying a graph that is in use)
    void abandon() { exec = nullptr; }
};

npw_status capture_steps(const Run1D& r, StepGraph& g) {
    cudaStream_t cs = nullptr;
    NPW_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    Run1D rc = r;
    rc.s = cs;
    cudaGraph_t graph = nullptr;
    npw_status st = NPW_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        t_capturing = true;
        for (int k = 0; k < GRAPH_STEPS && st == NPW_OK; ++k) st = step_kernels(rc, 1);
        t_capturing = false;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e2 != cudaSuccess) e = e2;
    }
    if (st == NPW_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st) return st;
    if (e != cudaSuccess) {
        g.exec = nullptr;
        return cuda_fail(e, "capture of the step graph");
    }
    return NPW_OK;
}

npw_status replay_steps(const Run1D& r, const StepGraph& g, long long graphs) {
    for (long long k = 0; k < graphs; ++k) {
        auto ev = stage_begin(r.s, -1, 3 * GRAPH_STEPS);
        const cudaError_t e = cudaGraphLaunch(g.exec, r.s);
        stage_end(ev, r.s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    }
    return NPW_OK;
}

npw_status run_to_end(Run1D& r, npw_solve_stats* out) {
    long long act = 0, rem = 0;
    npw_status st = poll(r, &act, &rem);
    StepGraph graph;
    bool direct_done = false;
    while (st == NPW_OK && act > 0) {
        long long chunk = rem < 1 ? 1 : (rem > 256 ? 256 : rem);
        // long chunks replay the captured graph (after one direct step has set up the kernels'
        // attributes); the remainder, and short runs, launch directly
        if (chunk > GRAPH_STEPS && direct_done) {
            if (!graph.exec && (st = capture_steps(r, graph))) break;
            if ((st = replay_steps(r, graph, chunk / GRAPH_STEPS))) break;
            chunk %= GRAPH_STEPS;
        }
        for (long long k = 0; k < chunk && st == NPW_OK; ++k) st = step_kernels(r, 1);
        direct_done = true;
        if (st == NPW_OK) st = poll(r, &act, &rem);
    }
    if (st == NPW_ETIMEOUT) graph.abandon();
    if (st == NPW_OK) st = comp_end(r);
    for (cudaEvent_t ev : r.joins) {  // resident kernels on the side streams
        cudaError_t e = cudaStreamWaitEvent(r.s, ev, 0);
        if (e != cudaSuccess && st == NPW_OK) st = cuda_fail(e, "cudaStreamWaitEvent");
        cudaEventDestroy(ev);  // released once the recorded work completes
    }
    r.joins.clear();
    if (st) return st;
    return collect_stats(r, out);
}

}  // namespace

npw_status npw::set_error(npw_status st, const char* msg) { return fail(st, "%s", msg); }

// =======================================================================================
// C ABI
// =======================================================================================
extern "C" {

void npw_default_params(npw_params* p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->k = 3;
    p->scheme = NPW_RBF_WENO;
    p->rbf = NPW_RBF_MQ;
    p->monotone_switch = 1;
    p->switch_variant = 0;
    p->characteristic = 0;
    p->precision = NPW_FP64;
    p->eps_M = 1e-12;
    p->eps_weno = 1e-6;
    p->gamma = 1.4;
    p->adv_speed = 1.0;
    p->adv_speed_y = 1.0;
    p->bc_y = -1;
}

const char* npw_last_error(void) { return g_err.c_str(); }

void npw_profile_enable(int32_t on) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.on = on != 0;
}

void npw_profile_reset(void) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.launches = p.stage_launches = p.timed = 0;
    p.stage_ms = 0.0;
    for (int c = 0; c < 4; ++c) {
        p.res_launches[c] = 0;
        p.res_ms[c] = 0.0;
    }
    for (auto& item : p.pending) p.pool.push_back(item.first);
    p.pending.clear();
}

void npw_profile_read(npw_profile* out) {
    if (!out) return;
    profile_collect();
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    out->kernel_launches = p.launches;
    out->stage_launches = p.stage_launches;
    out->stage_ms = p.stage_ms;
    out->timed_launches = p.timed;
    for (int c = 0; c < 4; ++c) {
        out->resident_launches[c] = p.res_launches[c];
        out->resident_ms[c] = p.res_ms[c];
    }
}

int32_t npw_version(void) { return 10200; }

npw_status npweno_reconstruct(const void* vbar, int64_t n, int32_t m, int32_t bc, const npw_params* params,
                              void* v_minus, void* v_plus, uint8_t* flags, void* eta, void* stream) {
    npw_status st = check_params(params);
    if (st) return st;
    if (!vbar || !v_minus || !v_plus) return fail(NPW_EINVAL, "null array pointer");
    if (n < 6) return fail(NPW_EINVAL, "n = %lld < 6", (long long)n);
    if (m < 1 || m > 4 || m == 2) return fail(NPW_EINVAL, "m = %d not supported", m);
    if (params->characteristic && m != 3) return fail(NPW_EINVAL, "characteristic reconstruction needs m = 3");
    if ((st = check_bc(bc))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    npw::MethodParams mp = method(params);
    cudaError_t e = params->precision == NPW_FP32_MIXED
                        ? npw::launch_reconstruct<float>((const float*)vbar, n, m, bc, mp, (float*)v_minus,
                                                         (float*)v_plus, flags, (float*)eta, s)
                        : npw::launch_reconstruct<double>((const double*)vbar, n, m, bc, mp, (double*)v_minus,
                                                          (double*)v_plus, flags, (double*)eta, s);
    if (e != cudaSuccess) return cuda_fail(e, "reconstruct launch");
    count_launch();
    return NPW_OK;
}

npw_status npweno_flux(const void* v_minus, const void* v_plus, int64_t nfaces, int32_t m, int32_t flux_kind,
                       double alpha, const npw_params* params, void* h, void* stream) {
    npw_status st = check_params(params);
    if (st) return st;
    if (!v_minus || !v_plus || !h) return fail(NPW_EINVAL, "null array pointer");
    if (nfaces < 1) return fail(NPW_EINVAL, "nfaces < 1");
    if (flux_kind == NPW_FLUX_EULER2D || flux_kind < 0 || flux_kind > NPW_FLUX_EULER2D)
        return fail(NPW_EINVAL, "flux kind %d not supported here", flux_kind);
    if (m != flux_m(flux_kind)) return fail(NPW_EINVAL, "m = %d does not match flux kind", m);
    if (!(alpha >= 0.0)) return fail(NPW_EINVAL, "alpha must be >= 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    npw::MethodParams mp = method(params);
    cudaError_t e = params->precision == NPW_FP32_MIXED
                        ? npw::launch_flux<float>((const float*)v_minus, (const float*)v_plus, nfaces, m, flux_kind,
                                                  alpha, mp, (float*)h, s)
                        : npw::launch_flux<double>((const double*)v_minus, (const double*)v_plus, nfaces, m,
                                                   flux_kind, alpha, mp, (double*)h, s);
    if (e != cudaSuccess) return cuda_fail(e, "flux launch");
    count_launch();
    return NPW_OK;
}

size_t npw_workspace_size(int64_t n, int32_t m, const npw_params* params) {
    if (!params || n < 1 || m < 1) return 0;
    return layout_1d(n * m, 1, tiles_of(n), elem_size(params)).total;
}

static npw_status single_run(void* u, int64_t n, int32_t m, double dx, double t_end, double cfl, int32_t flux_kind,
                             int32_t bc, const npw_params* params, void* workspace, size_t workspace_bytes,
                             cudaStream_t s, Run1D& r, npw_instance& in) {
    npw_status st = check_params(params);
    if (st) return st;
    if (!u || !workspace) return fail(NPW_EINVAL, "null pointer");
    if (n < 6) return fail(NPW_EINVAL, "n = %lld < 6", (long long)n);
    if (n > (int64_t)1 << 30) return fail(NPW_EINVAL, "n too large");
    if ((st = check_kind_1d(flux_kind, m, params))) return st;
    if ((st = check_bc(bc))) return st;
    if (!(dx > 0.0)) return fail(NPW_EINVAL, "dx must be > 0");
    r.arena = u;
    r.count = 1;
    r.m = m;
    r.kind = flux_kind;
    r.mp = method(params);
    r.fp32 = params->precision == NPW_FP32_MIXED;
    r.ws = static_cast<unsigned char*>(workspace);
    r.tile = resolve_tile(params, flux_kind, m);
    r.ntiles = tiles_of(n, r.tile);
    r.L = layout_1d(n * m, 1, tiles_of(n), elem_size(params));
    r.s = s;
    r.comp = compensated(params);
    if (workspace_bytes < r.L.total)
        return fail(NPW_EINVAL, "workspace too small: %zu < %zu bytes", workspace_bytes, r.L.total);
    in.offset = 0;
    in.n = n;
    in.dx = dx;
    in.t_end = t_end;
    in.cfl = cfl;
    in.bc = bc;
    return NPW_OK;
}

npw_status npweno_rk3_step(void* u, int64_t n, int32_t m, double dx, double dt, int32_t flux_kind, int32_t bc,
                           const npw_params* params, void* workspace, size_t workspace_bytes, double* alpha_out,
                           void* stream) {
    Run1D r{};
    npw_instance in{};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    npw_status st = single_run(u, n, m, dx, 0.0, 0.0, flux_kind, bc, params, workspace, workspace_bytes, s, r, in);
    if (st) return st;
    if (!(dt >= 0.0)) return fail(NPW_EINVAL, "dt must be >= 0");
    if ((st = setup_1d(r, &in, 1, dt, 2))) return st;
    if ((st = step_kernels(r, 0))) return st;
    if ((st = comp_end(r))) return st;
    if (alpha_out) {
        npw::Ctl c;
        if ((st = bounded_sync(s))) return st;
        NPW_CUDA(cudaMemcpyAsync(&c, r.ws + r.L.ctl, sizeof c, cudaMemcpyDeviceToHost, s));
        *alpha_out = c.alpha;
        if (c.status) return fail((npw_status)c.status, "state is not finite");
    }
    return NPW_OK;
}

npw_status npweno_solve(void* u, int64_t n, int32_t m, double dx, double t_end, double cfl, int32_t flux_kind,
                        int32_t bc, const npw_params* params, void* workspace, size_t workspace_bytes,
                        npw_solve_stats* out, void* stream) {
    Run1D r{};
    npw_instance in{};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    npw_status st = single_run(u, n, m, dx, t_end, cfl, flux_kind, bc, params, workspace, workspace_bytes, s, r, in);
    if (st) return st;
    if (!(cfl > 0.0)) return fail(NPW_EINVAL, "cfl must be > 0");
    if ((st = setup_1d(r, &in, 1, 0.0, 1))) return st;
    return run_to_end(r, out);
}

size_t npw_batch_workspace_size(const npw_instance* inst, int32_t count, int32_t m, const npw_params* params) {
    if (!inst || count < 1 || !params || m < 1) return 0;
    int64_t arena = 0, nt = 0;
    for (int i = 0; i < count; ++i) {
        int64_t end = inst[i].offset + inst[i].n * m;
        arena = end > arena ? end : arena;
        nt += tiles_of(inst[i].n);
    }
    return layout_1d(arena, count, nt, elem_size(params)).total;
}

npw_status npweno_batch_solve(void* arena, const npw_instance* inst, int32_t count, int32_t m, int32_t flux_kind,
                              const npw_params* params, void* workspace, size_t workspace_bytes,
                              npw_solve_stats* out, void* stream) {
    npw_status st = check_params(params);
    if (st) return st;
    if (!arena || !inst || !workspace || count < 1) return fail(NPW_EINVAL, "null pointer or empty batch");
    if ((st = check_kind_1d(flux_kind, m, params))) return st;
    int64_t arena_elems = 0, nt = 0;
    for (int i = 0; i < count; ++i) {
        if (inst[i].n < 6 || inst[i].n > ((int64_t)1 << 30)) return fail(NPW_EINVAL, "instance %d: bad n", i);
        if (!(inst[i].dx > 0.0) || !(inst[i].cfl > 0.0)) return fail(NPW_EINVAL, "instance %d: bad dx or cfl", i);
        if (inst[i].offset < 0) return fail(NPW_EINVAL, "instance %d: negative offset", i);
        if ((st = check_bc(inst[i].bc))) return st;
        int64_t end = inst[i].offset + inst[i].n * m;
        arena_elems = end > arena_elems ? end : arena_elems;
        nt += tiles_of(inst[i].n);
    }
    if (nt > (int64_t)1 << 30) return fail(NPW_EINVAL, "too many tiles");
    Run1D r{};
    r.arena = arena;
    r.count = count;
    r.m = m;
    r.kind = flux_kind;
    r.mp = method(params);
    r.fp32 = params->precision == NPW_FP32_MIXED;
    r.ws = static_cast<unsigned char*>(workspace);
    r.L = layout_1d(arena_elems, count, nt, elem_size(params));
    r.s = reinterpret_cast<cudaStream_t>(stream);
    if (workspace_bytes < r.L.total)
        return fail(NPW_EINVAL, "workspace too small: %zu < %zu bytes", workspace_bytes, r.L.total);
    r.comp = compensated(params);
    r.tile = resolve_tile(params, flux_kind, m);
    r.resident.assign(count, 0);
    bool any_res = false;
    for (int i = 0; i < count; ++i) {
        r.resident[i] = resident_ok(params, m, inst[i].n) ? 1 : 0;
        any_res |= r.resident[i] != 0;
    }
    r.ntiles = tiles_for(r, inst, count);
    if ((st = setup_1d(r, inst, count, 0.0, 1))) return st;
    if (any_res) {
        SideStreams* ss = nullptr;
        int joined = 0;
        if ((st = side_streams(&ss))) return st;
        if ((st = launch_resident(r, inst, ss, &joined))) return st;
    }
    return run_to_end(r, out);
}

// ---------------------------------------------------------------------------------------
// Tile autotuner
// ---------------------------------------------------------------------------------------
static const int64_t kTuneCells = (int64_t)1 << 21;

size_t npw_autotune_scratch_bytes(int32_t m, const npw_params* params) {
    if (!params || m < 1 || m > 3) return 0;
    return align256((size_t)(kTuneCells * m) * elem_size(params)) + npw_workspace_size(kTuneCells, m, params);
}

npw_status npw_autotune_1d(int32_t flux_kind, int32_t m, const npw_params* params, void* scratch,
                           size_t scratch_bytes, void* stream, int32_t* best_tile) {
    npw_status st = check_params(params);
    if (st) return st;
    if (!scratch || !best_tile) return fail(NPW_EINVAL, "null pointer");
    if ((st = check_kind_1d(flux_kind, m, params))) return st;
    const size_t need = npw_autotune_scratch_bytes(m, params);
    if (scratch_bytes < need) return fail(NPW_EINVAL, "autotune scratch too small: %zu < %zu bytes", scratch_bytes, need);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(scratch);
    const size_t arena_b = align256((size_t)(kTuneCells * m) * elem_size(params));
    void* u = base;
    void* ws = base + arena_b;
    const size_t ws_b = scratch_bytes - arena_b;
    const bool fp32 = params->precision == NPW_FP32_MIXED;
    const double dx = 1.0 / (double)kTuneCells, dt = 0.1 * dx;
    static const int kTiles[4] = {256, 512, 1024, 2048};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NPW_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(NPW_ECUDA, "cudaEventCreate");
    }
    int best = 0;
    float best_ms = 0.0f;
    for (int c = 0; c < 4 && st == NPW_OK; ++c) {
        npw_params q = *params;
        q.tile_1d = kTiles[c];
        cudaError_t e = fp32 ? npw::launch_tune_init<float>(static_cast<float*>(u), kTuneCells, m, s)
                             : npw::launch_tune_init<double>(static_cast<double*>(u), kTuneCells, m, s);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "autotune init");
            break;
        }
        for (int w = 0; w < 2 && st == NPW_OK; ++w)
            st = npweno_rk3_step(u, kTuneCells, m, dx, dt, flux_kind, NPW_BC_PERIODIC, &q, ws, ws_b, nullptr, stream);
        if (st) break;
        cudaEventRecord(e0, s);
        for (int k = 0; k < 4 && st == NPW_OK; ++k)
            st = npweno_rk3_step(u, kTuneCells, m, dx, dt, flux_kind, NPW_BC_PERIODIC, &q, ws, ws_b, nullptr, stream);
        cudaEventRecord(e1, s);
        if (st || (st = bounded_sync(s))) break;
        float ms = 0.0f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
            st = cuda_fail(e, "cudaEventElapsedTime");
            break;
        }
        if (best == 0 || ms < best_ms) {
            best = kTiles[c];
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune[tune_key(params, flux_kind, m)] = best;
    }
    *best_tile = best;
    return NPW_OK;
}

// ---------------------------------------------------------------------------------------
// 2D
// ---------------------------------------------------------------------------------------
size_t npw_workspace_size_2d(int64_t nx, int64_t ny, int32_t m, const npw_params* params) {
    if (!params || nx < 1 || ny < 1 || m < 1) return 0;
    size_t esz = elem_size(params);
    size_t o = 0;
    o = align256(o + (size_t)(nx * ny * m) * esz);
    o = align256(o + (size_t)(nx * ny * m) * esz);
    o = align256(o + sizeof(npw::Inst2D));
    o = align256(o + sizeof(npw::Ctl));
    o = align256(o + 4 * sizeof(long long));
    return o;
}

static npw_status run_2d(void* u, int64_t nx, int64_t ny, int32_t m, double dx, double dy, double dt_fixed,
                         double t_end, double cfl, int32_t flux_kind, int32_t bc, const npw_params* params,
                         void* workspace, size_t workspace_bytes, npw_solve_stats* out, cudaStream_t s, int mode) {
    npw_status st = check_params(params);
    if (st) return st;
    if (!u || !workspace) return fail(NPW_EINVAL, "null pointer");
    if (nx < 6 || ny < 6) return fail(NPW_EINVAL, "nx, ny must be >= 6");
    if (nx * ny > ((int64_t)1 << 31)) return fail(NPW_EINVAL, "grid too large");
    if (flux_kind != NPW_FLUX_ADVECTION && flux_kind != NPW_FLUX_BURGERS && flux_kind != NPW_FLUX_EULER2D)
        return fail(NPW_EINVAL, "flux kind %d is not a 2D flux", flux_kind);
    if (m != flux_m(flux_kind)) return fail(NPW_EINVAL, "m does not match the flux kind");
    if (params->characteristic) return fail(NPW_EINVAL, "2D runs are component-wise");
    if ((st = check_gauss(params))) return st;
    if ((st = check_bc(bc))) return st;
    if (params->bc_y >= 0 && (st = check_bc(params->bc_y))) return st;
    if (!(dx > 0.0) || !(dy > 0.0)) return fail(NPW_EINVAL, "dx, dy must be > 0");
    const bool fp32 = params->precision == NPW_FP32_MIXED;
    const size_t esz = elem_size(params);
    if (workspace_bytes < npw_workspace_size_2d(nx, ny, m, params)) return fail(NPW_EINVAL, "workspace too small");
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    size_t o = 0;
    void* u1 = ws + o;
    o = align256(o + (size_t)(nx * ny * m) * esz);
    void* u2 = ws + o;
    o = align256(o + (size_t)(nx * ny * m) * esz);
    npw::Inst2D* dinst = reinterpret_cast<npw::Inst2D*>(ws + o);
    o = align256(o + sizeof(npw::Inst2D));
    npw::Ctl* ctl = reinterpret_cast<npw::Ctl*>(ws + o);
    o = align256(o + sizeof(npw::Ctl));
    long long* dpoll = reinterpret_cast<long long*>(ws + o);

    npw::Inst2D hi{};
    hi.off = 0;
    hi.nx = nx;
    hi.ny = ny;
    hi.dx = dx;
    hi.dy = dy;
    hi.t_end = t_end;
    hi.cfl = cfl;
    hi.bc = bc;
    hi.bc_y = params->bc_y < 0 ? bc : params->bc_y;
    hi.tiles_x = (int32_t)((nx + npw::TX_2D - 1) / npw::TX_2D);
    hi.tiles_y = (int32_t)((ny + npw::TY_2D - 1) / npw::TY_2D);
    const int tiles = hi.tiles_x * hi.tiles_y;
    NPW_CUDA(cudaMemcpyAsync(dinst, &hi, sizeof hi, cudaMemcpyHostToDevice, s));
    npw::MethodParams mp = method(params);
    npw::ctl_start_2d_kernel<<<1, 32, 0, s>>>(ctl, dinst, 0, 0.0, 0);
    NPW_CUDA(cudaGetLastError());
    cudaError_t e = fp32 ? npw::launch_alpha_init_2d<float>(u, dinst, tiles, ctl, flux_kind, mp, s)
                         : npw::launch_alpha_init_2d<double>(u, dinst, tiles, ctl, flux_kind, mp, s);
    if (e != cudaSuccess) return cuda_fail(e, "alpha 2d launch");
    npw::ctl_start_2d_kernel<<<1, 32, 0, s>>>(ctl, dinst, mode, dt_fixed, mp.max_steps);
    NPW_CUDA(cudaGetLastError());
    count_launch(3);

    npw::Stage2DArgs a{};
    a.inst = dinst;
    a.ctl = ctl;
    a.mp = mp;
    a.advance = mode == 1;
    const void* in_[3] = {u, u1, u2};
    void* out_[3] = {u1, u2, u};
    auto one_step = [&]() -> npw_status {
        for (int stg = 0; stg < 3; ++stg) {
            a.uin = in_[stg];
            a.un = u;
            a.uout = out_[stg];
            a.stage = stg;
            auto ev = stage_begin(s);
            cudaError_t ee = fp32 ? npw::launch_stage2d<float>(a, tiles, flux_kind, s)
                                  : npw::launch_stage2d<double>(a, tiles, flux_kind, s);
            stage_end(ev, s);
            if (ee != cudaSuccess) return cuda_fail(ee, "stage 2d launch");
        }
        return NPW_OK;
    };
    if (mode == 2) return one_step();
    Run1D pr{};
    pr.ws = ws;
    pr.count = 1;
    pr.s = s;
    pr.L.ctl = (size_t)((unsigned char*)ctl - ws);
    pr.L.poll = (size_t)((unsigned char*)dpoll - ws);
    long long act = 0, rem = 0;
    st = poll(pr, &act, &rem, dinst);
    while (st == NPW_OK && act > 0) {
        long long chunk = rem < 1 ? 1 : (rem > 256 ? 256 : rem);
        for (long long k = 0; k < chunk && st == NPW_OK; ++k) st = one_step();
        if (st == NPW_OK) st = poll(pr, &act, &rem, dinst);
    }
    if (st) return st;
    npw::Ctl hc;
    if ((st = bounded_sync(s))) return st;
    NPW_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost, s));
    if (out) fill_stats(hc, out);
    if (hc.status) return fail((npw_status)hc.status, "state is not finite");
    return NPW_OK;
}

npw_status npweno_rk3_step_2d(void* u, int64_t nx, int64_t ny, int32_t m, double dx, double dy, double dt,
                              int32_t flux_kind, int32_t bc, const npw_params* params, void* workspace,
                              size_t workspace_bytes, void* stream) {
    if (!(dt >= 0.0)) return fail(NPW_EINVAL, "dt must be >= 0");
    return run_2d(u, nx, ny, m, dx, dy, dt, 0.0, 0.0, flux_kind, bc, params, workspace, workspace_bytes, nullptr,
                  reinterpret_cast<cudaStream_t>(stream), 2);
}

npw_status npweno_solve_2d(void* u, int64_t nx, int64_t ny, int32_t m, double dx, double dy, double t_end,
                           double cfl, int32_t flux_kind, int32_t bc, const npw_params* params, void* workspace,
                           size_t workspace_bytes, npw_solve_stats* out, void* stream) {
    if (!(cfl > 0.0)) return fail(NPW_EINVAL, "cfl must be > 0");
    return run_2d(u, nx, ny, m, dx, dy, 0.0, t_end, cfl, flux_kind, bc, params, workspace, workspace_bytes, out,
                  reinterpret_cast<cudaStream_t>(stream), 1);
}

}  // extern "C"

// =======================================================================================
// Work-queue runtime: 1D and 2D instances of any flux kind in one batch, every stage one
// launch of the persistent queue kernel over all (instance, tile) items; mixed-precision 1D
// instances that fit in shared memory run whole in the resident kernel beside it.
// =======================================================================================
namespace npw {

// mode 0: zero the control words; mode 1: start (alpha^0 from the running maxima, first dt,
// step limit).  1D instances without items (solved by the resident kernel) are marked done.
// list (may be NULL): the instances to start, else 0..count-1
__global__ void queue_ctl_kernel(Ctl* ctl, const InstDev* inst1, const Inst2D* inst2, const uint8_t* is2d,
                                 const int32_t* list, int count, int mode, int64_t max_steps) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const int i = list ? list[j] : j;
    Ctl* c = ctl + i;
    if (mode == 0) {
        memset(c, 0, sizeof(Ctl));
        return;
    }
    const bool two_d = is2d[i] != 0;
    const double ax = __longlong_as_double((long long)c->alpha_next_bits);
    const double ay = two_d ? __longlong_as_double((long long)c->alpha_y_next_bits) : 0.0;
    c->alpha_next_bits = 0ull;
    c->alpha_y_next_bits = 0ull;
    c->tiles_done = 0u;
    if (!(ax - ax == 0.0) || !(ay - ay == 0.0)) {
        c->status = NPW_ENONFINITE;
        c->done = 1;
        return;
    }
    c->alpha = ax;
    c->alpha_y = ay;
    c->alpha_max = ax > ay ? ax : ay;
    c->t = 0.0;
    double t_end, cfl, rate;
    if (two_d) {
        const Inst2D& in = inst2[i];
        t_end = in.t_end;
        cfl = in.cfl;
        rate = ax / in.dx + ay / in.dy;
    } else {
        const InstDev& in = inst1[i];
        if (in.ntiles == 0) {  // resident instance: its kernel owns the control word
            c->done = 1;
            return;
        }
        t_end = in.t_end;
        cfl = in.cfl;
        rate = ax / in.dx;
    }
    if (!(c->t < t_end)) {
        c->done = 1;
        return;
    }
    double dt = (rate > 0.0) ? cfl / rate : t_end - c->t;
    int last = 0;
    if (c->t + dt * (1.0 + 1e-10) >= t_end) {
        dt = t_end - c->t;
        last = 1;
    }
    c->dt = dt;
    c->last = last;
    c->step_cap = step_cap(t_end - c->t, dt, max_steps);
}

// poll[0] = active instances, poll[1] = largest remaining step estimate
__global__ void queue_poll_kernel(const Ctl* ctl, const InstDev* inst1, const Inst2D* inst2, const uint8_t* is2d,
                                  int count, long long* poll) {
    __shared__ long long s_act[256], s_rem[256];
    long long act = 0, rem = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const Ctl& c = ctl[i];
        if (!c.done) {
            ++act;
            const double t_end = is2d[i] ? inst2[i].t_end : inst1[i].t_end;
            const double r = (c.dt > 0.0) ? (t_end - c.t) / c.dt : 1.0;
            const long long ri = (long long)(r < 1e9 ? r : 1e9) + 1;
            rem = ri > rem ? ri : rem;
        }
    }
    s_act[threadIdx.x] = act;
    s_rem[threadIdx.x] = rem;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_act[threadIdx.x] += s_act[threadIdx.x + o];
            s_rem[threadIdx.x] = s_rem[threadIdx.x + o] > s_rem[threadIdx.x] ? s_rem[threadIdx.x + o] : s_rem[threadIdx.x];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        poll[0] = s_act[0];
        poll[1] = s_rem[0];
    }
}

cudaError_t launch_queue_ctl(Ctl* ctl, const InstDev* inst1, const Inst2D* inst2, const uint8_t* is2d,
                             const int32_t* list, int count, int mode, int64_t max_steps, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    queue_ctl_kernel<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(ctl, inst1, inst2, is2d, list, count, mode,
                                                                     max_steps);
    return cudaGetLastError();
}
cudaError_t launch_queue_poll(const Ctl* ctl, const InstDev* inst1, const Inst2D* inst2, const uint8_t* is2d,
                              int count, long long* poll, cudaStream_t s) {
    queue_poll_kernel<<<1, 256, 0, s>>>(ctl, inst1, inst2, is2d, count, poll);
    return cudaGetLastError();
}

}  // namespace npw

namespace {

struct QLayout {
    size_t u1, u2, sbuf, cbuf, inst1, inst2, kind, is2d, ctl, items, head, poll, list, total;
};

QLayout queue_layout(int64_t arena_elems, int count, int64_t nitems, size_t esz, bool comp) {
    QLayout L{};
    size_t o = 0;
    L.u1 = o;
    o = align256(o + (size_t)arena_elems * esz);
    L.u2 = o;
    o = align256(o + (size_t)arena_elems * esz);
    L.sbuf = o;  // compensated float 1D: next state and carry
    o = align256(o + (comp ? (size_t)arena_elems * sizeof(float) : 0));
    L.cbuf = o;
    o = align256(o + (comp ? (size_t)arena_elems * sizeof(float) : 0));
    L.inst1 = o;
    o = align256(o + sizeof(npw::InstDev) * (size_t)count);
    L.inst2 = o;
    o = align256(o + sizeof(npw::Inst2D) * (size_t)count);
    L.kind = o;
    o = align256(o + sizeof(int32_t) * (size_t)count);
    L.is2d = o;
    o = align256(o + (size_t)count);
    L.ctl = o;
    o = align256(o + sizeof(npw::Ctl) * (size_t)count);
    L.items = o;
    o = align256(o + sizeof(npw::Tile) * (size_t)nitems);
    L.head = o;
    o = align256(o + 2 * sizeof(unsigned int));
    L.poll = o;
    o = align256(o + 4 * sizeof(long long));
    L.list = o;
    o = align256(o + sizeof(int32_t) * (size_t)count);
    L.total = o;
    return L;
}

bool is_2d_kind(const npw_queue_instance& q) { return q.ny != 0; }
int64_t items_of(const npw_queue_instance& q, int tile) {
    if (is_2d_kind(q)) return ((q.nx + npw::TX_2D - 1) / npw::TX_2D) * ((q.ny + npw::TY_2D - 1) / npw::TY_2D);
    return (q.nx + tile - 1) / tile;
}
int64_t cells_of(const npw_queue_instance& q) { return q.nx * (q.ny ? q.ny : 1) * flux_m(q.flux_kind); }

npw_status check_queue(const npw_queue_instance* inst, int count, const npw_params* p, int64_t* arena_elems,
                       int64_t* items_bound) {
    if (!inst || count < 1) return fail(NPW_EINVAL, "null or empty instance list");
    int64_t arena = 0, items = 0;
    for (int i = 0; i < count; ++i) {
        const npw_queue_instance& q = inst[i];
        npw_status st;
        if (q.ny == 0) {
            if (q.flux_kind != NPW_FLUX_ADVECTION && q.flux_kind != NPW_FLUX_BURGERS && q.flux_kind != NPW_FLUX_EULER1D)
                return fail(NPW_EINVAL, "instance %d: flux kind %d is not a 1D flux", i, q.flux_kind);
            if (p->characteristic && q.flux_kind != NPW_FLUX_EULER1D)
                return fail(NPW_EINVAL, "instance %d: characteristic reconstruction needs the 1D Euler flux", i);
            if (q.nx < 6 || q.nx > ((int64_t)1 << 30)) return fail(NPW_EINVAL, "instance %d: bad n", i);
        } else {
            if (q.flux_kind != NPW_FLUX_ADVECTION && q.flux_kind != NPW_FLUX_BURGERS && q.flux_kind != NPW_FLUX_EULER2D)
                return fail(NPW_EINVAL, "instance %d: flux kind %d is not a 2D flux", i, q.flux_kind);
            if (q.nx < 6 || q.ny < 6 || q.nx * q.ny > ((int64_t)1 << 31) || !(q.dy > 0.0))
                return fail(NPW_EINVAL, "instance %d: bad 2D size or dy", i);
            if (q.bc_y >= 0 && (st = check_bc(q.bc_y))) return st;
            if ((st = check_gauss(p, true))) return st;
        }
        if ((st = check_bc(q.bc))) return st;
        if (!(q.dx > 0.0) || !(q.cfl > 0.0)) return fail(NPW_EINVAL, "instance %d: bad dx or cfl", i);
        if (q.offset < 0) return fail(NPW_EINVAL, "instance %d: negative offset", i);
        const int64_t end = q.offset + cells_of(q);
        arena = end > arena ? end : arena;
        items += items_of(q, npw::TILE_1D_MIN);
    }
    if (items > ((int64_t)1 << 30)) return fail(NPW_EINVAL, "too many work items");
    *arena_elems = arena;
    *items_bound = items;
    return NPW_OK;
}

struct QueueRun {
    unsigned char* ws = nullptr;
    QLayout L{};
    cudaStream_t s = nullptr;
    npw::QueueArgs q{};
    bool fp32 = false;
    bool characteristic = false;
    int shape = npw::QS_ANY;  // the one shape every queued instance has, else QS_ANY
    // compensated float 1D items only: one launch per RK3 step (step1d_fused_body), the two
    // state buffers u and s alternating with the step parity
    bool fused = false;
    int parity = 0;
    size_t smem = 0;
    int count = 0;
    // 1D items of each flux kind are contiguous: [begin, end) per kind, for the compensated copies
    int64_t kind_begin[3] = {0, 0, 0}, kind_end[3] = {0, 0, 0};
    bool comp = false;
    std::vector<cudaEvent_t> joins;
};

npw_status queue_step(QueueRun& r) {
    npw::QueueArgs q = r.q;
    if (r.fused) {
        q.stage = npw::QUEUE_FUSED_STEP;
        q.parity = r.parity;
        auto ev = stage_begin(r.s);
        const cudaError_t e = npw::launch_queue_stage<float>(q, false, r.shape, r.smem, 0, r.s);
        stage_end(ev, r.s);
        if (e != cudaSuccess) return cuda_fail(e, "queue step launch");
        r.parity ^= 1;
        return NPW_OK;
    }
    for (int st = 0; st < 3; ++st) {
        q.stage = st;
        auto ev = stage_begin(r.s);
        const cudaError_t e = r.fp32 ? npw::launch_queue_stage<float>(q, r.characteristic, r.shape, r.smem, 0, r.s)
                                     : npw::launch_queue_stage<double>(q, r.characteristic, r.shape, r.smem, 0, r.s);
        stage_end(ev, r.s);
        if (e != cudaSuccess) return cuda_fail(e, "queue stage launch");
    }
    return NPW_OK;
}

npw_status queue_poll(const QueueRun& r, long long* act, long long* rem) {
    long long* dpoll = reinterpret_cast<long long*>(r.ws + r.L.poll);
    NPW_CUDA(npw::launch_queue_poll(r.q.ctl, r.q.inst1, r.q.inst2, r.q.is2d, r.count, dpoll, r.s));
    count_launch();
    npw_status st = bounded_sync(r.s);  // before the (blocking) copy into pageable memory
    if (st) return st;
    long long h[2] = {0, 0};
    NPW_CUDA(cudaMemcpyAsync(h, dpoll, sizeof h, cudaMemcpyDeviceToHost, r.s));
    profile_collect();
    *act = h[0];
    *rem = h[1];
    return NPW_OK;
}

npw_status queue_capture(const QueueRun& r, StepGraph& g) {
    cudaStream_t cs = nullptr;
    NPW_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    QueueRun rc;
    rc.ws = r.ws;
    rc.L = r.L;
    rc.s = cs;
    rc.q = r.q;
    rc.fp32 = r.fp32;
    rc.characteristic = r.characteristic;
    rc.shape = r.shape;
    rc.fused = r.fused;
    rc.parity = 0;  // replays start at parity 0 (GRAPH_STEPS is even)
    rc.smem = r.smem;
    cudaGraph_t graph = nullptr;
    npw_status st = NPW_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        t_capturing = true;
        for (int k = 0; k < GRAPH_STEPS && st == NPW_OK; ++k) st = queue_step(rc);
        t_capturing = false;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e2 != cudaSuccess) e = e2;
    }
    if (st == NPW_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st) return st;
    if (e != cudaSuccess) {
        g.exec = nullptr;
        return cuda_fail(e, "capture of the queue step graph");
    }
    return NPW_OK;
}

npw_status queue_run_to_end(QueueRun& r, npw_solve_stats* out) {
    long long act = 0, rem = 0;
    npw_status st = queue_poll(r, &act, &rem);
    StepGraph graph;
    bool direct_done = false;
    while (st == NPW_OK && act > 0) {
        long long chunk = rem < 1 ? 1 : (rem > 256 ? 256 : rem);
        if (chunk > GRAPH_STEPS && direct_done) {
            if (r.parity) {  // the graph's steps start at parity 0
                if ((st = queue_step(r))) break;
                --chunk;
            }
            if (!graph.exec && (st = queue_capture(r, graph))) break;
            for (long long k = 0; k < chunk / GRAPH_STEPS && st == NPW_OK; ++k) {
                auto ev = stage_begin(r.s, -1, (r.fused ? 1 : 3) * GRAPH_STEPS);
                const cudaError_t e = cudaGraphLaunch(graph.exec, r.s);
                stage_end(ev, r.s);
                if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphLaunch");
            }
            chunk %= GRAPH_STEPS;
        }
        for (long long k = 0; k < chunk && st == NPW_OK; ++k) st = queue_step(r);
        direct_done = true;
        if (st == NPW_OK) st = queue_poll(r, &act, &rem);
    }
    if (st == NPW_ETIMEOUT) graph.abandon();
    if (st == NPW_OK && r.comp) {
        // compensated 1D items: the final states are in s (per-stage steps), or, with fused steps,
        // in s for the instances that took an odd number of steps
        for (int kind = 0; kind < 3 && st == NPW_OK; ++kind) {
            const int64_t b = r.kind_begin[kind], e = r.kind_end[kind];
            if (e <= b) continue;
            const cudaError_t ce = npw::launch_comp_end(reinterpret_cast<float*>(r.q.u), r.q.s, r.q.inst1, r.q.items + b,
                                                        (int)(e - b), r.q.tile, flux_m(kind), r.fused ? r.q.ctl : nullptr,
                                                        r.s);
            if (ce != cudaSuccess) st = cuda_fail(ce, "compensated end copy");
            count_launch();
        }
    }
    for (cudaEvent_t ev : r.joins) {
        const cudaError_t e = cudaStreamWaitEvent(r.s, ev, 0);
        if (e != cudaSuccess && st == NPW_OK) st = cuda_fail(e, "cudaStreamWaitEvent");
        cudaEventDestroy(ev);
    }
    r.joins.clear();
    if (st) return st;
    std::vector<npw::Ctl> hc(r.count);
    if ((st = bounded_sync(r.s))) return st;
    NPW_CUDA(cudaMemcpyAsync(hc.data(), r.q.ctl, sizeof(npw::Ctl) * r.count, cudaMemcpyDeviceToHost, r.s));
    profile_collect();
    npw_status first = NPW_OK;
    for (int i = 0; i < r.count; ++i) {
        if (out) fill_stats(hc[i], &out[i]);
        if (hc[i].status != NPW_OK && first == NPW_OK) first = (npw_status)hc[i].status;
    }
    if (first == NPW_ENONFINITE) return fail(first, "an instance became non-finite");
    if (first != NPW_OK) return fail(first, "an instance reached its step limit or stopped advancing");
    return NPW_OK;
}

}  // namespace

extern "C" {

size_t npw_queue_workspace_size(const npw_queue_instance* inst, int32_t count, const npw_params* params) {
    if (!params) return 0;
    int64_t arena = 0, items = 0;
    if (check_queue(inst, count, params, &arena, &items) != NPW_OK) return 0;
    return queue_layout(arena, count, items, elem_size(params), compensated(params)).total;
}

npw_status npweno_queue_solve(void* arena, const npw_queue_instance* inst, int32_t count, const npw_params* params,
                              void* workspace, size_t workspace_bytes, npw_solve_stats* out, void* stream) {
    npw_status st = check_params(params);
    if (st) return st;
    if (!arena || !workspace) return fail(NPW_EINVAL, "null pointer");
    int64_t arena_elems = 0, items_bound = 0;
    if ((st = check_queue(inst, count, params, &arena_elems, &items_bound))) return st;
    QueueRun r;
    r.count = count;
    r.fp32 = params->precision == NPW_FP32_MIXED;
    r.characteristic = params->characteristic != 0;
    r.comp = compensated(params);
    r.s = reinterpret_cast<cudaStream_t>(stream);
    r.ws = static_cast<unsigned char*>(workspace);
    r.L = queue_layout(arena_elems, count, items_bound, elem_size(params), r.comp);
    if (workspace_bytes < r.L.total)
        return fail(NPW_EINVAL, "workspace too small: %zu < %zu bytes", workspace_bytes, r.L.total);
    // 1D tile: the autotuned (or given) tile of the 1D kind with the most cells
    int64_t kind_cells[3] = {0, 0, 0};
    for (int i = 0; i < count; ++i)
        if (inst[i].ny == 0) kind_cells[inst[i].flux_kind] += cells_of(inst[i]);
    int main_kind = 0;
    for (int k = 1; k < 3; ++k) main_kind = kind_cells[k] > kind_cells[main_kind] ? k : main_kind;
    int tile = resolve_tile(params, main_kind, flux_m(main_kind));
    // a batch of compensated float 1D items alone takes one launch per RK3 step
    bool any2d = false;
    for (int i = 0; i < count; ++i) any2d |= inst[i].ny != 0;
    r.fused = r.comp && !any2d;
    // automatic tile of fused steps: at most the size whose shared memory (six arrays of
    // tile + 18 cells per field) still lets the register-bound 5 CTAs share an SM (on the 1D
    // Euler batch: 512 cells 5.3e9 cell-updates/s, 1024 4.6e9, 2048 2.3e9)
    if (params->tile_1d <= 0 && r.fused)
        while (tile > npw::TILE_1D_MIN && npw::fused1d_smem_floats(tile, flux_m(main_kind)) * sizeof(float) >
                                              (size_t)44 * 1024)
            tile /= 2;
    // descriptors; mixed-precision 1D instances that fit in shared memory run resident
    std::vector<npw::InstDev> h1(count);
    std::vector<npw::Inst2D> h2(count);
    std::vector<int32_t> hk(count);
    std::vector<uint8_t> h2d(count);
    std::vector<char> resident(count, 0);
    bool has1d = false, has2d = false;
    int m1d = 1, m2d = 1;
    for (int i = 0; i < count; ++i) {
        const npw_queue_instance& q = inst[i];
        hk[i] = q.flux_kind;
        h2d[i] = q.ny != 0;
        if (q.ny == 0) {
            const int m = flux_m(q.flux_kind);
            resident[i] = resident_ok(params, m, q.nx) ? 1 : 0;
            h1[i] = npw::InstDev{q.offset, q.nx, q.dx, q.t_end, q.cfl, q.bc,
                                 resident[i] ? 0 : (int32_t)((q.nx + tile - 1) / tile)};
            if (!resident[i]) {
                has1d = true;
                m1d = m > m1d ? m : m1d;
            }
        } else {
            npw::Inst2D& d = h2[i];
            d.off = q.offset;
            d.nx = q.nx;
            d.ny = q.ny;
            d.dx = q.dx;
            d.dy = q.dy;
            d.t_end = q.t_end;
            d.cfl = q.cfl;
            d.bc = q.bc;
            d.bc_y = q.bc_y < 0 ? q.bc : q.bc_y;
            d.tiles_x = (int32_t)((q.nx + npw::TX_2D - 1) / npw::TX_2D);
            d.tiles_y = (int32_t)((q.ny + npw::TY_2D - 1) / npw::TY_2D);
            has2d = true;
            m2d = flux_m(q.flux_kind) > m2d ? flux_m(q.flux_kind) : m2d;
        }
    }
    // work items: 1D tiles grouped by flux kind, then 2D tiles
    std::vector<npw::Tile> items;
    for (int kind = 0; kind < 3; ++kind) {
        r.kind_begin[kind] = (int64_t)items.size();
        for (int i = 0; i < count; ++i) {
            if (h2d[i] || hk[i] != kind) continue;
            for (int32_t t = 0; t < h1[i].ntiles; ++t) items.push_back(npw::Tile{i, t * tile});
        }
        r.kind_end[kind] = (int64_t)items.size();
    }
    for (int i = 0; i < count; ++i)
        if (h2d[i])
            for (int32_t t = 0; t < h2[i].tiles_x * h2[i].tiles_y; ++t) items.push_back(npw::Tile{i, t});
    // one shape for every instance with queue items: the kernel specialised for it
    r.shape = -1;
    for (int i = 0; i < count && r.shape != npw::QS_ANY; ++i) {
        if (!h2d[i] && resident[i]) continue;
        const int sh = npw::queue_shape_of(h2d[i] != 0, hk[i]);
        r.shape = (r.shape < 0 || r.shape == sh) ? sh : (int)npw::QS_ANY;
    }
    if (r.shape < 0) r.shape = npw::QS_ANY;
    unsigned char* ws = r.ws;
    NPW_CUDA(cudaMemcpyAsync(ws + r.L.inst1, h1.data(), sizeof(npw::InstDev) * count, cudaMemcpyHostToDevice, r.s));
    NPW_CUDA(cudaMemcpyAsync(ws + r.L.inst2, h2.data(), sizeof(npw::Inst2D) * count, cudaMemcpyHostToDevice, r.s));
    NPW_CUDA(cudaMemcpyAsync(ws + r.L.kind, hk.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, r.s));
    NPW_CUDA(cudaMemcpyAsync(ws + r.L.is2d, h2d.data(), (size_t)count, cudaMemcpyHostToDevice, r.s));
    if (!items.empty())
        NPW_CUDA(cudaMemcpyAsync(ws + r.L.items, items.data(), sizeof(npw::Tile) * items.size(), cudaMemcpyHostToDevice,
                                 r.s));
    NPW_CUDA(cudaMemsetAsync(ws + r.L.head, 0, 2 * sizeof(unsigned int), r.s));
    npw::QueueArgs& q = r.q;
    q.u = arena;
    q.u1 = ws + r.L.u1;
    q.u2 = ws + r.L.u2;
    q.s = reinterpret_cast<float*>(ws + r.L.sbuf);
    q.c = reinterpret_cast<float*>(ws + r.L.cbuf);
    q.inst1 = reinterpret_cast<const npw::InstDev*>(ws + r.L.inst1);
    q.inst2 = reinterpret_cast<const npw::Inst2D*>(ws + r.L.inst2);
    q.kind = reinterpret_cast<const int32_t*>(ws + r.L.kind);
    q.is2d = reinterpret_cast<const uint8_t*>(ws + r.L.is2d);
    q.ctl = reinterpret_cast<npw::Ctl*>(ws + r.L.ctl);
    q.items = reinterpret_cast<const npw::Tile*>(ws + r.L.items);
    q.nitems = (int32_t)items.size();
    q.advance = 1;
    q.tile = tile;
    q.head = reinterpret_cast<unsigned int*>(ws + r.L.head);
    q.mp = method(params);
    r.smem = r.fp32 ? npw::queue_smem_bytes<float>(tile, has1d, m1d, has2d, m2d, r.characteristic)
                    : npw::queue_smem_bytes<double>(tile, has1d, m1d, has2d, m2d, r.characteristic);
    if (r.fused) r.smem = npw::fused1d_smem_floats(tile, m1d) * sizeof(float);
    // start: reset, alpha^0 over the items, first dt
    NPW_CUDA(npw::launch_queue_ctl(q.ctl, q.inst1, q.inst2, q.is2d, nullptr, count, 0, 0, r.s));
    cudaError_t e = r.fp32 ? npw::launch_queue_alpha<float>(q, r.s) : npw::launch_queue_alpha<double>(q, r.s);
    if (e != cudaSuccess) return cuda_fail(e, "queue alpha launch");
    NPW_CUDA(npw::launch_queue_ctl(q.ctl, q.inst1, q.inst2, q.is2d, nullptr, count, 1, q.mp.max_steps, r.s));
    count_launch(3);
    if (r.comp) {  // compensated 1D items: s = u, c = 0
        for (int kind = 0; kind < 3; ++kind) {
            const int64_t b = r.kind_begin[kind], en = r.kind_end[kind];
            if (en <= b) continue;
            NPW_CUDA(npw::launch_comp_begin(reinterpret_cast<const float*>(arena), q.s, q.c, q.inst1, q.items + b,
                                            (int)(en - b), tile, flux_m(kind), r.s));
            count_launch();
        }
    }
    // resident 1D instances, one launch set per flux kind, on the side streams
    bool any_res = false;
    for (int i = 0; i < count; ++i) any_res |= resident[i] != 0;
    if (any_res) {
        SideStreams* ss = nullptr;
        if ((st = side_streams(&ss))) return st;
        std::vector<int64_t> n_of(count, 0);
        std::vector<double> cost(count, 0.0);
        for (int i = 0; i < count; ++i) {
            n_of[i] = inst[i].nx;
            cost[i] = (double)inst[i].nx * inst[i].t_end / (inst[i].cfl * inst[i].dx);
        }
        int64_t list_off = 0;  // the kinds' index lists occupy disjoint parts of the list buffer
        for (int kind = 0; kind < 3; ++kind) {
            std::vector<int32_t> ids;
            for (int i = 0; i < count; ++i)
                if (resident[i] && hk[i] == kind) ids.push_back(i);
            if (ids.empty()) continue;
            ResidentLaunch rl{arena, q.c, q.inst1, q.ctl, reinterpret_cast<int32_t*>(ws + r.L.list) + list_off,
                              flux_m(kind), kind, q.mp};
            if ((st = launch_resident_set(rl, ids, n_of, cost, ss, r.s, r.joins))) return st;
            list_off += (int64_t)ids.size();
        }
    }
    return queue_run_to_end(r, out);
}

}  // extern "C"

// =======================================================================================
// Request server: continuous batching over the work-queue kernel, one lane per precision
// =======================================================================================
namespace {

constexpr double kMixedTolerance = 1e-4;  // requests with tolerance >= this take the mixed lane
constexpr int kGroups = 7;                // instance shapes (npw::QueueShape): one launch group each
constexpr double kStepSliceS = 0.005;     // longest wait of npw_server_step for a round to end

struct LaneLayout {
    size_t inst1, inst2, kind, is2d, ctl, items, newitems, list, head, poll, heap_u, heap_u1, heap_u2, heap_s, heap_c;
    size_t begin, end;
    int64_t max_items;
};

// one lane's part of the arena, starting at byte `begin`
LaneLayout lane_layout(size_t begin, int64_t heap_cells, int max_slots, size_t esz, bool comp) {
    LaneLayout L{};
    L.max_items = heap_cells / (npw::TX_2D * npw::TY_2D) + 2 * (int64_t)max_slots;
    size_t o = align256(begin);
    L.begin = o;
    L.inst1 = o;
    o = align256(o + sizeof(npw::InstDev) * (size_t)max_slots);
    L.inst2 = o;
    o = align256(o + sizeof(npw::Inst2D) * (size_t)max_slots);
    L.kind = o;
    o = align256(o + sizeof(int32_t) * (size_t)max_slots);
    L.is2d = o;
    o = align256(o + (size_t)max_slots);
    L.ctl = o;
    o = align256(o + sizeof(npw::Ctl) * (size_t)max_slots);
    L.items = o;
    o = align256(o + sizeof(npw::Tile) * (size_t)L.max_items);
    L.newitems = o;
    o = align256(o + sizeof(npw::Tile) * (size_t)L.max_items);
    L.list = o;
    o = align256(o + sizeof(int32_t) * (size_t)max_slots);
    L.head = o;  // a queue counter pair per launch group
    o = align256(o + 2 * kGroups * sizeof(unsigned int));
    L.poll = o;
    o = align256(o + 256);
    L.heap_u = o;
    o = align256(o + (size_t)heap_cells * esz);
    L.heap_u1 = o;
    o = align256(o + (size_t)heap_cells * esz);
    L.heap_u2 = o;
    o = align256(o + (size_t)heap_cells * esz);
    const size_t extra = comp ? (size_t)heap_cells * sizeof(float) : 0;  // compensated float 1D
    L.heap_s = o;
    o = align256(o + extra);
    L.heap_c = o;
    o = align256(o + extra);
    L.end = o;
    return L;
}

// lane 0: NPW_FP32_MIXED (compensated 1D items), lane 1: NPW_FP64
size_t server_bytes(int64_t heap_cells, int max_slots) {
    const LaneLayout a = lane_layout(0, heap_cells, max_slots, sizeof(float), true);
    return lane_layout(a.end, heap_cells, max_slots, sizeof(double), false).end;
}

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// 1D tile of the float lane's fused steps: the largest whose six shared arrays (tile + 18 cells
// per field) stay within 44 KB, so that five CTAs share an SM (1024 cells for m = 1, 512 for
// 1D Euler)
int fused_tile(int m) {
    int t = npw::TILE_1D;
    while (t > npw::TILE_1D_MIN && npw::fused1d_smem_floats(t, m) * sizeof(float) > (size_t)44 * 1024) t /= 2;
    return t;
}

}  // namespace

struct npw_server {
    npw_params params;
    int max_slots = 0;
    cudaStream_t s = nullptr;  // the caller's stream: creation, lane 0 (float)
    unsigned char* arena = nullptr;
    int64_t heap_cells = 0;
    std::chrono::steady_clock::time_point t0;
    struct Pending {
        uint64_t id;
        npw_request req;
        double submit_s;
    };
    // A lane runs its rounds on its own stream, independently of the other lane: a round is
    // launched, and retired by a later npw_server_step once its completion event has fired.
    struct Lane {
        LaneLayout L{};
        npw::MethodParams mp{};
        bool fp32 = false;
        size_t esz = 8;
        cudaStream_t st = nullptr;             // lane 0: the caller's stream; lane 1: its own
        bool own_stream = false;
        cudaStream_t sub[kGroups] = {};        // one stream per instance shape within a round
        cudaEvent_t fork = nullptr, done = nullptr, join[kGroups] = {};
        bool in_flight = false;                // a round has been launched and not yet retired
        double launched_s = 0.0;               // when (seconds since creation)
        std::deque<Pending> pending;           // submitted, not yet admitted (first in first out)
        long long remaining_hint = 0;          // largest remaining step estimate after the last round
        std::vector<std::pair<int64_t, int64_t>> free_ranges;  // [begin, end), sorted, disjoint
        std::vector<npw::Ctl> host_ctl;
        bool heap_alloc(int64_t len, int64_t* off) {
            for (size_t k = 0; k < free_ranges.size(); ++k) {
                auto& r = free_ranges[k];
                if (r.second - r.first >= len) {
                    *off = r.first;
                    r.first += len;
                    if (r.first == r.second) free_ranges.erase(free_ranges.begin() + (long)k);
                    return true;
                }
            }
            return false;
        }
        void heap_free(int64_t off, int64_t len) {
            free_ranges.push_back({off, off + len});
            std::sort(free_ranges.begin(), free_ranges.end());
            std::vector<std::pair<int64_t, int64_t>> merged;
            for (auto& r : free_ranges) {
                if (!merged.empty() && merged.back().second == r.first)
                    merged.back().second = r.second;
                else
                    merged.push_back(r);
            }
            free_ranges.swap(merged);
        }
        void release() {
            if (st) bounded_sync(st);  // no round of this lane may outlive the server
            for (int g = 0; g < kGroups; ++g) {
                if (join[g]) cudaEventDestroy(join[g]);
                if (sub[g]) cudaStreamDestroy(sub[g]);
            }
            if (fork) cudaEventDestroy(fork);
            if (done) cudaEventDestroy(done);
            if (own_stream && st) cudaStreamDestroy(st);
        }
    } lanes[2];
    ~npw_server() {
        for (auto& ln : lanes) ln.release();
    }
    struct Slot {
        bool used = false;
        bool fresh = false;
        uint64_t id = 0;
        npw_request req{};
        int lane = 0;
        int m = 1;
        bool is2d = false;
        bool fused = false;  // float lane 1D: fused steps, the state alternating between u and s
        int64_t cells = 0;   // heap cells: m n (2D: m n ny)
        int64_t off = 0;
        double submit_s = 0.0, admit_s = 0.0;
    };
    std::vector<Slot> slots;  // a slot's index is its instance index in its lane's tables
    std::deque<npw_result> results;
    uint64_t next_id = 1;

    // the lane of a request: its tolerance, else the server's precision
    int lane_of(const npw_request& r) const {
        if (r.tolerance > 0.0) return r.tolerance >= kMixedTolerance ? 0 : 1;
        return params.precision == NPW_FP32_MIXED ? 0 : 1;
    }
    size_t pending_count() const { return lanes[0].pending.size() + lanes[1].pending.size(); }
};

namespace {

// the queue arguments of a lane (all its slots; items, counts, tile and counters filled per group)
npw::QueueArgs lane_queue(npw_server* sv, int ln) {
    npw_server::Lane& lane = sv->lanes[ln];
    const LaneLayout& L = lane.L;
    unsigned char* a = sv->arena;
    npw::QueueArgs q{};
    q.u = a + L.heap_u;
    q.u1 = a + L.heap_u1;
    q.u2 = a + L.heap_u2;
    q.s = reinterpret_cast<float*>(a + L.heap_s);
    q.c = reinterpret_cast<float*>(a + L.heap_c);
    q.inst1 = reinterpret_cast<const npw::InstDev*>(a + L.inst1);
    q.inst2 = reinterpret_cast<const npw::Inst2D*>(a + L.inst2);
    q.kind = reinterpret_cast<const int32_t*>(a + L.kind);
    q.is2d = reinterpret_cast<const uint8_t*>(a + L.is2d);
    q.ctl = reinterpret_cast<npw::Ctl*>(a + L.ctl);
    q.items = reinterpret_cast<const npw::Tile*>(a + L.items);
    q.advance = 1;
    q.tile = npw::TILE_1D;
    q.head = reinterpret_cast<unsigned int*>(a + L.head);
    q.mp = lane.mp;
    return q;
}

// Instance tables, work items and start of a lane's admitted requests; then `steps` RK3 steps
// (an even count) of every active request of the lane.  The requests are grouped by instance
// shape; each group runs on its own stream, forked from the lane's stream and joined back, with
// the queue kernel specialised for that shape (one persistent launch per stage; for the float
// lane's 1D requests one per fused RK3 step, whose two state buffers alternate with the step
// parity: every round starts at parity 0 because rounds have even length and requests are
// admitted only between rounds).
npw_status lane_round(npw_server* sv, int ln, int steps) {
    npw_server::Lane& lane = sv->lanes[ln];
    const cudaStream_t ls = lane.st;
    const int S = sv->max_slots;
    struct Group {
        std::vector<int> members;
        bool is2d = false, fused = false;
        int m = 1, tile = npw::TILE_1D;
        int64_t ib = 0, ie = 0, nb = 0, ne = 0;  // [ib, ie) in items, [nb, ne) in newitems
    } grp[kGroups];
    std::vector<npw::InstDev> h1(S);
    std::vector<npw::Inst2D> h2(S);
    std::vector<int32_t> hk(S, 0);
    std::vector<uint8_t> h2d(S, 0);
    std::vector<npw::Tile> items, newitems;
    std::vector<int32_t> fresh;
    for (int k = 0; k < S; ++k) {
        npw_server::Slot& sl = sv->slots[k];
        if (!sl.used || sl.lane != ln) continue;
        Group& g = grp[npw::queue_shape_of(sl.is2d, sl.req.flux_kind)];
        g.members.push_back(k);
        g.is2d = sl.is2d;
        g.m = sl.m;
        g.fused = sl.fused;
        g.tile = sl.fused ? fused_tile(sl.m) : npw::TILE_1D;
        hk[k] = sl.req.flux_kind;
        h2d[k] = sl.is2d;
        if (!sl.is2d) {
            h1[k] = npw::InstDev{sl.off, sl.req.n, sl.req.dx, sl.req.t_end, sl.req.cfl, sl.req.bc,
                                 (int32_t)tiles_of(sl.req.n, g.tile)};
        } else {
            npw::Inst2D& d = h2[k];
            d.off = sl.off;
            d.nx = sl.req.n;
            d.ny = sl.req.ny;
            d.dx = sl.req.dx;
            d.dy = sl.req.dy;
            d.t_end = sl.req.t_end;
            d.cfl = sl.req.cfl;
            d.bc = sl.req.bc;
            d.bc_y = sl.req.bc_y < 0 ? sl.req.bc : sl.req.bc_y;
            d.tiles_x = (int32_t)((sl.req.n + npw::TX_2D - 1) / npw::TX_2D);
            d.tiles_y = (int32_t)((sl.req.ny + npw::TY_2D - 1) / npw::TY_2D);
        }
        if (sl.fresh) fresh.push_back(k);
    }
    // work items, contiguous per group; the admitted requests' items likewise
    for (int gi = 0; gi < kGroups; ++gi) {
        Group& g = grp[gi];
        g.ib = (int64_t)items.size();
        g.nb = (int64_t)newitems.size();
        for (int k : g.members) {
            const bool fr = sv->slots[k].fresh;
            if (!g.is2d) {
                for (int32_t t = 0; t < h1[k].ntiles; ++t) {
                    items.push_back(npw::Tile{k, t * g.tile});
                    if (fr) newitems.push_back(npw::Tile{k, t * g.tile});
                }
            } else {
                for (int32_t t = 0; t < h2[k].tiles_x * h2[k].tiles_y; ++t) {
                    items.push_back(npw::Tile{k, t});
                    if (fr) newitems.push_back(npw::Tile{k, t});
                }
            }
        }
        g.ie = (int64_t)items.size();
        g.ne = (int64_t)newitems.size();
    }
    if (items.empty()) return NPW_OK;
    if ((int64_t)items.size() > lane.L.max_items) return fail(NPW_EINVAL, "server: too many work items");
    const LaneLayout& L = lane.L;
    unsigned char* a = sv->arena;
    NPW_CUDA(cudaMemcpyAsync(a + L.inst1, h1.data(), sizeof(npw::InstDev) * S, cudaMemcpyHostToDevice, ls));
    NPW_CUDA(cudaMemcpyAsync(a + L.inst2, h2.data(), sizeof(npw::Inst2D) * S, cudaMemcpyHostToDevice, ls));
    NPW_CUDA(cudaMemcpyAsync(a + L.kind, hk.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, ls));
    NPW_CUDA(cudaMemcpyAsync(a + L.is2d, h2d.data(), (size_t)S, cudaMemcpyHostToDevice, ls));
    NPW_CUDA(cudaMemcpyAsync(a + L.items, items.data(), sizeof(npw::Tile) * items.size(), cudaMemcpyHostToDevice,
                             ls));
    const npw::QueueArgs q0 = lane_queue(sv, ln);
    const npw::Tile* ditems = q0.items;
    const npw::Tile* dnew = reinterpret_cast<const npw::Tile*>(a + L.newitems);
    if (!fresh.empty()) {
        // start the admitted requests: reset, alpha^0 over their items, first dt and step limit
        int32_t* dlist = reinterpret_cast<int32_t*>(a + L.list);
        NPW_CUDA(cudaMemcpyAsync(dlist, fresh.data(), sizeof(int32_t) * fresh.size(), cudaMemcpyHostToDevice, ls));
        NPW_CUDA(cudaMemcpyAsync(a + L.newitems, newitems.data(), sizeof(npw::Tile) * newitems.size(),
                                 cudaMemcpyHostToDevice, ls));
        NPW_CUDA(npw::launch_queue_ctl(q0.ctl, q0.inst1, q0.inst2, q0.is2d, dlist, (int)fresh.size(), 0, 0, ls));
        count_launch();
        for (int gi = 0; gi < kGroups; ++gi) {
            const Group& g = grp[gi];
            if (g.ne <= g.nb) continue;
            npw::QueueArgs qn = q0;
            qn.items = dnew + g.nb;
            qn.nitems = (int32_t)(g.ne - g.nb);
            qn.tile = g.tile;
            const cudaError_t e = lane.fp32 ? npw::launch_queue_alpha<float>(qn, ls) : npw::launch_queue_alpha<double>(qn, ls);
            if (e != cudaSuccess) return cuda_fail(e, "server alpha launch");
            count_launch();
        }
        NPW_CUDA(npw::launch_queue_ctl(q0.ctl, q0.inst1, q0.inst2, q0.is2d, dlist, (int)fresh.size(), 1, q0.mp.max_steps,
                                       ls));
        count_launch();
        if (lane.fp32) {  // compensated float 1D items: s = u, c = 0
            for (int gi = 0; gi < kGroups; ++gi) {
                const Group& g = grp[gi];
                if (g.is2d || g.ne <= g.nb) continue;
                NPW_CUDA(npw::launch_comp_begin(reinterpret_cast<const float*>(q0.u), q0.s, q0.c, q0.inst1, dnew + g.nb,
                                                (int)(g.ne - g.nb), g.tile, g.m, ls));
                count_launch();
            }
        }
    }
    NPW_CUDA(cudaEventRecord(lane.fork, ls));
    for (int gi = 0; gi < kGroups; ++gi) {
        const Group& g = grp[gi];
        if (g.ie <= g.ib) continue;
        const cudaStream_t gs = lane.sub[gi];
        NPW_CUDA(cudaStreamWaitEvent(gs, lane.fork, 0));
        npw::QueueArgs q = q0;
        q.items = ditems + g.ib;
        q.nitems = (int32_t)(g.ie - g.ib);
        q.tile = g.tile;
        q.head = q0.head + 2 * gi;
        size_t smem;
        if (g.fused)
            smem = npw::fused1d_smem_floats(g.tile, g.m) * sizeof(float);
        else if (lane.fp32)
            smem = npw::queue_smem_bytes<float>(g.tile, !g.is2d, g.m, g.is2d, g.m, false);
        else
            smem = npw::queue_smem_bytes<double>(g.tile, !g.is2d, g.m, g.is2d, g.m, false);
        for (int step = 0; step < steps; ++step) {
            if (g.fused) {
                q.stage = npw::QUEUE_FUSED_STEP;
                q.parity = step & 1;
                auto ev = stage_begin(gs);
                const cudaError_t e = npw::launch_queue_stage<float>(q, false, gi, smem, 0, gs);
                stage_end(ev, gs);
                if (e != cudaSuccess) return cuda_fail(e, "server fused step launch");
                continue;
            }
            for (int st = 0; st < 3; ++st) {
                q.stage = st;
                auto ev = stage_begin(gs);
                const cudaError_t e = lane.fp32 ? npw::launch_queue_stage<float>(q, false, gi, smem, 0, gs)
                                                : npw::launch_queue_stage<double>(q, false, gi, smem, 0, gs);
                stage_end(ev, gs);
                if (e != cudaSuccess) return cuda_fail(e, "server queue stage launch");
            }
        }
        NPW_CUDA(cudaEventRecord(lane.join[gi], gs));
        NPW_CUDA(cudaStreamWaitEvent(ls, lane.join[gi], 0));
    }
    return NPW_OK;
}

// The lane's round has ended: read its control words, copy finished states to their host
// buffers, record their results and free their heap space.
npw_status lane_retire(npw_server* sv, int ln) {
    npw_server::Lane& lane = sv->lanes[ln];
    npw_status st = bounded_sync(lane.st);
    if (st) return st;
    lane.in_flight = false;
    NPW_CUDA(cudaMemcpyAsync(lane.host_ctl.data(), sv->arena + lane.L.ctl, sizeof(npw::Ctl) * sv->max_slots,
                             cudaMemcpyDeviceToHost, lane.st));
    if ((st = bounded_sync(lane.st))) return st;
    profile_collect();
    std::vector<int> finished;
    long long rem = 0;
    for (int k = 0; k < sv->max_slots; ++k) {
        const npw_server::Slot& sl = sv->slots[k];
        if (!sl.used || sl.lane != ln) continue;
        const npw::Ctl& c = lane.host_ctl[k];
        if (c.done) {
            finished.push_back(k);
        } else {
            const double r = c.dt > 0.0 ? (sl.req.t_end - c.t) / c.dt : 1.0;
            const long long ri = (long long)(r < 1e9 ? r : 1e9) + 1;
            rem = ri > rem ? ri : rem;
        }
    }
    lane.remaining_hint = rem;
    for (int k : finished) {
        // the float lane's 1D requests end in s after an odd number of fused steps, else in u
        const npw_server::Slot& sl = sv->slots[k];
        const size_t region = (sl.fused && (lane.host_ctl[k].steps & 1)) ? lane.L.heap_s : lane.L.heap_u;
        NPW_CUDA(cudaMemcpyAsync(sl.req.out_host, sv->arena + region + (size_t)sl.off * lane.esz,
                                 (size_t)sl.cells * lane.esz, cudaMemcpyDeviceToHost, lane.st));
    }
    if (!finished.empty() && (st = bounded_sync(lane.st))) return st;
    const double tdone = now_s(sv->t0);
    for (int k : finished) {
        npw_server::Slot& sl = sv->slots[k];
        const npw::Ctl& c = lane.host_ctl[k];
        npw_result r{};
        r.id = sl.id;
        r.tag = sl.req.tag;
        r.status = c.status;
        r.precision = ln == 0 ? NPW_FP32_MIXED : NPW_FP64;
        r.steps = c.steps;
        r.t = c.t;
        r.submit_s = sl.submit_s;
        r.admit_s = sl.admit_s;
        r.done_s = tdone;
        sv->results.push_back(r);
        lane.heap_free(sl.off, sl.cells);
        sl.used = false;
    }
    return NPW_OK;
}

// Admit the lane's pending requests (first in first out, while a slot and heap space are
// free), then launch its next round if it has active requests.
npw_status lane_next_round(npw_server* sv, int ln, int base_steps) {
    npw_server::Lane& lane = sv->lanes[ln];
    bool admitted = false;
    while (!lane.pending.empty()) {
        const npw_server::Pending& p = lane.pending.front();
        const int m = flux_m(p.req.flux_kind);
        const bool is2d = p.req.ny != 0;
        const int64_t cells = p.req.n * m * (is2d ? p.req.ny : 1);
        int slot = -1;
        for (int k = 0; k < sv->max_slots; ++k)
            if (!sv->slots[k].used) {
                slot = k;
                break;
            }
        int64_t off = 0;
        if (slot < 0 || !lane.heap_alloc(cells, &off)) break;
        // the request's host values are of its lane's element type
        NPW_CUDA(cudaMemcpyAsync(sv->arena + lane.L.heap_u + (size_t)off * lane.esz, p.req.u0_host,
                                 (size_t)cells * lane.esz, cudaMemcpyHostToDevice, lane.st));
        npw_server::Slot& sl = sv->slots[slot];
        sl.used = true;
        sl.fresh = true;
        sl.id = p.id;
        sl.req = p.req;
        sl.lane = ln;
        sl.m = m;
        sl.is2d = is2d;
        sl.fused = lane.fp32 && !is2d;
        sl.cells = cells;
        sl.off = off;
        sl.submit_s = p.submit_s;
        sl.admit_s = now_s(sv->t0);
        lane.pending.pop_front();
        admitted = true;
    }
    bool any = false;
    for (int k = 0; k < sv->max_slots && !any; ++k) any = sv->slots[k].used && sv->slots[k].lane == ln;
    if (!any) return NPW_OK;
    // a shorter round when nothing was admitted and every active request is close to its end
    int steps = base_steps;
    if (!admitted && lane.remaining_hint > 0 && lane.remaining_hint < steps)
        steps = (int)((lane.remaining_hint + 1) & ~1LL);
    if (steps < 2) steps = 2;
    const npw_status st = lane_round(sv, ln, steps);
    for (int k = 0; k < sv->max_slots; ++k)
        if (sv->slots[k].used && sv->slots[k].lane == ln) sv->slots[k].fresh = false;
    if (st) return st;
    NPW_CUDA(cudaEventRecord(lane.done, lane.st));
    lane.in_flight = true;
    lane.launched_s = now_s(sv->t0);
    return NPW_OK;
}

// Wait until the round of some lane in flight has ended, at most `slice` seconds; *which =
// that lane, or -1 when none ended (or none is in flight).  A round in flight for longer than
// the wait limit (NPW_WAIT_TIMEOUT_S) is an error (NPW_ETIMEOUT).
npw_status wait_any_lane(npw_server* sv, double slice, int* which) {
    *which = -1;
    if (!sv->lanes[0].in_flight && !sv->lanes[1].in_flight) return NPW_OK;
    const auto t0 = std::chrono::steady_clock::now();
    const double limit = wait_timeout_s();
    for (;;) {
        for (int ln = 0; ln < 2; ++ln) {
            const npw_server::Lane& lane = sv->lanes[ln];
            if (!lane.in_flight) continue;
            const cudaError_t e = cudaEventQuery(lane.done);
            if (e == cudaSuccess) {
                *which = ln;
                return NPW_OK;
            }
            if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery");
            if (now_s(sv->t0) - lane.launched_s > limit)
                return fail(NPW_ETIMEOUT, "a server round did not complete within %.0f s", limit);
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > slice) return NPW_OK;
        if (el > 1e-4) {
            struct timespec ts = {0, 20000};
            nanosleep(&ts, nullptr);
        }
    }
}

}  // namespace

extern "C" {

size_t npw_server_arena_bytes(int64_t heap_cells, int32_t max_slots, const npw_params* params) {
    if (!params || heap_cells < 1 || max_slots < 1) return 0;
    return server_bytes(heap_cells, max_slots);
}

npw_status npw_server_create(void* device_arena, size_t arena_bytes, int32_t max_slots, const npw_params* params,
                             void* stream, npw_server** out) {
    npw_status st = check_params(params);
    if (st) return st;
    if (!device_arena || !out || max_slots < 1 || max_slots > (1 << 20)) return fail(NPW_EINVAL, "bad server arguments");
    if (params->characteristic) return fail(NPW_EINVAL, "the server runs component-wise reconstruction");
    if (params->gauss_2d) return fail(NPW_EINVAL, "the server takes one quadrature point per face (gauss_2d = 0)");
    // largest heap (per lane) that fits the arena
    int64_t lo = 0, hi = (int64_t)(arena_bytes / 44) + 1;
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (server_bytes(mid, max_slots) <= arena_bytes)
            lo = mid;
        else
            hi = mid;
    }
    if (lo < 36) return fail(NPW_EINVAL, "arena too small for a server with %d slots", max_slots);
    npw_server* sv = new (std::nothrow) npw_server();
    if (!sv) return fail(NPW_ENOMEM, "host allocation of the server failed");
    sv->params = *params;
    sv->max_slots = max_slots;
    sv->s = reinterpret_cast<cudaStream_t>(stream);
    sv->arena = static_cast<unsigned char*>(device_arena);
    sv->heap_cells = lo;
    // the float lane's launch groups run at the greatest stream priority: where both lanes have
    // work queued, the GPU starts the float lane's short launches first as the FP64 lane's
    // persistent CTAs retire, so the low-latency class does not wait for whole FP64 rounds
    int prio_least = 0, prio_greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    for (int ln = 0; ln < 2 && e == cudaSuccess; ++ln) {
        npw_server::Lane& lane = sv->lanes[ln];
        npw_params pl = *params;
        pl.precision = ln == 0 ? NPW_FP32_MIXED : NPW_FP64;
        pl.batch_mode = 1;
        lane.mp = method(&pl);
        lane.fp32 = ln == 0;
        lane.esz = ln == 0 ? sizeof(float) : sizeof(double);
        lane.L = ln == 0 ? lane_layout(0, lo, max_slots, sizeof(float), true)
                         : lane_layout(sv->lanes[0].L.end, lo, max_slots, sizeof(double), false);
        lane.free_ranges.push_back({0, lo});
        lane.host_ctl.resize(max_slots);
        // zero the queue counters once; every launch leaves them zero
        e = cudaMemsetAsync(sv->arena + lane.L.head, 0, 2 * kGroups * sizeof(unsigned int), sv->s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lane.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lane.done, cudaEventDisableTiming);
        for (int g = 0; g < kGroups && e == cudaSuccess; ++g) {
            e = cudaStreamCreateWithPriority(&lane.sub[g], cudaStreamNonBlocking, ln == 0 ? prio_greatest : prio_least);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lane.join[g], cudaEventDisableTiming);
        }
        if (ln == 0) {
            lane.st = sv->s;
        } else if (e == cudaSuccess) {
            e = cudaStreamCreateWithPriority(&lane.st, cudaStreamNonBlocking, prio_least);
            lane.own_stream = e == cudaSuccess;
        }
    }
    // the FP64 lane's stream starts after the counters are zeroed on the caller's stream
    if (e == cudaSuccess) e = cudaEventRecord(sv->lanes[1].fork, sv->s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sv->lanes[1].st, sv->lanes[1].fork, 0);
    if (e != cudaSuccess) {
        delete sv;
        return cuda_fail(e, "server streams");
    }
    sv->slots.resize(max_slots);
    sv->t0 = std::chrono::steady_clock::now();
    *out = sv;
    return NPW_OK;
}

void npw_server_destroy(npw_server* s) { delete s; }

npw_status npw_server_submit(npw_server* sv, const npw_request* req, uint64_t* id) {
    if (!sv || !req) return fail(NPW_EINVAL, "null server or request");
    const bool is2d = req->ny != 0;
    if (!is2d && req->flux_kind != NPW_FLUX_ADVECTION && req->flux_kind != NPW_FLUX_BURGERS &&
        req->flux_kind != NPW_FLUX_EULER1D)
        return fail(NPW_EINVAL, "request flux kind %d is not a 1D flux", req->flux_kind);
    if (is2d && req->flux_kind != NPW_FLUX_ADVECTION && req->flux_kind != NPW_FLUX_BURGERS &&
        req->flux_kind != NPW_FLUX_EULER2D)
        return fail(NPW_EINVAL, "request flux kind %d is not a 2D flux", req->flux_kind);
    npw_status st = check_bc(req->bc);
    if (st) return st;
    if (req->n < 6 || req->n > ((int64_t)1 << 30) || !(req->dx > 0.0) || !(req->cfl > 0.0) || !req->u0_host ||
        !req->out_host || !(req->tolerance >= 0.0))
        return fail(NPW_EINVAL, "malformed request");
    if (is2d) {
        if (req->ny < 6 || req->ny > ((int64_t)1 << 30) || !(req->dy > 0.0))
            return fail(NPW_EINVAL, "malformed 2D request (ny >= 6, dy > 0)");
        if (req->bc_y >= 0 && (st = check_bc(req->bc_y))) return st;
    }
    const int m = flux_m(req->flux_kind);
    const int64_t cells = req->n * m * (is2d ? req->ny : 1);
    if (cells > sv->heap_cells) return fail(NPW_EINVAL, "request larger than the server heap");
    if ((int)sv->pending_count() >= sv->max_slots) return fail(NPW_EBUSY, "request queue full");
    npw_server::Pending p{sv->next_id++, *req, now_s(sv->t0)};
    sv->lanes[sv->lane_of(*req)].pending.push_back(p);
    if (id) *id = p.id;
    return NPW_OK;
}

npw_status npw_server_step(npw_server* sv, int32_t max_steps, int32_t* active, int32_t* queued) {
    if (!sv || max_steps < 1) return fail(NPW_EINVAL, "bad server step arguments");
    const int base_steps = max_steps >= 2 ? (max_steps & ~1) : 2;
    npw_status st = NPW_OK;
    bool retired = false;
    // every lane whose round has ended (or that has none): retire, admit, launch the next round
    for (int ln = 0; ln < 2; ++ln) {
        npw_server::Lane& lane = sv->lanes[ln];
        if (lane.in_flight) {
            const cudaError_t e = cudaEventQuery(lane.done);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventQuery");
            if ((st = lane_retire(sv, ln))) return st;
            retired = true;
        }
        if ((st = lane_next_round(sv, ln, base_steps))) return st;
    }
    // no round ended during this call: wait for the first one that does, at most a short slice,
    // so that the caller can submit requests that arrive meanwhile
    if (!retired) {
        int ln = -1;
        if ((st = wait_any_lane(sv, kStepSliceS, &ln))) return st;
        if (ln >= 0) {
            if ((st = lane_retire(sv, ln))) return st;
            if ((st = lane_next_round(sv, ln, base_steps))) return st;
        }
    }
    int n_active = 0;
    for (int k = 0; k < sv->max_slots; ++k) n_active += sv->slots[k].used ? 1 : 0;
    if (active) *active = n_active;
    if (queued) *queued = (int32_t)sv->pending_count();
    return NPW_OK;
}

npw_status npw_server_poll(npw_server* sv, npw_result* out, int32_t max, int32_t* nout) {
    if (!sv || (!out && max > 0) || !nout) return fail(NPW_EINVAL, "bad poll arguments");
    int32_t k = 0;
    while (k < max && !sv->results.empty()) {
        out[k++] = sv->results.front();
        sv->results.pop_front();
    }
    *nout = k;
    return NPW_OK;
}

}  // extern "C"
