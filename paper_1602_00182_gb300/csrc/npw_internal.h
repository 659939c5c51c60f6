// npw_internal.h -- types shared by the kernels and the host runtime of libnpweno.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "npweno.h"

namespace npw {

constexpr int NPW_ENO_ = NPW_ENO;
constexpr int NPW_WENO_JS_ = NPW_WENO_JS;
constexpr int NPW_RBF_ENO_ = NPW_RBF_ENO;
constexpr int NPW_RBF_WENO_ = NPW_RBF_WENO;
constexpr int NPW_RBF_MQ_ = NPW_RBF_MQ;
constexpr int NPW_RBF_GA_ = NPW_RBF_GA;
constexpr int NPW_FLUX_ADVECTION_ = NPW_FLUX_ADVECTION;
constexpr int NPW_FLUX_BURGERS_ = NPW_FLUX_BURGERS;
constexpr int NPW_FLUX_EULER1D_ = NPW_FLUX_EULER1D;
constexpr int NPW_FLUX_EULER2D_ = NPW_FLUX_EULER2D;

// Flag byte of a face (npweno_reconstruct's flags output; the kernels count from it).
constexpr uint32_t FL_SWITCH = 0x01u;       // monotone switch fired (k = 2: of the left cell)
constexpr uint32_t FL_NEAR_TIE = 0x02u;     // a switch or ENO decision within the tie margin
constexpr uint32_t FL_SWITCH_R_K2 = 0x08u;  // k = 2: switch of the right cell
constexpr uint32_t FL_ZERO_GUARD = 0x40u;   // an evaluated eta set to 0 by the guard (k = 2: of v^-)
constexpr uint32_t FL_ZERO_BOUND = 0x80u;   // an evaluated eta set to 0 by the bound (k = 2: of v^-)
// k = 2, in the 32-bit flag word only: the same for the eta of v^+ (the byte of
// npweno_reconstruct folds them into bits 6 and 7)
constexpr uint32_t FL_ZERO_GUARD_R_K2 = 0x100u;
constexpr uint32_t FL_ZERO_BOUND_R_K2 = 0x200u;
__host__ __device__ __forceinline__ uint8_t flag_byte(uint32_t fl) {
    return (uint8_t)((fl & 0xFFu) | ((fl >> 2) & 0xC0u));
}

// Per-thread counts of the shape-parameter decisions (per face for k = 3, per face value for
// k = 2): the switch fired, eta evaluated, and of those zeroed by the guard / the bound.
struct EtaCount {
    uint32_t sw = 0, ev = 0, guard = 0, bound = 0;
    // one face of k = 3 from its flag word
    __device__ __forceinline__ void face_k3(uint32_t fl) {
        sw += fl & FL_SWITCH;
        ev += (fl & FL_SWITCH) ^ 1u;
        guard += (fl >> 6) & 1u;
        bound += (fl >> 7) & 1u;
    }
    // both face values (v^- of the left cell, v^+ of the right cell) of a k = 2 face
    __device__ __forceinline__ void face_k2(uint32_t fl) {
        const uint32_t s = (fl & FL_SWITCH) + ((fl >> 3) & 1u);
        sw += s;
        ev += 2u - s;
        guard += ((fl >> 6) & 1u) + ((fl >> 8) & 1u);
        bound += ((fl >> 7) & 1u) + ((fl >> 9) & 1u);
    }
    __device__ __forceinline__ void face(uint32_t fl, int k) {
        if (k == 2)
            face_k2(fl);
        else
            face_k3(fl);
    }
};

// Method parameters as the kernels see them (by value in the launch arguments).
struct MethodParams {
    int scheme;
    int rbf;
    int monotone_switch;
    int switch_variant;
    int characteristic;
    int eta_eval;  // mixed precision, k = 3: 0 = double-float quotient (no FP64), 1 = FP64 evaluation
    int k;         // 2 (ENO2 / WENO3) or 3 (ENO3 / WENO5)
    int cross_2d;  // k = 2 in 2D: shape parameter on the 5-cell cross (Sec. 6)
    int gauss_2d;  // k = 2 in 2D: two Gauss points per face (eq. 2DIntegral), else the midpoint
    double eps_M;
    double eps_weno;
    double gamma;
    double adv_speed;
    double adv_speed_y;
    double inflow[4];
    double eta_guard;  // resolved threshold (0 = off)
    double eta_max;    // resolved bound on |eta| (0 = off)
    double tie_tol;    // relative margin of the near-tie bit of npweno_reconstruct
    int64_t max_steps; // step limit of a solve (0 = automatic, see step_cap)
    // the same values rounded once to float on the host, for the float state (a conversion
    // in the kernels would take FP64-pipe slots)
    float eps_weno_f, eps_M_f, eps_M_lo_f, eta_guard_f, eta_max_f;  // eps_M ~ eps_M_f + eps_M_lo_f
    float gamma_f, adv_speed_f, adv_speed_y_f;
    float inflow_f[4];
};

// a method parameter in the arithmetic type R: the double value, or its float copy
template <typename R>
__host__ __device__ __forceinline__ R mp_val(double d, float f) {
    if constexpr (sizeof(R) == sizeof(float))
        return f;
    else
        return R(d);
}

// One 1D problem (device copy of npw_instance plus its tile range).
struct InstDev {
    int64_t off;  // element offset of the [m][n] block in the arena
    int64_t n;
    double dx;
    double t_end;
    double cfl;
    int32_t bc;
    int32_t ntiles;
};

// Per-instance time control, owned by the device.  Written only by the last CTA of the
// instance in stage 3 (or by the init kernels); read by every CTA of the next step.
struct Ctl {
    double t;
    double dt;
    double alpha;       // Lax-Friedrichs alpha of the current step (max |f'(u^n)|)
    double alpha_max;   // largest alpha seen
    unsigned long long alpha_next_bits;  // running max for the next step (bits of a double >= 0)
    unsigned long long alpha_y_next_bits;
    double alpha_y;
    int64_t steps;
    int32_t done;
    int32_t status;
    int32_t last;
    uint32_t tiles_done;
    // shape-parameter decisions of the RBF schemes over the run (see EtaCount)
    unsigned long long n_switch, n_eval, n_guard, n_bound;
    int64_t step_cap;   // the run ends with NPW_ETIMEOUT after this many steps
};

// Step limit of a solve: the caller's max_steps, or 64 times the step count that the first
// time step implies plus 1024, at most 2^24.  A run that reaches it, or whose time stops
// advancing (t + dt == t), ends with NPW_ETIMEOUT instead of looping on the device.
__host__ __device__ __forceinline__ int64_t step_cap(double t_rem, double dt, int64_t max_steps) {
    if (max_steps > 0) return max_steps;
    const double est = dt > 0.0 ? t_rem / dt : 1.0;
    const double cap = 64.0 * (est < 1e12 ? est : 1e12) + 1024.0;
    return cap < 16777216.0 ? (int64_t)cap : (int64_t)16777216;
}

// Work item: (instance, first cell of the tile).
struct Tile {
    int32_t inst;
    int32_t start;
};

// 2D problem: one square/rectangle, tiles of TX x TY cells.
struct Inst2D {
    int64_t off;
    int64_t nx, ny;
    double dx, dy;
    double t_end, cfl;
    int32_t bc;      // boundary of the x direction (columns)
    int32_t tiles_x, tiles_y;
    int32_t bc_y;    // boundary of the y direction (rows)
};

struct Stage1DArgs {
    const void* uin;   // stage input u^(k)
    const void* un;    // u^n (stages 2, 3)
    void* uout;        // stage output
    // compensated float path (stage1d_fast_kernel): u^n in `u` (arena), increments d1 and d2,
    // the next state s (written by stage 3, copied into u by the next stage 1) and the carry c
    float* u;
    float* d1;
    float* d2;
    float* s;
    float* c;
    const InstDev* inst;
    Ctl* ctl;
    const Tile* tiles;
    int32_t ntiles;
    int32_t stage;     // 0, 1, 2
    int32_t advance;   // stage 2 finalises the step (time control on the device)
    int32_t tile;      // cells per tile
    MethodParams mp;
};

// Whole-solve kernel for instances that fit in one CTA's shared memory: every RK3 step of
// the instance runs inside the CTA, the state never leaves shared memory until t_end.
struct ResidentArgs {
    void* arena;             // state of all instances ([m][n] at inst.off), in/out
    float* carry;            // per-cell compensation of the step update (arena-shaped scratch)
    const InstDev* inst;
    Ctl* ctl;
    const int32_t* list;     // instance indices handled by this launch, one per CTA
    int32_t count;
    MethodParams mp;
};

struct Stage2DArgs {
    const void* uin;
    const void* un;
    void* uout;
    const Inst2D* inst;
    Ctl* ctl;
    int32_t stage;
    int32_t advance;
    MethodParams mp;
};

// Persistent work-queue stage kernel: the CTAs of one launch pull work items (instance, tile)
// from a device counter until the list is exhausted; 1D items are tiles of `tile` cells (start
// cell in Tile.start), 2D items tiles of TX_2D x TY_2D cells (tile index in Tile.start).  Every
// instance has its own descriptor, control word and step; items of finished instances return
// at once.  The last CTA to leave resets the counter for the next launch.
struct QueueArgs {
    void* u;                 // state of all instances (arena, element type of the run)
    void* u1;                // stage buffers (arena-shaped); the compensated 1D float items
    void* u2;                //   keep their increments d1, d2 there
    float* s;                // compensated 1D float items: next state and carry (arena-shaped)
    float* c;
    const InstDev* inst1;    // [count] 1D descriptor (used when !is2d)
    const Inst2D* inst2;     // [count] 2D descriptor (used when is2d)
    const int32_t* kind;     // [count] flux kind
    const uint8_t* is2d;     // [count]
    Ctl* ctl;                // [count]
    const Tile* items;
    int32_t nitems;
    int32_t stage;
    int32_t advance;
    int32_t tile;            // cells per 1D item
    int32_t parity;          // QUEUE_FUSED_STEP: 0 = u^n in u, u^{n+1} to s; 1 = the other way round
    unsigned int* head;      // [2]: next item, CTAs finished
    MethodParams mp;
};
// QueueArgs.stage of a whole RK3 step of compensated float 1D items in one launch
// (step1d_fused_body); stages 0..2 are the per-stage launches
constexpr int QUEUE_FUSED_STEP = 3;
// halo of a fused step (three stages, each reaching 3 cells) and its shared memory in floats:
// u^n, the stage input, d, eta, v^-, v^+ over tile + 18 cells per field
constexpr int FUSE_HALO = 9;
__host__ __device__ constexpr size_t fused1d_smem_floats(int tile, int m) { return (size_t)6 * (tile + 2 * FUSE_HALO) * m; }

// Instance shape of a queue batch whose instances all have one dimension and flux kind: the
// queue kernel instantiated for it carries only that body (and that body's register count);
// QS_ANY dispatches per item.
enum QueueShape { QS_ANY = 0, QS_1D_ADV, QS_1D_BURG, QS_1D_EULER, QS_2D_ADV, QS_2D_BURG, QS_2D_EULER };
inline int queue_shape_of(bool is2d, int kind) {
    return (is2d ? QS_2D_ADV : QS_1D_ADV) + (kind == NPW_FLUX_ADVECTION ? 0 : kind == NPW_FLUX_BURGERS ? 1 : 2);
}

// ---- launchers (one definition per precision translation unit) ---------------------------
template <typename R>
cudaError_t launch_reconstruct(const R* u, int64_t n, int m, int bc, const MethodParams& mp, R* vm, R* vp,
                               uint8_t* flags, R* eta, cudaStream_t s);
template <typename R>
cudaError_t launch_flux(const R* vm, const R* vp, int64_t nf, int m, int kind, double alpha,
                        const MethodParams& mp, R* h, cudaStream_t s);
template <typename R>
cudaError_t launch_alpha_init(const void* u, const InstDev* inst, Ctl* ctl, const Tile* tiles, int ntiles,
                              int tile, int m, int kind, const MethodParams& mp, cudaStream_t s);
template <typename R>
cudaError_t launch_stage1d(const Stage1DArgs& a, int m, int kind, cudaStream_t s);
template <typename R>
cudaError_t launch_alpha_init_2d(const void* u, const Inst2D* inst, int tiles, Ctl* ctl, int kind,
                                 const MethodParams& mp, cudaStream_t s);
template <typename R>
cudaError_t launch_stage2d(const Stage2DArgs& a, int tiles, int kind, cudaStream_t s);
// queue kernels: smem_bytes for the instance kinds present (see queue_smem_bytes); blocks = 0
// asks for one wave of resident CTAs (occupancy x SMs)
// shape: a QueueShape that every instance of the batch has, or QS_ANY
template <typename R>
cudaError_t launch_queue_stage(const QueueArgs& q, bool characteristic, int shape, size_t smem_bytes, int blocks,
                               cudaStream_t s);
template <typename R>
cudaError_t launch_queue_alpha(const QueueArgs& q, cudaStream_t s);
template <typename R>
size_t queue_smem_bytes(int tile, bool has1d, int m1d, bool has2d, int m2d, bool characteristic);
// resident whole-solve launch (float state only); max_n = largest n in the list
cudaError_t launch_resident_f32(const ResidentArgs& a, int m, int kind, int64_t max_n, int threads, cudaStream_t s);
size_t resident_smem_bytes(int64_t n, int m);

// records msg as the calling thread's npw_last_error() text and returns st (npw_api.cu)
npw_status set_error(npw_status st, const char* msg);

// precision-independent helpers (npw_api.cu)
cudaError_t launch_queue_ctl(Ctl* ctl, const InstDev* inst1, const Inst2D* inst2, const uint8_t* is2d,
                             const int32_t* list, int count, int mode, int64_t max_steps, cudaStream_t s);
cudaError_t launch_queue_poll(const Ctl* ctl, const InstDev* inst1, const Inst2D* inst2, const uint8_t* is2d,
                              int count, long long* poll, cudaStream_t s);
// compensated float path: before the first step s = u and c = 0; after the last, u = s (odd:
// only for the instances whose control word counts an odd number of steps, NULL = all)
cudaError_t launch_comp_begin(const float* u, float* s, float* c, const InstDev* inst, const Tile* tiles, int ntiles,
                              int tile, int m, cudaStream_t st);
cudaError_t launch_comp_end(float* u, const float* s, const InstDev* inst, const Tile* tiles, int ntiles, int tile,
                            int m, const Ctl* odd, cudaStream_t st);
// fills [m][n] with smooth data for the tile autotuner (m = 3: a quiet Euler state)
template <typename R>
cudaError_t launch_tune_init(R* u, int64_t n, int m, cudaStream_t st);

constexpr int TILE_1D = 1024;     // default cells per CTA tile in the 1D stage kernels
constexpr int TILE_1D_MIN = 256;  // smallest tile a run may choose (sizes the tile tables)
constexpr int RES_GHOST = 3;       // ghost cells on each side of the resident kernel's state arrays
constexpr size_t RESIDENT_SMEM_MAX = 200 * 1024;  // shared memory a resident CTA may use
constexpr int THREADS_1D = 256;
constexpr int TX_2D = 32;      // 2D tile
constexpr int TY_2D = 8;

}  // namespace npw
