/*
 * npweno.h -- C ABI of the GB300 (sm_103a) library for the non-polynomial (RBF-perturbed)
 * ENO3 / WENO5 finite-volume method of Guo & Jung, arXiv 1602.00182.
 *
 * The method (paper Sec. 2-5): cell averages vbar_i on a uniform grid are reconstructed to
 * the two one-sided values v^-_{i+1/2}, v^+_{i-1/2} at every face by the polynomial ENO3 or
 * WENO5 coefficients perturbed by an RBF shape parameter eta = eps^2 dx^2 (Table k3; the
 * multiquadric rows are printed, the Gaussian rows follow Sec. 3.3's recipe).  eta is set per
 * face by the optimisation condition of Table k3 and forced to 0 by the monotone-polynomial
 * switch of Sec. 4 (eq. adaptation).  The face values feed the Lax-Friedrichs flux, the
 * conservative difference of eq. PDE1 and the TVD Runge-Kutta 3 update (Sec. 5.1).
 *
 * Conventions shared by every entry point:
 *   - Array pointers are DEVICE pointers owned by the caller unless stated otherwise.
 *     Element type: double when params->precision == NPW_FP64, float when NPW_FP32_MIXED.
 *   - 1D fields are laid out field-major, [m][n] contiguous; 2D fields are [m][ny][nx].
 *     Face arrays are [m][n+1]: face f lies between cell f-1 and cell f (faces 1/2 .. n+1/2
 *     of the paper, shifted to start at 0).
 *   - The library allocates no device memory.  Entry points that need scratch take a
 *     caller-owned device `workspace` of at least the size returned by the matching
 *     npw_*_workspace_size() call; its contents on entry are ignored.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream except where a result must reach the host (the solve
 *     calls poll a 4-byte completion word between launches and return when done).
 *   - Errors are returned as npw_status and never abort; npw_last_error() gives the text
 *     of the most recent failure on the calling thread.
 *   - n >= 6 cells (3 ghost cells per side feed the WENO5 stencil); dx > 0; k is 2 or 3.
 */
#ifndef NPWENO_H
#define NPWENO_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NPW_OK = 0,
    NPW_EINVAL = -1,      /* bad argument (size, enum, null pointer, workspace too small) */
    NPW_ENOMEM = -2,      /* reserved: the library itself never allocates */
    NPW_ECUDA = -3,       /* a CUDA runtime call failed; see npw_last_error() */
    NPW_ETIMEOUT = -4,    /* a bounded wait ran out */
    NPW_ENONFINITE = -5,  /* the state became non-finite (per instance in batch mode) */
    NPW_EBUSY = -6        /* server: request does not fit the memory budget now */
} npw_status;

/* Flux functions of the paper's examples: f = a u (Sec. 5.2 Ex. 1, 2), f = u^2/2 (Ex. 3),
 * 1D Euler (Ex. 4, m = 3), 2D Euler (Sec. 7 form, m = 4). */
typedef enum { NPW_FLUX_ADVECTION = 0, NPW_FLUX_BURGERS = 1, NPW_FLUX_EULER1D = 2, NPW_FLUX_EULER2D = 3 } npw_flux_kind;
/* Boundary conditions: periodic (Ex. 1, 3), transmissive = zero-gradient ghost cells
 * (Ex. 4), inflow = constant left ghost state params->inflow (Ex. 2), right transmissive.
 * 2D: bc applies to x and, unless params->bc_y >= 0, to y (inflow: bottom side, top transmissive). */
typedef enum { NPW_BC_PERIODIC = 0, NPW_BC_TRANSMISSIVE = 1, NPW_BC_INFLOW = 2 } npw_bc;
/* Schemes compared in the paper (Sec. 5.2): ENO3, WENO-JS5 (eta = 0), RBF-ENO3, RBF-WENO5. */
typedef enum { NPW_ENO = 0, NPW_WENO_JS = 1, NPW_RBF_ENO = 2, NPW_RBF_WENO = 3 } npw_scheme;
typedef enum { NPW_RBF_MQ = 0, NPW_RBF_GA = 1 } npw_rbf;
/* NPW_FP64: everything in double.  NPW_FP32_MIXED: float state, candidates, WENO weights and
 * smoothness indicators, flux and update; the shape parameter eta is evaluated from exact
 * differences in extended precision (see eta_eval), and the monotone-switch and ENO decisions
 * are those of FP64 evaluation (taken from
 * float values with a certified error bound, recomputed in double when the bound does not
 * decide them). */
typedef enum { NPW_FP64 = 0, NPW_FP32_MIXED = 1 } npw_precision;

typedef struct {
    int32_t k;               /* 3: ENO3 / WENO5 (Table k3); 2: ENO2 / WENO3 (Table k2, Sec. 3.2-3.5: one
                                shape parameter per face value, from the cell's 3-cell stencil,
                                and the switch of eq. root_value per cell; switch_variant unused) */
    int32_t scheme;          /* npw_scheme */
    int32_t rbf;             /* npw_rbf: perturbation rows of Table k3 (MQ) or Sec. 3.3 (GA) */
    int32_t monotone_switch; /* 1: eta = 0 where the stencil polynomial is non-monotone */
    int32_t switch_variant;  /* 0: cubic on the 4-cell eta stencil; 1: eq. root_value on both 3-cell halves */
    int32_t characteristic;  /* 1D Euler only: reconstruct Roe characteristic fields */
    int32_t precision;       /* npw_precision */
    int32_t eta_eval;        /* NPW_FP32_MIXED, k = 3: 0 = eta from the exact differences a = w0 - w3,
                                b = w2 - w1 held as float pairs, double-float quotient (no FP64
                                instruction; within one float ulp plus ~2^-44 of the conditioning
                                (|a| + 3|b|) / |num| + (|a| + 15|b|) / |den|); 1 = in FP64 (numerator
                                and denominator from the widened averages by FP64 differences and
                                multiply-adds, Newton quotient; within half an ulp plus 2^-52 of the
                                conditioning).  k = 2 always takes the FP64 form. */
    double eps_M;            /* additive guard of the eta denominator (Table k3), e.g. 1e-12 */
    double eps_weno;         /* WENO epsilon of Sec. 2, 1e-6 */
    double gamma;            /* ratio of specific heats, 1.4 */
    double adv_speed;        /* advection speed a (x) for NPW_FLUX_ADVECTION */
    double adv_speed_y;      /* advection speed (y) for 2D advection */
    double inflow[4];        /* ghost state of NPW_BC_INFLOW (conserved variables) */
    double eta_guard;        /* eta = 0 where |den| <= eta_guard * (|w0| + 15|w1| + 15|w2| + |w3|), i.e.
                                where the eta denominator is below the round-off of its cell averages;
                                0 = automatic (off for NPW_FP64, 8 * 2^-24 for NPW_FP32_MIXED), < 0 = off */
    int32_t batch_mode;      /* npweno_batch_solve, NPW_FP32_MIXED: 0 = instances whose state fits in one
                                CTA's shared memory run whole in one CTA (resident), the rest through the
                                per-stage kernels; 1 = every instance through the per-stage kernels */
    int32_t tile_1d;         /* cells per CTA of the 1D per-stage kernels: 256, 512, 1024 or 2048; 0 = the
                                value npw_autotune_1d chose for this flux kind, m, k, precision and
                                characteristic flag on this device, else 1024.  Results do not depend on
                                it (each face gets the same arithmetic in any tiling) */
    double eta_max;          /* optional bound, not in the paper: eta = 0 where |eta| > eta_max.  The printed eta
                                (Table k3, Table k2) is singular where its denominator crosses zero (a monotone
                                stencil with zero slope at the face for k = 3, v ~ 0 at the face for k = 2), and
                                the perturbation argument of Sec. 3 assumes a small eta.  <= 0 (the default) = off:
                                the shape parameter exactly as printed.  Faces it zeroes are counted in
                                npw_solve_stats.eta_bound and flagged by npweno_reconstruct */
    int32_t cross_2d;        /* 2D runs with k = 2 and an RBF scheme: 1 = the shape parameter of Sec. 6 on the
                                5-cell cross, which also cancels the transverse curvature of the cell averages
                                at the face midpoint (third-order face values); 0 = the line form of Table k2 */
    int32_t bc_y;            /* 2D entry points: boundary condition of the y direction (rows), NPW_BC_*; < 0
                                (npw_default_params: -1) = the bc argument, which then applies to both
                                directions and otherwise to x only.  An inflow side (left for x, bottom
                                for y) holds params.inflow; 1D entry points ignore it */
    double tie_tol;          /* npweno_reconstruct: relative margin of the near-tie flag bit (a switch, ENO,
                                guard or bound decision whose deciding quantity lies within tie_tol of its
                                threshold); <= 0 = 1e-10 */
    int64_t max_steps;       /* step limit of every solve (npweno_solve, _solve_2d, _batch_solve, the server):
                                a run that reaches it, or whose time stops advancing (t + dt == t), ends
                                with status NPW_ETIMEOUT instead of looping on the device; <= 0 = automatic:
                                64 x the step count the first time step implies + 1024, at most 2^24 */
    int32_t gauss_2d;        /* 2D entry points, k = 2 (RBF schemes: with cross_2d): 1 = the integral
                                of eq. 2DIntegral by two Gauss points per face (Sec. 7 names two points as
                                needed for third order): the reconstruction of Sec. 6 at -+ 1/(2 sqrt 3) cell
                                widths from the face midpoint, its Taylor error there cancelled by the shape
                                parameter (the v_xy term with the diagonal neighbour), and the mean of the two
                                Lax-Friedrichs fluxes; 0 = one point at the midpoint, as in the paper's runs.
                                NPW_FP32_MIXED: float state, candidates, weights, flux and update, the shape
                                parameters, switch, ENO choices and smoothness indicators in double from the
                                float averages (npweno_rk3_step_2d / npweno_solve_2d; the work queue and the
                                server take it in NPW_FP64 only, else NPW_EINVAL) */
    int32_t reserved_;       /* 0 */
} npw_params;

typedef struct {
    int64_t steps;    /* RK3 steps taken */
    double t;         /* time reached (== t_end on success) */
    double alpha_max; /* largest Lax-Friedrichs alpha seen */
    int32_t status;   /* npw_status of this problem */
    int32_t pad_;
    /* Shape-parameter decisions of the RBF schemes over the run, every stage of every step:
     * per face and field for k = 3, per face value (v^- and v^+ of a face) for k = 2.  A line of
     * n cells has n + 1 faces per stage (a 2D grid: rows x (nx + 1) + columns x (ny + 1)).
     * eta_switch: the monotone switch (Sec. 4) set eta = 0; eta_eval: eta was evaluated; of
     * those, eta_guard / eta_bound were set to 0 by the round-off guard / the optional bound.
     * All four are 0 for ENO and WENO-JS. */
    int64_t eta_switch, eta_eval, eta_guard, eta_bound;
} npw_solve_stats;

/* One problem of a batch: a 1D field set of n cells at element `offset` of the arena,
 * [m][n] contiguous.  The time step of each instance is its own. */
typedef struct {
    int64_t offset;  /* element offset of the instance in the arena */
    int64_t n;       /* cells */
    double dx;       /* cell width */
    double t_end;    /* final time */
    double cfl;      /* dt = cfl * dx / alpha^n */
    int32_t bc;      /* npw_bc */
    int32_t pad_;
} npw_instance;

/* Fill *p with the defaults: k = 3, RBF-WENO5, multiquadric, switch on (variant 0),
 * component-wise, FP64, eps_M = 1e-12, eps_weno = 1e-6, gamma = 1.4, a = (1, 1),
 * eta_eval = 0, eta_guard = 0 (automatic), eta_max = 0 (no bound), tie_tol = 0 (1e-10). */
void npw_default_params(npw_params* p);

/* Text of the last error on the calling thread ("" if none). */
const char* npw_last_error(void);

/* ABI version (major*10000 + minor*100 + patch). */
int32_t npw_version(void);

/*
 * Reconstruction only (paper Sec. 2 and 3.5, eq. weno_re, Table k3 / Table k2, Sec. 4 eq.
 * adaptation): for each of the n+1 faces, the left/right states v^-, v^+ of every field.
 *   vbar    [m][n] cell averages (device)
 *   v_minus [m][n+1] out: v^-_f from cell f-1;  v_plus [m][n+1] out: v^+_f from cell f
 *   flags   [m][n+1] out, may be NULL.  k = 3: bit0 = monotone switch fired (eta set to 0),
 *           bits 2-3 = ENO stencil r of cell f-1, bits 4-5 = ENO stencil r of cell f.
 *           k = 2: bit0 / bit3 = switch fired for cell f-1 / cell f, bit2 / bit4 = ENO
 *           stencil r (0 or 1) of cell f-1 / cell f.
 *           Both: bit1 = near tie (a decision at the face within params->tie_tol of its
 *           threshold, where another correct rounding order may decide otherwise); bit6 /
 *           bit7 = an evaluated eta set to 0 by the guard / the bound (k = 2: of either face
 *           value).  Characteristic runs: per characteristic field.
 *   eta     [m][n+1] out, may be NULL: the shape parameter used at each face (k = 2: that of
 *           v^-_f, the central row), after the switch, guard and bound; state element type.
 * m = 1, or m = 3 with params->characteristic for the 1D Euler characteristic fields.
 * Returns NPW_EINVAL for n < 6, m outside 1..4, characteristic with m != 3, null pointers.
 */
npw_status npweno_reconstruct(const void* vbar, int64_t n, int32_t m, int32_t bc, const npw_params* params,
                              void* v_minus, void* v_plus, uint8_t* flags, void* eta, void* stream);

/*
 * Lax-Friedrichs numerical flux (Sec. 5.1): h = (f(v^-) + f(v^+) - alpha (v^+ - v^-)) / 2
 * for every face and field.  v_minus, v_plus, h are [m][nfaces] (device); m must match the
 * flux kind (1, 3 for 1D Euler); alpha >= 0 is the constant of Sec. 5.1.
 */
npw_status npweno_flux(const void* v_minus, const void* v_plus, int64_t nfaces, int32_t m, int32_t flux_kind,
                       double alpha, const npw_params* params, void* h, void* stream);

/* Bytes of device workspace npweno_rk3_step / npweno_solve need for n cells, m fields. */
size_t npw_workspace_size(int64_t n, int32_t m, const npw_params* params);

/*
 * One TVD-RK3 step (Sec. 5.1, Shu-Osher form) of u [m][n] (device, in/out) with the given
 * dt.  alpha of the Lax-Friedrichs flux is max_i |f'(u_i^n)| over the field, frozen over the
 * three stages.  Each stage is one fused kernel: halo load, shape parameter, switch,
 * candidates, weights, flux, flux difference (eq. PDE1) and the stage combination.
 * If alpha_out is not NULL the alpha used is written there (host double; the call then
 * synchronises the stream).
 */
npw_status npweno_rk3_step(void* u, int64_t n, int32_t m, double dx, double dt, int32_t flux_kind, int32_t bc,
                           const npw_params* params, void* workspace, size_t workspace_bytes, double* alpha_out,
                           void* stream);

/*
 * Advance u [m][n] (device, in/out) from t = 0 to t_end with dt = cfl * dx / alpha^n, alpha^n
 * = max_i |f'(u_i^n)| (Sec. 5.1 with the CFL rule of Sec. 5.2); the step that reaches t_end to
 * within 1e-10 of a step is shortened to end exactly at t_end.  Time control runs on the
 * device; the host polls a completion word between launches.  out (host) may be NULL.
 * Returns NPW_ENONFINITE if the state stops being finite.
 */
npw_status npweno_solve(void* u, int64_t n, int32_t m, double dx, double t_end, double cfl, int32_t flux_kind,
                        int32_t bc, const npw_params* params, void* workspace, size_t workspace_bytes,
                        npw_solve_stats* out, void* stream);

/*
 * Many independent 1D problems in one arena (device), advanced together by the same fused
 * stage kernels over a work list of (instance, tile) pairs; each instance keeps its own t,
 * dt and alpha on the device and drops out of the work when it reaches its t_end.  In
 * NPW_FP32_MIXED (batch_mode 0, component-wise) an instance whose state fits in one CTA's
 * shared memory (n up to about 10000 for m = 1, 3400 for m = 3) is instead solved whole by one
 * CTA: all its RK3 steps run in shared memory and only the initial and final states cross HBM;
 * those CTAs run on library-owned side streams concurrently with the per-stage work and the
 * call returns when both are done.
 * inst (host, count entries) describes the instances; out (host, count entries, may be
 * NULL) receives per-instance statistics.  The returned status is NPW_OK when every
 * instance finished; otherwise the first failing instance's status.
 */
size_t npw_batch_workspace_size(const npw_instance* inst, int32_t count, int32_t m, const npw_params* params);
npw_status npweno_batch_solve(void* arena, const npw_instance* inst, int32_t count, int32_t m, int32_t flux_kind,
                              const npw_params* params, void* workspace, size_t workspace_bytes,
                              npw_solve_stats* out, void* stream);

/*
 * 2D dimension-by-dimension form (Sec. 7, eq. 2DIntegral with one midpoint quadrature point
 * per face): the x faces are reconstructed along grid rows and the y faces along columns;
 * L = -(h^x_{i+1/2,j} - h^x_{i-1/2,j})/dx - (h^y_{i,j+1/2} - h^y_{i,j-1/2})/dy; one fused
 * kernel per stage.  u is [m][ny][nx] (device); m = 4 for NPW_FLUX_EULER2D, m = 1 for scalar
 * advection / Burgers.  dt of npweno_solve_2d = cfl / (alpha_x/dx + alpha_y/dy).
 */
size_t npw_workspace_size_2d(int64_t nx, int64_t ny, int32_t m, const npw_params* params);
npw_status npweno_rk3_step_2d(void* u, int64_t nx, int64_t ny, int32_t m, double dx, double dy, double dt,
                              int32_t flux_kind, int32_t bc, const npw_params* params, void* workspace,
                              size_t workspace_bytes, void* stream);
npw_status npweno_solve_2d(void* u, int64_t nx, int64_t ny, int32_t m, double dx, double dy, double t_end,
                           double cfl, int32_t flux_kind, int32_t bc, const npw_params* params, void* workspace,
                           size_t workspace_bytes, npw_solve_stats* out, void* stream);

/*
 * Work-queue batch: uneven 1D and 2D instances of any flux kind (the batching pattern around
 * the method; the paper has no counterpart) advanced together, each with its own dt, alpha,
 * t_end and step count.  Every RK3 stage is one launch of a persistent kernel whose CTAs take
 * (instance, tile) work items from a device counter until none is left -- 1D tiles of
 * params->tile_1d cells (0: the autotuned or default size), 2D tiles of 32 x 8 cells -- and run
 * the per-stage body of that instance's kind (the same arithmetic as npweno_batch_solve and
 * npweno_solve_2d, so the same bits); steps are replayed as CUDA graphs between bounded polls.
 * NPW_FP32_MIXED component-wise runs solve 1D instances that fit in shared memory whole in one
 * CTA (the resident kernel, batch_mode 0) beside the queue; when the queued instances are all
 * 1D, each RK3 step is a single launch (u^n loaded once per tile with a 9-cell halo, the three
 * stages in shared memory, the same bits as the per-stage launches; tile_1d 0 then takes at most
 * the tile whose 44 KB of shared memory leaves 5 CTAs per SM).  A batch whose instances share one
 * dimension and flux kind runs a kernel compiled for that shape.  Characteristic runs take 1D
 * Euler instances only.
 *   arena: device, the instances' fields ([m][n] or [m][ny][nx] at `offset`, element type of
 *          params->precision); in/out.
 *   inst:  host, count descriptors (ny = 0 for a 1D instance; m follows the flux kind).
 *   out:   host, count statistics (may be NULL).
 * Returns NPW_OK when every instance finished, else the first failing instance's status.
 */
typedef struct {
    int64_t offset;    /* element offset of the instance in the arena */
    int64_t nx;        /* cells (1D) or cells per row (2D) */
    int64_t ny;        /* 0: a 1D instance; >= 6: rows of a 2D instance */
    double dx, dy;     /* cell sizes (dy: 2D only) */
    double t_end, cfl; /* dt = cfl dx / alpha (1D), cfl / (alpha_x / dx + alpha_y / dy) (2D) */
    int32_t flux_kind; /* 1D: NPW_FLUX_ADVECTION, _BURGERS, _EULER1D; 2D: _ADVECTION, _BURGERS, _EULER2D */
    int32_t bc;        /* npw_bc (2D: of x) */
    int32_t bc_y;      /* 2D: npw_bc of y; < 0: bc */
    int32_t pad_;
} npw_queue_instance;
size_t npw_queue_workspace_size(const npw_queue_instance* inst, int32_t count, const npw_params* params);
npw_status npweno_queue_solve(void* arena, const npw_queue_instance* inst, int32_t count, const npw_params* params,
                              void* workspace, size_t workspace_bytes, npw_solve_stats* out, void* stream);

/*
 * Request server: continuous batching of 1D and 2D solves (no counterpart in the paper; the
 * serving loop around the method).  Requests are queued by npw_server_submit (non-blocking) and
 * admitted first-in first-out whenever a slot and heap space are free.  Each request carries its
 * own end time and tolerance; the tolerance picks its precision lane: NPW_FP32_MIXED for a
 * tolerance >= 1e-4 (the mixed path's stated L1 class), NPW_FP64 below (0: the server's
 * params->precision).  Each lane runs rounds on its own stream (the mixed lane on `stream`, the
 * FP64 lane on a stream of the server's), independently of the other lane: a round advances
 * every admitted request of the lane -- each with its own dt, alpha, step count and t_end -- by
 * an even number of RK3 steps (max_steps rounded down to even, at least 2) through the work-
 * queue kernel, with the requests grouped by instance shape (1D or 2D, flux kind), each group on
 * a stream of its own with the kernel specialised for that shape (per stage one persistent
 * launch over the group's work items; the mixed lane's 1D requests take one launch per fused
 * RK3 step; the mixed lane's groups at the greatest stream priority, so that its short launches
 * start first as the FP64 lane's CTAs retire).  npw_server_step retires every lane whose round
 * has ended (copies finished states to their host buffers, frees their space), admits that
 * lane's queued requests and launches its next round; when no round has ended yet it waits for
 * the first that does, at most 5 ms, and returns (a round in flight longer than the wait limit
 * NPW_WAIT_TIMEOUT_S gives NPW_ETIMEOUT).  Each
 * request's arithmetic depends only on its own data, so its result is the same bits alone or in
 * any mix (and equal to npweno_batch_solve with batch_mode 1 or npweno_solve_2d of the same
 * request in its lane's precision).
 *   device_arena / arena_bytes: caller-owned device memory, at least
 *       npw_server_arena_bytes(heap_cells, max_slots, params): a heap of heap_cells elements per
 *       lane (a request occupies m * n, 2D m * n * ny, heap cells of its lane).
 *   params: method of every request; params->precision is the lane of requests with tolerance 0.
 *   stream: cudaStream_t (void*) of the mixed lane and of creation; npw_server_destroy waits
 *       (bounded) for both lanes' rounds before it returns.
 * Host buffers of a request (u0_host read at admission, out_host written at completion, both
 * [m][n] ([m][ny][nx]) of its lane's element type: float for the mixed lane, double for FP64)
 * must stay valid until its result has been polled.  Timestamps are seconds since
 * npw_server_create.  Not thread-safe: one thread drives a server.
 */
typedef struct npw_server npw_server;
typedef struct {
    int32_t flux_kind;     /* 1D (ny == 0): NPW_FLUX_ADVECTION, NPW_FLUX_BURGERS or NPW_FLUX_EULER1D;
                              2D (ny > 0): NPW_FLUX_ADVECTION, NPW_FLUX_BURGERS or NPW_FLUX_EULER2D */
    int32_t bc;            /* npw_bc (2D: of the x direction) */
    int64_t n;             /* cells (2D: nx); m = 1, 3 for 1D Euler, 4 for 2D Euler */
    double dx;
    double t_end;
    double cfl;
    const void* u0_host;   /* initial cell averages, host: [m][n] (2D: [m][ny][nx]) */
    void* out_host;        /* final state, host, same layout */
    uint64_t tag;          /* returned with the result */
    int64_t ny;            /* 0: a 1D request; >= 6: a 2D request of n x ny cells (dimension by dimension) */
    double dy;             /* 2D: cell size in y */
    int32_t bc_y;          /* 2D: npw_bc of the y direction; < 0: bc */
    int32_t reserved_;
    double tolerance;      /* 0: the server's precision; >= 1e-4: NPW_FP32_MIXED; below: NPW_FP64 */
} npw_request;
typedef struct {
    uint64_t id;           /* as returned by npw_server_submit */
    uint64_t tag;
    int32_t status;        /* npw_status of this request */
    int32_t precision;     /* the lane it ran in: NPW_FP32_MIXED or NPW_FP64 */
    int64_t steps;
    double t;
    double submit_s;       /* when submitted */
    double admit_s;        /* when its state reached the device */
    double done_s;         /* when its final state reached out_host */
} npw_result;
size_t npw_server_arena_bytes(int64_t heap_cells, int32_t max_slots, const npw_params* params);
npw_status npw_server_create(void* device_arena, size_t arena_bytes, int32_t max_slots, const npw_params* params,
                             void* stream, npw_server** out);
/* Queue a request.  NPW_EINVAL for a malformed request or one larger than the whole heap;
 * NPW_EBUSY when max_slots requests are already waiting. */
npw_status npw_server_submit(npw_server* s, const npw_request* req, uint64_t* id);
/* Retire the lanes whose rounds have ended (waiting up to 5 ms for one if none has), admit their
 * queued requests and launch their next rounds of max_steps steps (rounded down to even, at least
 * 2).  *active / *queued (may be NULL) receive the admitted and the queued request counts. */
npw_status npw_server_step(npw_server* s, int32_t max_steps, int32_t* active, int32_t* queued);
/* Completed results, oldest first; *nout <= max. */
npw_status npw_server_poll(npw_server* s, npw_result* out, int32_t max, int32_t* nout);
void npw_server_destroy(npw_server* s);

/*
 * Tile autotuner for the 1D per-stage kernels (the batching pattern's autotuned tile shape).
 * Times TVD-RK3 steps of a 2^21-cell periodic instance of smooth synthetic data (a quiet
 * Euler state for m = 3) with each tile size 256, 512, 1024, 2048 cells per CTA, keeps the
 * fastest in a process-wide table keyed by device, flux kind, m, k, precision and
 * characteristic flag, and returns it.  Later runs with params->tile_1d = 0 use it.
 *   scratch: caller-owned device memory of at least npw_autotune_scratch_bytes(m, params)
 *            bytes (its contents are overwritten).
 *   stream:  cudaStream_t (void*); the call synchronises with it (bounded wait).
 * Returns NPW_EINVAL for bad arguments or a small scratch, NPW_ECUDA / NPW_ETIMEOUT on device
 * errors (the table is then unchanged).
 */
size_t npw_autotune_scratch_bytes(int32_t m, const npw_params* params);
npw_status npw_autotune_1d(int32_t flux_kind, int32_t m, const npw_params* params, void* scratch,
                           size_t scratch_bytes, void* stream, int32_t* best_tile);

/*
 * npweno_rk3_step_noalloc -- the same TVD-RK3 step as npweno_rk3_step (identical kernels and
 * results), for callers that cannot allocate device memory.  The paper has no counterpart:
 * this is an interface for embedding.  Some callers own only device pointers to their state
 * and cannot obtain more device memory where they call the solver -- a host framework that
 * places every buffer itself and keeps the rest of the GPU in its own pool, or a job confined
 * to a fixed share of GPU memory where a late allocation could fail.  This entry point takes no
 * workspace: its scratch is one fixed 8 MiB array inside the library, placed on every GPU
 * that loads the library and kept there until the process exits.
 *   - Allocates no device memory (no cudaMalloc, cudaFree or allocating library call).
 *   - Limit: npw_workspace_size(n, m, params) must not exceed npw_noalloc_scratch_bytes()
 *     (8 MiB: n * m up to about 5.2e5 cells in either precision -- two 8-byte stage buffers in
 *     NPW_FP64, four 4-byte arrays in NPW_FP32_MIXED); larger sizes return NPW_EINVAL with an
 *     explanatory npw_last_error().
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 *     with that device current) and caches it; make that first call before any stream capture.
 *   - Every call on a device uses the same array and the array keeps the last call's contents
 *     (each call re-initialises what it reads), so calls that overlap on the GPU -- on
 *     different streams or host threads at the same time -- race and must be serialised.
 *   - The cached address does not survive cudaDeviceReset: after a reset in the same process
 *     this entry point must not be called again on that device.
 *   - u, n, m, dx, dt, flux_kind, bc, params and stream have the meaning of npweno_rk3_step.
 */
npw_status npweno_rk3_step_noalloc(void* u, int64_t n, int32_t m, double dx, double dt, int32_t flux_kind,
                                   int32_t bc, const npw_params* params, void* stream);
/* Size in bytes of the fixed scratch array used by npweno_rk3_step_noalloc. */
size_t npw_noalloc_scratch_bytes(void);

/*
 * npw_format_check -- self-check of the integer float<->double format changes that the
 * mixed-precision shape parameter uses instead of hardware conversions (no counterpart in the
 * paper).  For i < count it writes, from the device arrays f_in[count] (float) and
 * d_in[count] (double):
 *   widen_out[i]   the exact widening of f_in[i] by integer operations (every float class);
 *   widen_nz_out[i] the fast widening, meaningful where f_in[i] is zero or normal;
 *   narrow_out[i]  d_in[i] rounded to float by integer operations (round to nearest, ties away
 *                  from zero; below 2^-126 in magnitude: signed zero; beyond the float range:
 *                  signed infinity; d_in finite);
 *   seed_out[i]    d_in[i] truncated to float for a reciprocal seed;
 *   flags_out[i]   bit 0: f_in[i] is zero or normal; bit 1: d_in[i] is in the seed range
 *                  [2^-99, 2^99) in magnitude;
 *   hw_widen_out[i], hw_narrow_out[i]  the hardware conversions (double)f_in[i] and
 *                  (float)d_in[i], for comparison.
 * All pointers are device pointers of the stated lengths, owned by the caller; stream is a
 * cudaStream_t (NULL: the legacy default stream).  Returns NPW_EINVAL for count < 0 or a null
 * pointer with count > 0, NPW_ECUDA on a launch error; it does not synchronise.
 */
npw_status npw_format_check(const float* f_in, const double* d_in, int64_t count, double* widen_out,
                            double* widen_nz_out, float* narrow_out, float* seed_out, int32_t* flags_out,
                            double* hw_widen_out, float* hw_narrow_out, void* stream);

/*
 * Process-wide launch counters and stage-kernel timing (no counterpart in the paper; used to
 * put each kernel against its roofline).  When enabled, every launch of the fused stage
 * kernel is bracketed by two CUDA events recorded on the launching stream; the elapsed times
 * are summed at the next point where the runtime waits for its stream.  Counters are
 * cumulative until npw_profile_reset().
 */
typedef struct {
    int64_t kernel_launches; /* every kernel this library launched */
    int64_t stage_launches;  /* launches of the fused stage kernel (1D and 2D) */
    double stage_ms;         /* summed device time of the timed stage launches (enabled only) */
    int64_t timed_launches;  /* stage launches that were timed */
    int64_t resident_launches[4]; /* resident whole-solve launches per size class (n > 4096,
                                     > 2048, > 1024, <= 1024) */
    double resident_ms[4];   /* their summed device time (enabled only; the classes overlap) */
} npw_profile;
void npw_profile_enable(int32_t on);
void npw_profile_reset(void);
void npw_profile_read(npw_profile* out);

#ifdef __cplusplus
}
#endif
#endif /* NPWENO_H */
