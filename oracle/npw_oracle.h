/*
 * npw_oracle.h -- interface of the FP64 CPU oracle (test infrastructure only; see
 * npw_oracle.c).  Private to oracle/: the CUDA library neither includes nor links it.
 *
 * Layouts: 1D fields are [m][n] (field-major); face arrays are [m][n+1] with face f
 * between cell f-1 and cell f; 2D fields are [m][ny][nx].
 */
#ifndef NPW_ORACLE_H
#define NPW_ORACLE_H
#include <stdint.h>

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ENONFINITE = -5 };
enum { ORC_ENO = 0, ORC_WENO_JS = 1, ORC_RBF_ENO = 2, ORC_RBF_WENO = 3 };
enum { ORC_RBF_MQ = 0, ORC_RBF_GA = 1 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_TRANSMISSIVE = 1, ORC_BC_INFLOW = 2 };
enum { ORC_FLUX_ADVECTION = 0, ORC_FLUX_BURGERS = 1, ORC_FLUX_EULER1D = 2, ORC_FLUX_EULER2D = 3 };

/* per-face flag byte */
#define ORC_FLAG_SWITCH 0x01     /* monotone switch fired: eta forced to 0 */
#define ORC_FLAG_SWITCH_TIE 0x02 /* a switch quantity lies within tie_tol of its threshold */
/* bits 2-3: ENO stencil r of the left cell (for v^-); bits 4-5: of the right cell (v^+) */
#define ORC_FLAG_ENO_TIE_L 0x40
#define ORC_FLAG_ENO_TIE_R 0x80
/* k = 2: the switch belongs to a cell (its 3-cell stencil), so a face has two: bit 0 is the
 * switch of the left cell (v^-), bit 3 that of the right cell (v^+); bit 2 / bit 4 hold the
 * ENO stencil r (0 or 1) of the left / right cell; bit 1 marks a near tie of either switch. */
#define ORC_FLAG_SWITCH_R_K2 0x08

/* per-face "zero reason" byte of orc_reconstruct: an evaluated shape parameter set to 0 by the
 * optional guard or bound (neither is in the paper; both are off by default).  k = 3 has one
 * eta per face (the _L bits); k = 2 has one per face value: _L for v^- (the left cell), _R for
 * v^+ (the right cell). */
#define ORC_ZERO_GUARD_L 0x01
#define ORC_ZERO_BOUND_L 0x02
#define ORC_ZERO_GUARD_R 0x04
#define ORC_ZERO_BOUND_R 0x08

/* orc_params.counters[ORC_NCOUNTERS] (optional): shape-parameter decisions, per face (k = 3)
 * or per face value (k = 2), accumulated over every reconstruction that sees the params */
enum { ORC_CNT_SWITCH = 0, ORC_CNT_EVAL = 1, ORC_CNT_GUARD = 2, ORC_CNT_BOUND = 3, ORC_NCOUNTERS = 4 };

typedef struct {
    int scheme;          /* ORC_ENO .. ORC_RBF_WENO */
    int rbf;             /* ORC_RBF_MQ / ORC_RBF_GA */
    int monotone_switch; /* 0/1 */
    int switch_variant;  /* 0: cubic on the 4-cell eta stencil; 1: k=2 ratio test on both 3-cell halves */
    int characteristic;  /* 1D Euler: reconstruct characteristic fields */
    int k;               /* order parameter of the ENO stencils: 2 or 3 (0 means 3) */
    int cross_2d;        /* 2D, k = 2: shape parameter of Sec. 6 on the 5-cell cross (1) or of the line (0) */
    int bc_y;            /* 2D: boundary condition of the y direction (columns); < 0: the bc argument */
    int gauss_2d;        /* 2D, k = 2: eq. 2DIntegral with two Gauss points per face (1) or the midpoint (0) */
    double eps_M;     /* additive guard of the eta denominator */
    double eps_weno;  /* WENO epsilon (1e-6) */
    double gamma;     /* ratio of specific heats */
    double adv_speed; /* advection speed, x */
    double adv_speed_y;
    double inflow[4]; /* ghost state for the inflow boundary */
    double tie_tol;   /* relative margin that marks a decision as a near tie */
    double eta_guard; /* eta = 0 where |den| <= eta_guard * (|w0| + 15|w1| + 15|w2| + |w3|); 0 = off */
    double eta_max;   /* eta = 0 where |eta| > eta_max; 0 = off (the paper's eta) */
    long* counters;   /* NULL, or ORC_NCOUNTERS counts that the reconstructions add to */
} orc_params;

typedef struct {
    long steps;
    double t;
    double alpha_max;
    int status;
    int pad_;
} orc_solve_stats;

double orc_table_coef(int rbf, int r, int j, double eta);
int orc_switch_k3(const double w[4], int variant, double tol, int* near_tie);
int orc_switch_k2(const double c[3], double tol, int* near_tie);
double orc_eta_k2(const double c[3], int side, const orc_params* p);
double orc_eta_k2_cross(const double c[3], int side, int central, double trans, const orc_params* p);
int orc_reconstruct_2d(const double* u, long nx, long ny, int m, int bc, const orc_params* p, double* vmx, double* vpx,
                       double* vmy, double* vpy);
int orc_reconstruct_2d_at(const double* u, long nx, long ny, int m, int bc, const orc_params* p, double sigma,
                          double* vmx, double* vpx, double* vmy, double* vpy);
double orc_eta_k2_point(const double c[3], int side, int central, double trans, double sg, double xy, double sigma,
                        const orc_params* p);
double orc_table_coef_k2(int rbf, int r, int j, double eta);
int orc_eno_choice(const double c[5], double tol, int* near_tie);
void orc_beta_k3(const double c[5], double beta[3]);
int orc_euler_eigvec(const double UL[3], const double UR[3], double gamma, double R[3][3], double L[3][3]);
int orc_reconstruct(const double* u, long n, int m, int bc, const orc_params* p, double* vm, double* vp,
                    uint8_t* flags, double* eta, const uint8_t* replay, uint8_t* reason);
int orc_flux(const double* vm, const double* vp, long nf, int m, int kind, int dir, double alpha,
             const orc_params* p, double* h);
double orc_max_speed(const double* u, long ncell, int m, int kind, int dir, const orc_params* p);
int orc_rk3_step(double* u, long n, int m, double dx, double dt, int kind, int bc, const orc_params* p,
                 double* alpha_out);
int orc_rk3_step_2d(double* u, long nx, long ny, int m, double dx, double dy, double dt, int kind, int bc,
                    const orc_params* p);
int orc_solve(double* u, long n, int m, double dx, double t_end, double cfl, int kind, int bc, const orc_params* p,
              long max_steps, orc_solve_stats* out);
int orc_solve_2d(double* u, long nx, long ny, int m, double dx, double dy, double t_end, double cfl, int kind,
                 int bc, const orc_params* p, long max_steps, orc_solve_stats* out);
#endif
