/*
 * npw_oracle.c -- plain, slow, FP64 CPU oracle for the non-polynomial (RBF-perturbed)
 * ENO3 / WENO5 finite-volume method of Guo & Jung, "Non-polynomial ENO and WENO finite
 * volume methods for hyperbolic conservation laws" (arXiv 1602.00182).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Every routine follows the paper's steps in the paper's order, as plain loops in
 * double precision.  Compile with -O2 -ffp-contract=off so that no multiply-add is
 * fused behind the reader's back.
 *
 * Paper sections used:
 *   Sec. 2   grid, cell averages, stencils S_r(i), primitive V(x), generic linear
 *            reconstruction v^{(r)-}_{i+1/2} = sum_j c_rj vbar_{i-r+j}, and the WENO
 *            convex combination (eq. weno_re) with alpha_r = d_r/(eps+beta_r)^2.
 *   Sec. 3.5 Table k3 (polynomial rows and MQ perturbed rows, eta = eps^2 dx^2).  The
 *            r = -1 row prints 6/11 where the row sum, the Taylor expansion and the flat
 *            limit of the RBF interpolant all require 11/6; 11/6 is used.
 *   Sec. 3.2-3.5 Table k2 (k = 2: polynomial rows, MQ perturbed rows, eta of eq.
 *            i+1/2_eps_approx; Gaussian eta of eq. i+1/2_eps_approx1 and its r = 0 row of eq.
 *            i+1/2_approx1; the Gaussian r = -1, 1 rows are not printed and are derived by
 *            the flat limit of the Gaussian interpolant, as for k = 3).
 *   Sec. 3.3 Gaussian RBF recipe; its k = 3 rows are not printed and are derived from the
 *            same recipe (flat limit of the pure Gaussian interpolant of the primitive,
 *            anchored V(x_{i+1/2}) = 0, first order in eta).
 *   Sec. 4   monotone-polynomial switch (eq. root_value, eq. adaptation), stated for
 *            k = 2 on three cells; generalised here to the four-cell eta stencil of k = 3
 *            (the cubic p on cells i-1..i+2 must be monotone on x_{i-3/2} < x < x_{i+5/2}).
 *   Sec. 5.1 semi-discrete update (eq. PDE1), Lax-Friedrichs flux with a constant alpha,
 *            TVD Runge-Kutta 3.
 *   Sec. 5.2 Example 4: Euler equations, gamma = 1.4.
 *   Sec. 6   2D perturbed reconstruction for k = 2 at a face midpoint (eq. rbf_recon_2d,
 *            eq. i+1/2_eps_2d, eq. i+1/2_eps_approx_2d): the shape parameter also cancels the
 *            transverse term v_yy dy^2 / 24 of the cell averages, using the 5-cell cross.
 *            The same stencil and cancellation at any point of the face (cross_side).
 *   Sec. 7   2D finite volume form (eq. 2DIntegral), applied dimension by dimension, with one
 *            midpoint quadrature point per cell boundary (the paper's experiments) or the two
 *            Gauss points that Sec. 7 names as needed for third order (gauss_2d).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "npw_oracle.h"

/* ------------------------------------------------------------------------------------ */
/* Coefficient tables, Sec. 3.5 Table k3.  Row r (r = -1..2, stored at index r+1) gives   */
/* the value at face x_{i+1/2} from the cells i-r, i-r+1, i-r+2.                          */
/* ------------------------------------------------------------------------------------ */
static const double POLY[4][3] = {
    {11.0 / 6.0, -7.0 / 6.0, 1.0 / 3.0}, /* r = -1 (printed 6/11: typo for 11/6) */
    {1.0 / 3.0, 5.0 / 6.0, -1.0 / 6.0},  /* r = 0 */
    {-1.0 / 6.0, 5.0 / 6.0, 1.0 / 3.0},  /* r = 1 */
    {1.0 / 3.0, -7.0 / 6.0, 11.0 / 6.0}, /* r = 2 */
};
/* Multiquadric perturbation: coefficient of eta in Table k3 (right). */
static const double PERT_MQ[4][3] = {
    {-9.0 / 2.0, 6.0, -3.0 / 2.0},
    {5.0 / 6.0, -2.0 / 3.0, -1.0 / 6.0},
    {-1.0 / 6.0, -2.0 / 3.0, 5.0 / 6.0},
    {-3.0 / 2.0, 6.0, -9.0 / 2.0},
};
/* Gaussian perturbation for k = 3 (not printed; Sec. 3.3 recipe applied to k = 3). */
static const double PERT_GA[4][3] = {
    {-3.0, 3.0, 0.0},
    {2.0 / 3.0, -1.0 / 3.0, -1.0 / 3.0},
    {-1.0 / 3.0, -1.0 / 3.0, 2.0 / 3.0},
    {0.0, 3.0, -3.0},
};
/* Linear WENO weights d_r for v^-_{i+1/2} (r = 0,1,2, r = cells to the left), Sec. 2
 * (deferred by the paper to Shu's lecture notes).  v^+_{i-1/2} uses them mirrored. */
static const double D_MINUS[3] = {3.0 / 10.0, 3.0 / 5.0, 1.0 / 10.0};
static const double D_PLUS[3] = {1.0 / 10.0, 3.0 / 5.0, 3.0 / 10.0};

/* ------------------------------------------------------------------------------------ */
/* k = 2 tables, Sec. 3.5 Table k2.  Row r (r = -1, 0, 1 at index r+1) gives the value at */
/* face x_{i+1/2} from the cells i-r, i-r+1.                                              */
/* ------------------------------------------------------------------------------------ */
static const double POLY2[3][2] = {
    {3.0 / 2.0, -1.0 / 2.0}, /* r = -1 */
    {1.0 / 2.0, 1.0 / 2.0},  /* r = 0 */
    {-1.0 / 2.0, 3.0 / 2.0}, /* r = 1 */
};
/* Multiquadric: coefficient of eta in Table k2 (right). */
static const double PERT2_MQ[3][2] = {
    {-3.0 / 2.0, 1.0 / 2.0},
    {1.0 / 4.0, 1.0 / 4.0},
    {1.0 / 2.0, -3.0 / 2.0},
};
/* Gaussian: r = 0 is eq. i+1/2_approx1 (1/2 + eta/2 on both cells); r = -1 and r = 1 are not
 * printed and follow from the flat limit of the pure Gaussian interpolant of the primitive. */
static const double PERT2_GA[3][2] = {
    {-2.0, 0.0},
    {1.0 / 2.0, 1.0 / 2.0},
    {0.0, -2.0},
};
/* WENO3 linear weights for v^-_{i+1/2}, r = 0 (cells i, i+1) and r = 1 (cells i-1, i);
 * v^+_{i-1/2} uses them mirrored. */
static const double D2_MINUS[2] = {2.0 / 3.0, 1.0 / 3.0};
static const double D2_PLUS[2] = {1.0 / 3.0, 2.0 / 3.0};

double orc_table_coef_k2(int rbf, int r, int j, double eta) {
    if (r < -1 || r > 1 || j < 0 || j > 1) return NAN;
    const double(*q)[2] = (rbf == ORC_RBF_GA) ? PERT2_GA : PERT2_MQ;
    return POLY2[r + 1][j] + q[r + 1][j] * eta;
}

double orc_table_coef(int rbf, int r, int j, double eta) {
    if (r < -1 || r > 2 || j < 0 || j > 2) return NAN;
    const double(*q)[3] = (rbf == ORC_RBF_GA) ? PERT_GA : PERT_MQ;
    return POLY[r + 1][j] + q[r + 1][j] * eta;
}

/* ------------------------------------------------------------------------------------ */
/* Shape parameter, Table k3: eta = (v_{i-1} - 3v_i + 3v_{i+1} - v_{i+2}) /              */
/*                                  (v_{i-1} - 15v_i + 15v_{i+1} - v_{i+2} + eps_M).      */
/* w[0..3] = cells i-1, i, i+1, i+2 around face i+1/2.                                    */
/* ------------------------------------------------------------------------------------ */
static double eta_numerator(const double w[4]) { return w[0] - 3.0 * w[1] + 3.0 * w[2] - w[3]; }
static double eta_denominator(const double w[4]) { return w[0] - 15.0 * w[1] + 15.0 * w[2] - w[3]; }

/* Solve the n x n system A x = b (n <= 4) by Gaussian elimination with partial pivoting. */
static int small_solve(int n, double A[4][4], double b[4], double x[4]) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return -1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                double t = A[c][k];
                A[c][k] = A[piv][k];
                A[piv][k] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r][c] / A[c][c];
            for (int k = c; k < n; ++k) A[r][k] -= f * A[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Monotone-polynomial switch, Sec. 4.                                                    */
/*                                                                                        */
/* Variant 0 (k = 3 generalisation of eq. root_value / eq. adaptation): p is the cubic    */
/* whose averages over cells i-1, i, i+1, i+2 are w[0..3].  In s = (x - x_{i+1/2})/dx the */
/* stencil spans -2 < s < 2.  p is non-monotone there iff p' takes both signs on the open */
/* interval, i.e. min < 0 < max over {p'(-2), p'(2), p'(s*) when the vertex s* of the    */
/* quadratic p' lies strictly inside}.  The cubic is obtained by solving the 4x4 system   */
/* of cell averages of 1, s, s^2, s^3 (no closed form used).                              */
/*                                                                                        */
/* Variant 1 (the paper's k = 2 test applied literally): the ratio of eq. root_value is  */
/* tested on cells {i-1, i, i+1} and on {i, i+1, i+2}; eta = 0 when 0 < ratio < 3 on      */
/* either.  A zero denominator (linear data, no extremum) counts as monotone.             */
/*                                                                                        */
/* Returns 1 when the stencil is non-monotone (eta must be set to 0).  *near is set when  */
/* a deciding quantity lies within tol * scale of its threshold.                          */
/* ------------------------------------------------------------------------------------ */
static int k2_ratio_fires(double a, double b, double c, double tol, int* near) {
    /* three equal averages: p is constant, hence monotone, in exact arithmetic (no tie) */
    if (a == b && b == c) return 0;
    /* x_p / dx = (-2a + 3b - c) / (-a + 2b - c), eq. root_value, cells a, b, c. */
    double num = -2.0 * a + 3.0 * b - c;
    double den = -a + 2.0 * b - c;
    double scale = fabs(a) + fabs(b) + fabs(c);
    if (fabs(den) <= tol * scale) *near = 1;
    if (den == 0.0) return 0;
    double ratio = num / den;
    if (fabs(ratio) <= tol * 4.0 || fabs(ratio - 3.0) <= tol * 4.0) *near = 1;
    return (ratio > 0.0 && ratio < 3.0) ? 1 : 0;
}

int orc_switch_k3(const double w[4], int variant, double tol, int* near_tie) {
    int near = 0, fires;
    if (variant == 1) {
        int f1 = k2_ratio_fires(w[0], w[1], w[2], tol, &near);
        int f2 = k2_ratio_fires(w[1], w[2], w[3], tol, &near);
        fires = f1 || f2;
    } else if (w[0] == w[1] && w[1] == w[2] && w[2] == w[3]) {
        /* four equal averages: p is constant, hence monotone; decided exactly (the elimination
         * below would leave rounding noise in the coefficients of s, s^2, s^3 and decide by its
         * signs) */
        fires = 0;
    } else {
        double A[4][4], b[4], lam[4];
        for (int k = 0; k < 4; ++k) {
            double lo = -2.0 + k, hi = -1.0 + k; /* cell k in s units */
            for (int j = 0; j < 4; ++j) A[k][j] = (pow(hi, j + 1) - pow(lo, j + 1)) / (j + 1);
            b[k] = w[k];
        }
        if (small_solve(4, A, b, lam) != 0) return 0;
        /* p'(s) = qa s^2 + qb s + qc */
        double qa = 3.0 * lam[3], qb = 2.0 * lam[2], qc = lam[1];
        double scale = fabs(w[0]) + fabs(w[1]) + fabs(w[2]) + fabs(w[3]);
        double vals[3];
        int nv = 0;
        vals[nv++] = qa * 4.0 - qb * 2.0 + qc; /* p'(-2) */
        vals[nv++] = qa * 4.0 + qb * 2.0 + qc; /* p'(2) */
        if (qa != 0.0) {
            double sv = -qb / (2.0 * qa);
            if (fabs(fabs(sv) - 2.0) <= tol * 8.0) near = 1;
            if (sv > -2.0 && sv < 2.0) vals[nv++] = qa * sv * sv + qb * sv + qc;
        }
        double mn = vals[0], mx = vals[0];
        for (int k = 0; k < nv; ++k) {
            if (vals[k] < mn) mn = vals[k];
            if (vals[k] > mx) mx = vals[k];
            if (fabs(vals[k]) <= tol * 8.0 * scale) near = 1;
        }
        fires = (mn < 0.0 && mx > 0.0) ? 1 : 0;
    }
    if (near_tie) *near_tie = near;
    return fires;
}

/* ------------------------------------------------------------------------------------ */
/* ENO stencil choice, Sec. 2 / Sec. 3.1: Newton divided differences of the primitive.   */
/* c[0..4] = cells i-2..i+2.  Returns r (cells to the left of i in the chosen stencil).   */
/* The left candidate is taken only when strictly smaller.                                */
/* ------------------------------------------------------------------------------------ */
int orc_eno_choice(const double c[5], double tol, int* near_tie) {
    int near = 0;
    /* first step: add x_{i-3/2} (left) or x_{i+3/2} (right) to {x_{i-1/2}, x_{i+1/2}} */
    double dl = fabs(c[2] - c[1]);
    double dr = fabs(c[3] - c[2]);
    if (fabs(dl - dr) <= tol * fmax(dl, dr)) near = 1;
    int r;
    if (dl < dr) {
        /* stencil cells {i-1, i}: compare the third divided differences */
        double ddl = fabs(c[0] - 2.0 * c[1] + c[2]);
        double ddr = fabs(c[1] - 2.0 * c[2] + c[3]);
        if (fabs(ddl - ddr) <= tol * fmax(ddl, ddr)) near = 1;
        r = (ddl < ddr) ? 2 : 1;
    } else {
        /* stencil cells {i, i+1} */
        double ddl = fabs(c[1] - 2.0 * c[2] + c[3]);
        double ddr = fabs(c[2] - 2.0 * c[3] + c[4]);
        if (fabs(ddl - ddr) <= tol * fmax(ddl, ddr)) near = 1;
        r = (ddl < ddr) ? 1 : 0;
    }
    if (near_tie) *near_tie = near;
    return r;
}

/* ------------------------------------------------------------------------------------ */
/* Jiang-Shu smoothness indicators for k = 3 (cited by the paper, Sec. 2).  c[0..4] =    */
/* cells i-2..i+2; beta[r] is the indicator of stencil S_r(i) = {i-r, .., i-r+2}.          */
/* ------------------------------------------------------------------------------------ */
void orc_beta_k3(const double c[5], double beta[3]) {
    double a, b;
    a = c[2] - 2.0 * c[3] + c[4];
    b = 3.0 * c[2] - 4.0 * c[3] + c[4];
    beta[0] = 13.0 / 12.0 * a * a + 0.25 * b * b;
    a = c[1] - 2.0 * c[2] + c[3];
    b = c[1] - c[3];
    beta[1] = 13.0 / 12.0 * a * a + 0.25 * b * b;
    a = c[0] - 2.0 * c[1] + c[2];
    b = c[0] - 4.0 * c[1] + 3.0 * c[2];
    beta[2] = 13.0 / 12.0 * a * a + 0.25 * b * b;
}

/* ------------------------------------------------------------------------------------ */
/* Reconstruction of one cell's face value.                                               */
/* c[0..4] = cells i-2..i+2; side = 0 gives v^-_{i+1/2} (rows r), side = 1 gives          */
/* v^+_{i-1/2} (rows r-1).  eta is the shape parameter of that face (0 for ENO/WENO-JS).  */
/* forced_r >= 0 replays a given ENO choice.                                              */
/* ------------------------------------------------------------------------------------ */
static double cell_face_value(const double c[5], int side, double eta, const orc_params* p, int forced_r,
                              int* r_out, int* near_out) {
    const double(*q)[3] = (p->rbf == ORC_RBF_GA) ? PERT_GA : PERT_MQ;
    double cand[3];
    for (int r = 0; r < 3; ++r) {
        int row = (side == 0) ? r : r - 1; /* table row */
        double s = 0.0;
        for (int j = 0; j < 3; ++j) {
            double coef = POLY[row + 1][j] + q[row + 1][j] * eta; /* c_rj(eta), Table k3 */
            s += coef * c[2 - r + j];                               /* cell i - r + j */
        }
        cand[r] = s;
    }
    *near_out = 0;
    *r_out = 0;
    if (p->scheme == ORC_ENO || p->scheme == ORC_RBF_ENO) {
        int near = 0;
        int r = orc_eno_choice(c, p->tie_tol, &near);
        if (forced_r >= 0) r = forced_r;
        *r_out = r;
        *near_out = near;
        return cand[r];
    }
    /* WENO: eq. weno_re */
    double beta[3], alpha[3], asum = 0.0;
    orc_beta_k3(c, beta);
    const double* d = (side == 0) ? D_MINUS : D_PLUS;
    for (int r = 0; r < 3; ++r) {
        double den = p->eps_weno + beta[r];
        alpha[r] = d[r] / (den * den);
        asum += alpha[r];
    }
    double v = 0.0;
    for (int r = 0; r < 3; ++r) v += (alpha[r] / asum) * cand[r];
    return v;
}

/* ------------------------------------------------------------------------------------ */
/* One face, one field.  w[0..5] = cells i-2..i+3 around face i+1/2 (left cell i = w[2]). */
/* Writes v^- (from cell i), v^+ (from cell i+1), the flag byte and eta.                  */
/* ------------------------------------------------------------------------------------ */
typedef struct cross_face_ cross_face;
static void face_field_k2(const double w[6], const orc_params* p, const uint8_t* replay, double* vm, double* vp,
                          uint8_t* flag, double* eta_out, const cross_face* cf, uint8_t* reason);

/* Counts of the shape-parameter decisions (orc_params.counters, optional): where the switch
 * set eta = 0, where eta was evaluated, and where the optional guard or bound (neither is in
 * the paper) set the evaluated eta to 0. */
static void count_eta(const orc_params* p, int fired, int guard, int bound) {
    if (!p->counters) return;
    p->counters[ORC_CNT_SWITCH] += fired;
    p->counters[ORC_CNT_EVAL] += !fired;
    p->counters[ORC_CNT_GUARD] += guard;
    p->counters[ORC_CNT_BOUND] += bound;
}

/* cf: transverse data of the face for k = 2 on the 5-cell cross of Sec. 6 (NULL on a line).
 * reason (may be NULL): ORC_ZERO_* bits of the face. */
static void face_field(const double w[6], const orc_params* p, const uint8_t* replay, double* vm, double* vp,
                       uint8_t* flag, double* eta_out, const cross_face* cf, uint8_t* reason) {
    if (p->k == 2) {
        face_field_k2(w, p, replay, vm, vp, flag, eta_out, cf, reason);
        return;
    }
    uint8_t fl = 0, zr = 0;
    double eta = 0.0;
    int rbf_scheme = (p->scheme == ORC_RBF_ENO || p->scheme == ORC_RBF_WENO);
    if (rbf_scheme) {
        int near = 0, fires = 0;
        if (p->monotone_switch) {
            fires = orc_switch_k3(&w[1], p->switch_variant, p->tie_tol, &near);
            if (replay) fires = (*replay & ORC_FLAG_SWITCH) ? 1 : 0;
        }
        if (fires) {
            eta = 0.0; /* eq. adaptation: vanishing shape parameter */
            fl |= ORC_FLAG_SWITCH;
        } else {
            /* optional guard (not in the paper): a denominator below the round-off of the cell
             * averages of a float state is noise; eta = 0 there */
            double den0 = eta_denominator(&w[1]);
            double mag = fabs(w[1]) + 15.0 * fabs(w[2]) + 15.0 * fabs(w[3]) + fabs(w[4]);
            if (!(p->eta_guard > 0.0 && fabs(den0) <= p->eta_guard * mag)) {
                double den = den0 + p->eps_M;
                eta = eta_numerator(&w[1]) / den; /* Table k3 */
                /* optional bound (not in the paper, off by default): the perturbation argument of
                 * Sec. 3 needs a small eta; a monotone stencil with zero slope at the face sends
                 * eta to num/eps_M */
                if (p->eta_max > 0.0 && fabs(eta) > p->eta_max) {
                    eta = 0.0;
                    zr |= ORC_ZERO_BOUND_L;
                }
            } else {
                zr |= ORC_ZERO_GUARD_L;
            }
        }
        count_eta(p, fires, (zr & ORC_ZERO_GUARD_L) != 0, (zr & ORC_ZERO_BOUND_L) != 0);
        if (near) fl |= ORC_FLAG_SWITCH_TIE;
    }
    if (reason) *reason = zr;
    int rl = 0, rr = 0, nl = 0, nr = 0;
    int fl_r = -1, fr_r = -1;
    if (replay && (p->scheme == ORC_ENO || p->scheme == ORC_RBF_ENO)) {
        fl_r = (*replay >> 2) & 3;
        fr_r = (*replay >> 4) & 3;
    }
    *vm = cell_face_value(&w[0], 0, eta, p, fl_r, &rl, &nl);
    *vp = cell_face_value(&w[1], 1, eta, p, fr_r, &rr, &nr);
    fl |= (uint8_t)((rl & 3) << 2) | (uint8_t)((rr & 3) << 4);
    if (nl) fl |= ORC_FLAG_ENO_TIE_L;
    if (nr) fl |= ORC_FLAG_ENO_TIE_R;
    *flag = fl;
    if (eta_out) *eta_out = eta;
}

/* ------------------------------------------------------------------------------------ */
/* k = 2.  A cell i has the 3-cell stencil c[0..2] = cells i-1, i, i+1.                   */
/*                                                                                        */
/* Switch (Sec. 4, eq. root_value, eq. adaptation, as printed for k = 2): the vertex of   */
/* the quadratic p on the stencil lies at x_p / dx = (-2c0 + 3c1 - c2) / (-c0 + 2c1 - c2)  */
/* from x_{i-3/2}; eta = 0 for both faces of the cell when 0 < x_p / dx < 3.              */
/* ------------------------------------------------------------------------------------ */
int orc_switch_k2(const double c[3], double tol, int* near_tie) {
    int near = 0;
    int fires = k2_ratio_fires(c[0], c[1], c[2], tol, &near);
    if (near_tie) *near_tie = near;
    return fires;
}

/* Shape parameter of cell i, Table k2 / eq. i+1/2_eps_approx (MQ) and eq. i+1/2_eps_approx1
 * (Gaussian, half the MQ value; eps_M added as for MQ).  side 0: eta of v^-_{i+1/2}, which
 * estimates v and v'' at x_{i+1/2} from the cells i-1, i, i+1; side 1: eta of v^+_{i-1/2},
 * the mirror image (the same cells read from the right).  Applies the optional guard and
 * bound of the k = 3 path, with the magnitudes of the denominator's terms. */
/* Sec. 6 (k = 2, 2D): the 3-cell polynomial stencil of eq. poly_recon2d (the two cells of the
 * ENO row along the face normal and the transverse neighbour that ENO picks) evaluated at a point
 * of the face, offset sigma transverse cell widths from its midpoint: the value of the Table k2
 * row plus sigma times the one-sided transverse difference sy toward that neighbour (side sg =
 * +1 or -1).  A Taylor expansion at the point (the row's cells sit half a cell behind the face)
 * gives the error e v_xx dx^2 + (1/24 + sg sigma/2 - sigma^2/2) v_yy dy^2 - (sigma/2) v_xy dx dy,
 * e = 1/6 for the stencil of the two cells at the face and -1/3 for the extrapolating one; the
 * perturbation of eq. rbf_recon_2d adds (sum of its q) eta v.  With the second differences a2
 * (along the normal) and trans (across it) for v_xx dx^2 and v_yy dy^2, the mixed difference xy
 * (the cell, the cell across the face and their neighbours on the sg side) for v_xy dx dy, and
 * the face value v from the cells far, centre, across (eq. i+1/2_eps_approx), the cancelling
 * eta is F (-a2 + t trans + x xy) / (-far + 5 centre + 2 across + eps_M), F = 2 (MQ), 1
 * (Gaussian); central stencil: t = -1/4 - 3 sg sigma + 3 sigma^2, x = 3 sigma; extrapolating
 * (whose q sum to -2 times those of the central row): t = 1/8 + 3/2 sg sigma - 3/2 sigma^2,
 * x = -3/2 sigma.  At the midpoint (sigma = 0) this is eq. i+1/2_eps_approx_2d, whose printed
 * denominator lists the coefficients -2, 1, -5, a permutation of the 1, -5, -2 that the
 * derivation gives; with trans = 0 it is the line formula of Table k2.  At sigma = +-1/(2 sqrt 3)
 * (the Gauss points of eq. 2DIntegral) the v_yy term of the midpoint cancels and the sg term
 * remains; a v_xy estimate needs one cell off the 5-cell cross (the diagonal neighbour). */
typedef struct {
    double trans, sg, sy, xy; /* of one cell of the face; see above */
} cross_side;
struct cross_face_ {
    cross_side l, r; /* l: the cell behind v^- (left / lower), r: behind v^+ */
    double sigma;
};

/* zr (may be NULL) receives 1 where the guard, 2 where the bound set the eta to 0 */
static double eta_k2_point_z(const double c[3], int side, int central, const cross_side* cs, double sigma,
                             const orc_params* p, int* zr) {
    double a = (side == 0) ? c[0] : c[2]; /* far cell behind the face's cell */
    double b = c[1];
    double d = (side == 0) ? c[2] : c[0]; /* cell across the face */
    double s = cs->sg;
    double t_tr = central ? (-0.25 + 3.0 * sigma * sigma - 3.0 * s * sigma) : (0.125 - 1.5 * sigma * sigma + 1.5 * s * sigma);
    double t_xy = central ? 3.0 * sigma : -1.5 * sigma;
    double num = -a + 2.0 * b - d + t_tr * cs->trans + t_xy * cs->xy;
    double den0 = -a + 5.0 * b + 2.0 * d;
    double mag = fabs(a) + 5.0 * fabs(b) + 2.0 * fabs(d);
    if (zr) *zr = 0;
    if (p->eta_guard > 0.0 && fabs(den0) <= p->eta_guard * mag) {
        if (zr) *zr = 1;
        return 0.0;
    }
    double eta = ((p->rbf == ORC_RBF_GA) ? 1.0 : 2.0) * num / (den0 + p->eps_M);
    if (p->eta_max > 0.0 && fabs(eta) > p->eta_max) {
        eta = 0.0;
        if (zr) *zr = 2;
    }
    return eta;
}

double orc_eta_k2_point(const double c[3], int side, int central, double trans, double sg, double xy, double sigma,
                        const orc_params* p) {
    cross_side cs = {trans, sg, 0.0, xy};
    return eta_k2_point_z(c, side, central, &cs, sigma, p, NULL);
}

double orc_eta_k2_cross(const double c[3], int side, int central, double trans, const orc_params* p) {
    return orc_eta_k2_point(c, side, central, trans, 1.0, 0.0, 0.0, p);
}

double orc_eta_k2(const double c[3], int side, const orc_params* p) { return orc_eta_k2_cross(c, side, 1, 0.0, p); }

/* Value of cell i at its right face (side 0: v^-_{i+1/2}, rows r) or left face (side 1:   */
/* v^+_{i-1/2}, rows r - 1), k = 2.  c[0..2] = cells i-1, i, i+1; stencil r uses cells     */
/* i-r, i-r+1.                                                                             */
/* eta_c: shape parameter of the stencil of the two cells at the face (row 0), eta_x: of the   */
/* extrapolating stencil (rows -1, 1); equal except on the 5-cell cross of Sec. 6.  shift: the  */
/* transverse term sigma sy of a point off the face midpoint (Sec. 6), added to each candidate. */
static double cell_face_value_k2(const double c[3], int side, double eta_c, double eta_x, const orc_params* p,
                                 int forced_r, int* r_out, int* near_out, double shift) {
    const double(*q)[2] = (p->rbf == ORC_RBF_GA) ? PERT2_GA : PERT2_MQ;
    double cand[2];
    for (int r = 0; r < 2; ++r) {
        int row = (side == 0) ? r : r - 1;
        double eta = (row == 0) ? eta_c : eta_x;
        double s = 0.0;
        for (int j = 0; j < 2; ++j) s += (POLY2[row + 1][j] + q[row + 1][j] * eta) * c[1 - r + j];
        cand[r] = s + shift;
    }
    *near_out = 0;
    *r_out = 0;
    double dl = fabs(c[1] - c[0]), dr = fabs(c[2] - c[1]);
    if (p->scheme == ORC_ENO || p->scheme == ORC_RBF_ENO) {
        /* ENO, Sec. 2: add the left interface point only when its divided difference is
         * strictly smaller */
        if (fabs(dl - dr) <= p->tie_tol * fmax(dl, dr)) *near_out = 1;
        int r = (dl < dr) ? 1 : 0;
        if (forced_r >= 0) r = forced_r;
        *r_out = r;
        return cand[r];
    }
    /* WENO3 (Jiang-Shu): beta_0 = (c2 - c1)^2, beta_1 = (c1 - c0)^2 */
    double beta[2] = {(c[2] - c[1]) * (c[2] - c[1]), (c[1] - c[0]) * (c[1] - c[0])};
    const double* dw = (side == 0) ? D2_MINUS : D2_PLUS;
    double alpha[2], asum = 0.0;
    for (int r = 0; r < 2; ++r) {
        double den = p->eps_weno + beta[r];
        alpha[r] = dw[r] / (den * den);
        asum += alpha[r];
    }
    double v = 0.0;
    for (int r = 0; r < 2; ++r) v += (alpha[r] / asum) * cand[r];
    return v;
}

/* One face, one field, k = 2.  w[0..5] = cells i-2..i+3 around face i+1/2: v^- comes from
 * cell i (stencil w[1..3]) with that cell's side-0 eta, v^+ from cell i+1 (stencil w[2..4])
 * with its side-1 eta.  eta_out receives the eta of v^-. */
static void face_field_k2(const double w[6], const orc_params* p, const uint8_t* replay, double* vm, double* vp,
                          uint8_t* flag, double* eta_out, const cross_face* cf, uint8_t* reason) {
    static const cross_face line = {{0.0, 1.0, 0.0, 0.0}, {0.0, 1.0, 0.0, 0.0}, 0.0};
    if (!cf) cf = &line;
    uint8_t fl = 0, zr = 0;
    double eta_l = 0.0, eta_r = 0.0, eta_lx = 0.0, eta_rx = 0.0;
    if (p->scheme == ORC_RBF_ENO || p->scheme == ORC_RBF_WENO) {
        int near_l = 0, near_r = 0, fires_l = 0, fires_r = 0;
        if (p->monotone_switch) {
            fires_l = orc_switch_k2(&w[1], p->tie_tol, &near_l);
            fires_r = orc_switch_k2(&w[2], p->tie_tol, &near_r);
            if (replay) {
                fires_l = (*replay & ORC_FLAG_SWITCH) ? 1 : 0;
                fires_r = (*replay & ORC_FLAG_SWITCH_R_K2) ? 1 : 0;
            }
        }
        int z1 = 0, z2 = 0;
        if (fires_l) {
            fl |= ORC_FLAG_SWITCH;
        } else {
            eta_l = eta_k2_point_z(&w[1], 0, 1, &cf->l, cf->sigma, p, &z1);
            eta_lx = eta_k2_point_z(&w[1], 0, 0, &cf->l, cf->sigma, p, &z2);
            zr |= (uint8_t)(z1 | z2); /* ORC_ZERO_GUARD_L = 1, ORC_ZERO_BOUND_L = 2 */
        }
        count_eta(p, fires_l, (zr & ORC_ZERO_GUARD_L) != 0, (zr & ORC_ZERO_BOUND_L) != 0);
        if (fires_r) {
            fl |= ORC_FLAG_SWITCH_R_K2;
        } else {
            eta_r = eta_k2_point_z(&w[2], 1, 1, &cf->r, cf->sigma, p, &z1);
            eta_rx = eta_k2_point_z(&w[2], 1, 0, &cf->r, cf->sigma, p, &z2);
            zr |= (uint8_t)((z1 | z2) << 2); /* ORC_ZERO_GUARD_R, ORC_ZERO_BOUND_R */
        }
        count_eta(p, fires_r, (zr & ORC_ZERO_GUARD_R) != 0, (zr & ORC_ZERO_BOUND_R) != 0);
        if (near_l || near_r) fl |= ORC_FLAG_SWITCH_TIE;
    }
    if (reason) *reason = zr;
    int rl = 0, rr = 0, nl = 0, nr = 0, fl_r = -1, fr_r = -1;
    if (replay && (p->scheme == ORC_ENO || p->scheme == ORC_RBF_ENO)) {
        fl_r = (*replay >> 2) & 1;
        fr_r = (*replay >> 4) & 1;
    }
    *vm = cell_face_value_k2(&w[1], 0, eta_l, eta_lx, p, fl_r, &rl, &nl, cf->sigma * cf->l.sy);
    *vp = cell_face_value_k2(&w[2], 1, eta_r, eta_rx, p, fr_r, &rr, &nr, cf->sigma * cf->r.sy);
    fl |= (uint8_t)((rl & 1) << 2) | (uint8_t)((rr & 1) << 4);
    if (nl) fl |= ORC_FLAG_ENO_TIE_L;
    if (nr) fl |= ORC_FLAG_ENO_TIE_R;
    *flag = fl;
    if (eta_out) *eta_out = eta_l;
}

/* ------------------------------------------------------------------------------------ */
/* Boundary conditions: the value of cell k (any integer) of a line of n cells.           */
/* ------------------------------------------------------------------------------------ */
static double line_get(const double* u, long n, long stride, long k, int bc, double inflow) {
    if (bc == ORC_BC_PERIODIC) {
        long kk = k % n;
        if (kk < 0) kk += n;
        return u[kk * stride];
    }
    if (k < 0) return (bc == ORC_BC_INFLOW) ? inflow : u[0];
    if (k >= n) return u[(n - 1) * stride];
    return u[k * stride];
}

/* ------------------------------------------------------------------------------------ */
/* Euler eigen-structure for the characteristic-wise variant.  The paper reconstructs     */
/* the conserved variables of Example 4; the characteristic projection is an option of   */
/* this implementation: Roe average at the face, right eigenvectors R of dF/dU, and       */
/* L = R^{-1} in closed form (L R = I is checked by a test).                              */
/* ------------------------------------------------------------------------------------ */
int orc_euler_eigvec(const double UL[3], const double UR[3], double gamma, double R[3][3], double L[3][3]) {
    double rl = UL[0], rr = UR[0];
    double ul = UL[1] / rl, ur = UR[1] / rr;
    double pl = (gamma - 1.0) * (UL[2] - 0.5 * rl * ul * ul);
    double pr = (gamma - 1.0) * (UR[2] - 0.5 * rr * ur * ur);
    double hl = (UL[2] + pl) / rl, hr = (UR[2] + pr) / rr;
    double sl = sqrt(rl), sr = sqrt(rr);
    double u = (sl * ul + sr * ur) / (sl + sr);
    double h = (sl * hl + sr * hr) / (sl + sr);
    double c2 = (gamma - 1.0) * (h - 0.5 * u * u);
    if (!(c2 > 0.0)) return -1;
    double c = sqrt(c2);
    R[0][0] = 1.0;
    R[0][1] = 1.0;
    R[0][2] = 1.0;
    R[1][0] = u - c;
    R[1][1] = u;
    R[1][2] = u + c;
    R[2][0] = h - u * c;
    R[2][1] = 0.5 * u * u;
    R[2][2] = h + u * c;
    /* L = R^{-1} in closed form, with b1 = (gamma - 1)/c^2 and b2 = b1 u^2 / 2 (the rows are
     * the left eigenvectors of the Euler Jacobian at the Roe state; L R = I is pinned by a test) */
    double b1 = (gamma - 1.0) / c2;
    double b2 = 0.5 * b1 * u * u;
    double uc = u / c, ic = 1.0 / c;
    L[0][0] = 0.5 * (b2 + uc);
    L[0][1] = -0.5 * (b1 * u + ic);
    L[0][2] = 0.5 * b1;
    L[1][0] = 1.0 - b2;
    L[1][1] = b1 * u;
    L[1][2] = -b1;
    L[2][0] = 0.5 * (b2 - uc);
    L[2][1] = -0.5 * (b1 * u - ic);
    L[2][2] = 0.5 * b1;
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Reconstruction along one line of n cells with m fields.  u[k*m_stride + i*stride] is  */
/* field k of cell i.  Face f (f = 0..n) separates cell f-1 and cell f.  Outputs          */
/* vm/vp/flags/eta are [m][n+1].                                                           */
/* ------------------------------------------------------------------------------------ */
/* Transverse data of the cells and faces of one grid line for k = 2 on the 5-cell cross of
 * Sec. 6 (see cross_side): per cell [m][n] the second difference, ENO side and one-sided
 * difference across the line; per face [m][n+1] the mixed difference seen from the cell
 * behind v^- (xyl) and from the cell behind v^+ (xyr); sigma: the point on the faces. */
typedef struct {
    const double *trans, *sg, *sy, *xyl, *xyr;
    double sigma;
} cross_line;

/* cx: transverse data of the line (NULL: a line of its own, no cross). */
static int recon_line(const double* u, long n, int m, long stride, long m_stride, int bc, const orc_params* p,
                      double* vm, double* vp, uint8_t* flags, double* eta, const uint8_t* replay, long out_stride,
                      const cross_line* cx, uint8_t* reason) {
    for (long f = 0; f <= n; ++f) {
        if (p->characteristic && m == 3) {
            double U[6][3], W[6][3], R[3][3], L[3][3];
            for (int j = 0; j < 6; ++j)
                for (int k = 0; k < 3; ++k)
                    U[j][k] = line_get(u + k * m_stride, n, stride, f - 3 + j, bc, p->inflow[k]);
            if (orc_euler_eigvec(U[2], U[3], p->gamma, R, L) != 0) return ORC_ENONFINITE;
            for (int j = 0; j < 6; ++j)
                for (int a = 0; a < 3; ++a) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k) s += L[a][k] * U[j][k];
                    W[j][a] = s;
                }
            double wm[3], wp[3];
            for (int a = 0; a < 3; ++a) {
                double line[6];
                for (int j = 0; j < 6; ++j) line[j] = W[j][a];
                uint8_t fl;
                double et;
                const uint8_t* rp = replay ? &replay[a * out_stride + f] : NULL;
                face_field(line, p, rp, &wm[a], &wp[a], &fl, &et, NULL, reason ? &reason[a * out_stride + f] : NULL);
                if (flags) flags[a * out_stride + f] = fl;
                if (eta) eta[a * out_stride + f] = et;
            }
            for (int k = 0; k < 3; ++k) {
                double sm = 0.0, sp = 0.0;
                for (int a = 0; a < 3; ++a) {
                    sm += R[k][a] * wm[a];
                    sp += R[k][a] * wp[a];
                }
                vm[k * out_stride + f] = sm;
                vp[k * out_stride + f] = sp;
            }
        } else {
            for (int k = 0; k < m; ++k) {
                double line[6];
                for (int j = 0; j < 6; ++j) line[j] = line_get(u + k * m_stride, n, stride, f - 3 + j, bc, p->inflow[k]);
                uint8_t fl;
                double et;
                const uint8_t* rp = replay ? &replay[k * out_stride + f] : NULL;
                cross_face cf = {{0.0, 1.0, 0.0, 0.0}, {0.0, 1.0, 0.0, 0.0}, 0.0};
                if (cx) {
                    /* a ghost cell carries the data of the cell it copies (an inflow ghost:
                     * a constant state, no differences, side +1) */
                    cf.l.trans = line_get(cx->trans + k * n, n, 1, f - 1, bc, 0.0);
                    cf.r.trans = line_get(cx->trans + k * n, n, 1, f, bc, 0.0);
                    cf.l.sg = line_get(cx->sg + k * n, n, 1, f - 1, bc, 1.0);
                    cf.r.sg = line_get(cx->sg + k * n, n, 1, f, bc, 1.0);
                    cf.l.sy = line_get(cx->sy + k * n, n, 1, f - 1, bc, 0.0);
                    cf.r.sy = line_get(cx->sy + k * n, n, 1, f, bc, 0.0);
                    cf.l.xy = cx->xyl[k * (n + 1) + f];
                    cf.r.xy = cx->xyr[k * (n + 1) + f];
                    cf.sigma = cx->sigma;
                }
                face_field(line, p, rp, &vm[k * out_stride + f], &vp[k * out_stride + f], &fl, &et, cx ? &cf : NULL,
                           reason ? &reason[k * out_stride + f] : NULL);
                if (flags) flags[k * out_stride + f] = fl;
                if (eta) eta[k * out_stride + f] = et;
            }
        }
    }
    return ORC_OK;
}

static int check_params(long n, int m, const orc_params* p) {
    if (!p || n < 6 || m < 1 || m > 4) return ORC_EINVAL;
    if (p->scheme < 0 || p->scheme > 3 || p->rbf < 0 || p->rbf > 1) return ORC_EINVAL;
    if (p->k != 0 && p->k != 2 && p->k != 3) return ORC_EINVAL;
    if (p->characteristic && m != 3) return ORC_EINVAL;
    if (p->bc_y > 2) return ORC_EINVAL;
    return ORC_OK;
}

int orc_reconstruct(const double* u, long n, int m, int bc, const orc_params* p, double* vm, double* vp,
                    uint8_t* flags, double* eta, const uint8_t* replay, uint8_t* reason) {
    int st = check_params(n, m, p);
    if (st) return st;
    return recon_line(u, n, m, 1, n, bc, p, vm, vp, flags, eta, replay, n + 1, NULL, reason);
}

/* ------------------------------------------------------------------------------------ */
/* Fluxes (Sec. 5.2 examples) and the Lax-Friedrichs numerical flux (Sec. 5.1).          */
/* dir = 0 for x, 1 for y (2D).                                                           */
/* ------------------------------------------------------------------------------------ */
static void phys_flux(int kind, int dir, const double* U, const orc_params* p, double* F) {
    double g = p->gamma;
    switch (kind) {
        case ORC_FLUX_ADVECTION:
            F[0] = ((dir == 0) ? p->adv_speed : p->adv_speed_y) * U[0];
            break;
        case ORC_FLUX_BURGERS:
            F[0] = 0.5 * U[0] * U[0];
            break;
        case ORC_FLUX_EULER1D: {
            double rho = U[0], u = U[1] / rho, E = U[2];
            double P = (g - 1.0) * (E - 0.5 * rho * u * u);
            F[0] = rho * u;
            F[1] = rho * u * u + P;
            F[2] = (E + P) * u;
            break;
        }
        case ORC_FLUX_EULER2D: {
            double rho = U[0], u = U[1] / rho, v = U[2] / rho, E = U[3];
            double P = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v));
            double un = (dir == 0) ? u : v;
            F[0] = rho * un;
            F[1] = U[1] * un + ((dir == 0) ? P : 0.0);
            F[2] = U[2] * un + ((dir == 0) ? 0.0 : P);
            F[3] = (E + P) * un;
            break;
        }
    }
}

static double wave_speed(int kind, int dir, const double* U, const orc_params* p) {
    double g = p->gamma;
    switch (kind) {
        case ORC_FLUX_ADVECTION:
            return fabs((dir == 0) ? p->adv_speed : p->adv_speed_y);
        case ORC_FLUX_BURGERS:
            return fabs(U[0]);
        case ORC_FLUX_EULER1D: {
            double rho = U[0], u = U[1] / rho;
            double P = (g - 1.0) * (U[2] - 0.5 * rho * u * u);
            return fabs(u) + sqrt(g * P / rho);
        }
        case ORC_FLUX_EULER2D: {
            double rho = U[0], u = U[1] / rho, v = U[2] / rho;
            double P = (g - 1.0) * (U[3] - 0.5 * rho * (u * u + v * v));
            return fabs((dir == 0) ? u : v) + sqrt(g * P / rho);
        }
    }
    return NAN;
}

static int flux_m(int kind) {
    return (kind == ORC_FLUX_EULER1D) ? 3 : (kind == ORC_FLUX_EULER2D) ? 4 : 1;
}

int orc_flux(const double* vm, const double* vp, long nf, int m, int kind, int dir, double alpha,
             const orc_params* p, double* h) {
    if (m != flux_m(kind) || nf < 1) return ORC_EINVAL;
    for (long f = 0; f < nf; ++f) {
        double a[4], b[4], fa[4], fb[4];
        for (int k = 0; k < m; ++k) {
            a[k] = vm[k * nf + f];
            b[k] = vp[k * nf + f];
        }
        phys_flux(kind, dir, a, p, fa);
        phys_flux(kind, dir, b, p, fb);
        for (int k = 0; k < m; ++k) h[k * nf + f] = 0.5 * (fa[k] + fb[k] - alpha * (b[k] - a[k]));
    }
    return ORC_OK;
}

/* alpha = max_i |f'(u_i)|, a constant over the domain (Sec. 5.1). */
double orc_max_speed(const double* u, long ncell, int m, int kind, int dir, const orc_params* p) {
    double amax = 0.0;
    for (long i = 0; i < ncell; ++i) {
        double U[4];
        for (int k = 0; k < m; ++k) U[k] = u[k * ncell + i];
        double s = wave_speed(kind, dir, U, p);
        if (!(s == s)) return NAN;
        if (s > amax) amax = s;
    }
    return amax;
}

/* ------------------------------------------------------------------------------------ */
/* Semi-discrete right-hand side, eq. PDE1: L_i = -(h_{i+1/2} - h_{i-1/2}) / dx.           */
/* ------------------------------------------------------------------------------------ */
static int rhs_1d(const double* u, long n, int m, double dx, int kind, int bc, double alpha, const orc_params* p,
                  double* L) {
    long nf = n + 1;
    double* vm = malloc(sizeof(double) * m * nf);
    double* vp = malloc(sizeof(double) * m * nf);
    double* h = malloc(sizeof(double) * m * nf);
    int st = (vm && vp && h) ? ORC_OK : ORC_ENOMEM;
    if (!st) st = recon_line(u, n, m, 1, n, bc, p, vm, vp, NULL, NULL, NULL, nf, NULL, NULL);
    if (!st) st = orc_flux(vm, vp, nf, m, kind, 0, alpha, p, h);
    if (!st)
        for (int k = 0; k < m; ++k)
            for (long i = 0; i < n; ++i) L[k * n + i] = -(h[k * nf + i + 1] - h[k * nf + i]) / dx;
    free(vm);
    free(vp);
    free(h);
    return st;
}

/* Cell (i, j) of one field of an nx x ny grid, for any integers i, j: columns follow bc, rows
 * bc_y (periodic: wrapped; otherwise the nearest cell of the grid), and an inflow side (the
 * left for bc, the bottom for bc_y) gives the inflow state whatever the other index. */
static double grid_cell(const double* uk, long nx, long ny, long i, long j, int bc, int bcy, double inflow) {
    if (bcy == ORC_BC_INFLOW && j < 0) return inflow;
    if (bc == ORC_BC_INFLOW && i < 0) return inflow;
    if (bc == ORC_BC_PERIODIC) {
        i %= nx;
        if (i < 0) i += nx;
    } else {
        i = (i < 0) ? 0 : (i >= nx ? nx - 1 : i);
    }
    if (bcy == ORC_BC_PERIODIC) {
        j %= ny;
        if (j < 0) j += ny;
    } else {
        j = (j < 0) ? 0 : (j >= ny ? ny - 1 : j);
    }
    return uk[j * nx + i];
}

/* Cell a of grid line `line` (a row for dir 0, a column for dir 1) shifted b cells across it. */
static double line_cell(const double* uk, long nx, long ny, int dir, long line, long a, long b, int bc, int bcy,
                        double inflow) {
    return (dir == 0) ? grid_cell(uk, nx, ny, a, line + b, bc, bcy, inflow)
                      : grid_cell(uk, nx, ny, line + b, a, bc, bcy, inflow);
}

/* ENO side across the line of cell a (Sec. 6: the transverse neighbour that Newton's divided
 * differences pick, the lower one only where its difference is strictly smaller, as in 1D). */
static double cross_side_of(const double* uk, long nx, long ny, int dir, long line, long a, int bc, int bcy,
                            double inflow, double* sy) {
    double c = line_cell(uk, nx, ny, dir, line, a, 0, bc, bcy, inflow);
    double dn = c - line_cell(uk, nx, ny, dir, line, a, -1, bc, bcy, inflow);
    double up = line_cell(uk, nx, ny, dir, line, a, 1, bc, bcy, inflow) - c;
    double s = (fabs(dn) < fabs(up)) ? -1.0 : 1.0;
    if (sy) *sy = (s < 0.0) ? dn : up;
    return s;
}

/* Transverse data of grid line `line` for k = 2 on the 5-cell cross (Sec. 6), see cross_line:
 * dir 0 = row j (faces of the x sweep, points along y), dir 1 = column i.  Buffers: tr, sg, sy
 * [m][n], xyl, xyr [m][n+1], n the cells of the line. */
static void cross_data(const double* u, long nx, long ny, int m, int bc, int bcy, const orc_params* p, int dir,
                       long line, double sigma, double* tr, double* sg, double* sy, double* xyl, double* xyr,
                       cross_line* cx) {
    long cells = nx * ny, n = (dir == 0) ? nx : ny;
    for (int k = 0; k < m; ++k) {
        const double* uk = u + k * cells;
        double in = p->inflow[k];
        for (long a = 0; a < n; ++a) {
            double dn = line_cell(uk, nx, ny, dir, line, a, -1, bc, bcy, in);
            double c = line_cell(uk, nx, ny, dir, line, a, 0, bc, bcy, in);
            double up = line_cell(uk, nx, ny, dir, line, a, 1, bc, bcy, in);
            tr[k * n + a] = dn - 2.0 * c + up;
            sg[k * n + a] = cross_side_of(uk, nx, ny, dir, line, a, bc, bcy, in, &sy[k * n + a]);
        }
        /* face f between cells f-1 and f of the line: the mixed difference of the cell behind
         * v^- with the cell across the face, on the cell's ENO side, and the same seen from the
         * cell behind v^+ (a ghost cell by the boundary rule of grid_cell) */
        for (long f = 0; f <= n; ++f) {
            long L = f - 1, R = f;
            double sl = cross_side_of(uk, nx, ny, dir, line, L, bc, bcy, in, NULL);
            double sr = cross_side_of(uk, nx, ny, dir, line, R, bc, bcy, in, NULL);
            long bl = (long)sl, br = (long)sr;
            double dl = (line_cell(uk, nx, ny, dir, line, R, bl, bc, bcy, in) -
                         line_cell(uk, nx, ny, dir, line, L, bl, bc, bcy, in)) -
                        (line_cell(uk, nx, ny, dir, line, R, 0, bc, bcy, in) -
                         line_cell(uk, nx, ny, dir, line, L, 0, bc, bcy, in));
            double dr = (line_cell(uk, nx, ny, dir, line, L, br, bc, bcy, in) -
                         line_cell(uk, nx, ny, dir, line, R, br, bc, bcy, in)) -
                        (line_cell(uk, nx, ny, dir, line, L, 0, bc, bcy, in) -
                         line_cell(uk, nx, ny, dir, line, R, 0, bc, bcy, in));
            xyl[k * (n + 1) + f] = sl * dl;
            xyr[k * (n + 1) + f] = sr * dr;
        }
    }
    cx->trans = tr;
    cx->sg = sg;
    cx->sy = sy;
    cx->xyl = xyl;
    cx->xyr = xyr;
    cx->sigma = sigma;
}

static int use_cross(const orc_params* p) {
    return p->cross_2d && p->k == 2 && (p->scheme == ORC_RBF_ENO || p->scheme == ORC_RBF_WENO);
}

/* 2D parameters: Gauss points need k = 2, and the RBF schemes the shape parameter of the cross */
static int check_2d(long nx, long ny, int m, const orc_params* p) {
    int st = check_params(nx, m, p);
    if (st || ny < 6 || p->characteristic) return ORC_EINVAL;
    if (p->gauss_2d && (p->k != 2 || ((p->scheme == ORC_RBF_ENO || p->scheme == ORC_RBF_WENO) && !p->cross_2d)))
        return ORC_EINVAL;
    return ORC_OK;
}

/* The two Gauss points of a face of eq. 2DIntegral: +-1/(2 sqrt 3) cell widths from the midpoint */
#define ORC_GAUSS2 0.28867513459481288225

/* Work buffers of the 2D sweeps */
typedef struct {
    double *vm, *vp, *h, *h2, *tr, *sg, *sy, *xyl, *xyr;
} work2d;

static int work2d_alloc(work2d* w, long nmax, int m) {
    size_t f = sizeof(double) * m * (nmax + 1), c = sizeof(double) * m * nmax;
    w->vm = malloc(f);
    w->vp = malloc(f);
    w->h = malloc(f);
    w->h2 = malloc(f);
    w->xyl = malloc(f);
    w->xyr = malloc(f);
    w->tr = malloc(c);
    w->sg = malloc(c);
    w->sy = malloc(c);
    return (w->vm && w->vp && w->h && w->h2 && w->xyl && w->xyr && w->tr && w->sg && w->sy) ? ORC_OK : ORC_ENOMEM;
}

static void work2d_free(work2d* w) {
    free(w->vm);
    free(w->vp);
    free(w->h);
    free(w->h2);
    free(w->xyl);
    free(w->xyr);
    free(w->tr);
    free(w->sg);
    free(w->sy);
}

/* Face values of grid line `line` of direction dir at the point sigma of every face (Sec. 6;
 * sigma = 0: the midpoint).  Outputs vm/vp [m][n+1]. */
static int line_points(const double* u, long nx, long ny, int m, int bc, int bcy, const orc_params* p, int dir,
                       long line, double sigma, work2d* w) {
    long cells = nx * ny;
    cross_line cx;
    int need = use_cross(p) || sigma != 0.0;
    if (need) cross_data(u, nx, ny, m, bc, bcy, p, dir, line, sigma, w->tr, w->sg, w->sy, w->xyl, w->xyr, &cx);
    if (dir == 0)
        return recon_line(u + line * nx, nx, m, 1, cells, bc, p, w->vm, w->vp, NULL, NULL, NULL, nx + 1,
                          need ? &cx : NULL, NULL);
    return recon_line(u + line, ny, m, nx, cells, bcy, p, w->vm, w->vp, NULL, NULL, NULL, ny + 1, need ? &cx : NULL,
                      NULL);
}

/* Face values of the 2D grid at the point sigma of every face (sigma in [-1/2, 1/2] cell
 * widths from the midpoint along the face; sigma != 0 needs k = 2): x faces vmx/vpx
 * [m][ny][nx+1] (face i of row j between cells i-1 and i, the point at y_j + sigma dy), y faces
 * vmy/vpy [m][ny+1][nx] (face j of column i between rows j-1 and j, at x_i + sigma dx). */
int orc_reconstruct_2d_at(const double* u, long nx, long ny, int m, int bc, const orc_params* p, double sigma,
                          double* vmx, double* vpx, double* vmy, double* vpy) {
    int st = check_2d(nx, ny, m, p);
    if (st || !(fabs(sigma) <= 0.5) || (sigma != 0.0 && p->k != 2)) return ORC_EINVAL;
    const int bcy = p->bc_y < 0 ? bc : p->bc_y; /* boundary of the y sweeps */
    work2d w;
    st = work2d_alloc(&w, (nx > ny) ? nx : ny, m);
    for (long j = 0; j < ny && !st; ++j) {
        st = line_points(u, nx, ny, m, bc, bcy, p, 0, j, sigma, &w);
        for (int k = 0; k < m && !st; ++k)
            for (long i = 0; i <= nx; ++i) {
                vmx[(k * ny + j) * (nx + 1) + i] = w.vm[k * (nx + 1) + i];
                vpx[(k * ny + j) * (nx + 1) + i] = w.vp[k * (nx + 1) + i];
            }
    }
    for (long i = 0; i < nx && !st; ++i) {
        st = line_points(u, nx, ny, m, bc, bcy, p, 1, i, sigma, &w);
        for (int k = 0; k < m && !st; ++k)
            for (long j = 0; j <= ny; ++j) {
                vmy[(k * (ny + 1) + j) * nx + i] = w.vm[k * (ny + 1) + j];
                vpy[(k * (ny + 1) + j) * nx + i] = w.vp[k * (ny + 1) + j];
            }
    }
    work2d_free(&w);
    return st;
}

int orc_reconstruct_2d(const double* u, long nx, long ny, int m, int bc, const orc_params* p, double* vmx, double* vpx,
                       double* vmy, double* vpy) {
    return orc_reconstruct_2d_at(u, nx, ny, m, bc, p, 0.0, vmx, vpx, vmy, vpy);
}

/* Numerical flux of every face of grid line `line` (Sec. 7, eq. 2DIntegral divided by the face
 * length): the Lax-Friedrichs flux at the face midpoint, or (gauss_2d) the mean of the fluxes at
 * the two Gauss points.  Output w->h [m][n+1]. */
static int line_flux(const double* u, long nx, long ny, int m, int kind, int bc, int bcy, double alpha,
                     const orc_params* p, int dir, long line, work2d* w) {
    long n = (dir == 0) ? nx : ny;
    if (!p->gauss_2d) {
        int st = line_points(u, nx, ny, m, bc, bcy, p, dir, line, 0.0, w);
        return st ? st : orc_flux(w->vm, w->vp, n + 1, m, kind, dir, alpha, p, w->h);
    }
    int st = line_points(u, nx, ny, m, bc, bcy, p, dir, line, -ORC_GAUSS2, w);
    if (!st) st = orc_flux(w->vm, w->vp, n + 1, m, kind, dir, alpha, p, w->h2);
    if (!st) st = line_points(u, nx, ny, m, bc, bcy, p, dir, line, ORC_GAUSS2, w);
    if (!st) st = orc_flux(w->vm, w->vp, n + 1, m, kind, dir, alpha, p, w->h);
    for (long f = 0; f < m * (n + 1) && !st; ++f) w->h[f] = 0.5 * (w->h2[f] + w->h[f]);
    return st;
}

/* 2D: eq. 2DIntegral, the x and y sweeps each a reconstruction along a grid line (k = 2 with
 * cross_2d: the shape parameter of Sec. 6), one quadrature point per face (the midpoint, as in
 * the paper's experiments) or two Gauss points (gauss_2d).  u is [m][ny][nx]. */
static int rhs_2d(const double* u, long nx, long ny, int m, double dx, double dy, int kind, int bc, double ax,
                  double ay, const orc_params* p, double* L) {
    long cells = nx * ny;
    const int bcy = p->bc_y < 0 ? bc : p->bc_y; /* boundary of the y sweeps */
    work2d w;
    int st = work2d_alloc(&w, (nx > ny) ? nx : ny, m);
    for (long i = 0; i < m * cells && !st; ++i) L[i] = 0.0;
    /* x sweeps: row j */
    for (long j = 0; j < ny && !st; ++j) {
        st = line_flux(u, nx, ny, m, kind, bc, bcy, ax, p, 0, j, &w);
        for (int k = 0; k < m && !st; ++k)
            for (long i = 0; i < nx; ++i)
                L[k * cells + j * nx + i] -= (w.h[k * (nx + 1) + i + 1] - w.h[k * (nx + 1) + i]) / dx;
    }
    /* y sweeps: column i */
    for (long i = 0; i < nx && !st; ++i) {
        st = line_flux(u, nx, ny, m, kind, bc, bcy, ay, p, 1, i, &w);
        for (int k = 0; k < m && !st; ++k)
            for (long j = 0; j < ny; ++j)
                L[k * cells + j * nx + i] -= (w.h[k * (ny + 1) + j + 1] - w.h[k * (ny + 1) + j]) / dy;
    }
    work2d_free(&w);
    return st;
}

/* ------------------------------------------------------------------------------------ */
/* TVD Runge-Kutta 3 (Sec. 5.1, the Shu-Osher form), alpha frozen over the step.           */
/* nx, ny: ny == 0 means 1D.                                                               */
/* ------------------------------------------------------------------------------------ */
static int rhs_any(const double* u, long nx, long ny, int m, double dx, double dy, int kind, int bc, double ax,
                   double ay, const orc_params* p, double* L) {
    if (ny == 0) return rhs_1d(u, nx, m, dx, kind, bc, ax, p, L);
    return rhs_2d(u, nx, ny, m, dx, dy, kind, bc, ax, ay, p, L);
}

static int rk3_any(double* u, long nx, long ny, int m, double dx, double dy, double dt, int kind, int bc, double ax,
                   double ay, const orc_params* p) {
    long len = m * nx * (ny ? ny : 1);
    double* L = malloc(sizeof(double) * len);
    double* u1 = calloc(len, sizeof(double));
    double* u2 = calloc(len, sizeof(double));
    int st = (L && u1 && u2) ? ORC_OK : ORC_ENOMEM;
    if (!st) st = rhs_any(u, nx, ny, m, dx, dy, kind, bc, ax, ay, p, L);
    if (!st)
        for (long i = 0; i < len; ++i) u1[i] = u[i] + dt * L[i];
    if (!st) st = rhs_any(u1, nx, ny, m, dx, dy, kind, bc, ax, ay, p, L);
    if (!st)
        for (long i = 0; i < len; ++i) u2[i] = 0.75 * u[i] + 0.25 * (u1[i] + dt * L[i]);
    if (!st) st = rhs_any(u2, nx, ny, m, dx, dy, kind, bc, ax, ay, p, L);
    if (!st)
        for (long i = 0; i < len; ++i) u[i] = (1.0 / 3.0) * u[i] + (2.0 / 3.0) * (u2[i] + dt * L[i]);
    for (long i = 0; i < len && !st; ++i)
        if (!(u[i] - u[i] == 0.0)) st = ORC_ENONFINITE;
    free(L);
    free(u1);
    free(u2);
    return st;
}

int orc_rk3_step(double* u, long n, int m, double dx, double dt, int kind, int bc, const orc_params* p,
                 double* alpha_out) {
    int st = check_params(n, m, p);
    if (st) return st;
    if (m != flux_m(kind) || kind == ORC_FLUX_EULER2D) return ORC_EINVAL;
    double a = orc_max_speed(u, n, m, kind, 0, p);
    if (!(a == a)) return ORC_ENONFINITE;
    if (alpha_out) *alpha_out = a;
    return rk3_any(u, n, 0, m, dx, 1.0, dt, kind, bc, a, 0.0, p);
}

int orc_rk3_step_2d(double* u, long nx, long ny, int m, double dx, double dy, double dt, int kind, int bc,
                    const orc_params* p) {
    int st = check_2d(nx, ny, m, p);
    if (st) return st;
    if (m != ((kind == ORC_FLUX_EULER2D) ? 4 : 1) || kind == ORC_FLUX_EULER1D) return ORC_EINVAL;
    double ax = orc_max_speed(u, nx * ny, m, kind, 0, p);
    double ay = orc_max_speed(u, nx * ny, m, kind, 1, p);
    if (!(ax == ax) || !(ay == ay)) return ORC_ENONFINITE;
    return rk3_any(u, nx, ny, m, dx, dy, dt, kind, bc, ax, ay, p);
}

/* ------------------------------------------------------------------------------------ */
/* Time loop: dt = cfl * dx / alpha^n (1D) or cfl / (ax/dx + ay/dy) (2D); the last step is */
/* shortened to end exactly at t_end.                                                     */
/* ------------------------------------------------------------------------------------ */
static int solve_any(double* u, long nx, long ny, int m, double dx, double dy, double t_end, double cfl, int kind,
                     int bc, const orc_params* p, long max_steps, orc_solve_stats* out) {
    double t = 0.0;
    long steps = 0;
    double amax = 0.0;
    int st = ORC_OK;
    long cells = nx * (ny ? ny : 1);
    while (t < t_end) {
        if (max_steps >= 0 && steps >= max_steps) break;
        double ax = orc_max_speed(u, cells, m, kind, 0, p);
        double ay = ny ? orc_max_speed(u, cells, m, kind, 1, p) : 0.0;
        if (!(ax == ax) || !(ay == ay)) {
            st = ORC_ENONFINITE;
            break;
        }
        double rate = ny ? (ax / dx + ay / dy) : (ax / dx);
        if (ax > amax) amax = ax;
        if (ay > amax) amax = ay;
        double dt = (rate > 0.0) ? cfl / rate : t_end - t;
        int last = 0;
        /* the step that reaches t_end to within 1e-10 of a step is the last one */
        if (t + dt * (1.0 + 1e-10) >= t_end) {
            dt = t_end - t;
            last = 1;
        }
        st = rk3_any(u, nx, ny, m, dx, dy, dt, kind, bc, ax, ay, p);
        if (st) break;
        ++steps;
        t = last ? t_end : t + dt;
    }
    if (out) {
        out->steps = steps;
        out->t = t;
        out->alpha_max = amax;
        out->status = st;
    }
    return st;
}

int orc_solve(double* u, long n, int m, double dx, double t_end, double cfl, int kind, int bc, const orc_params* p,
              long max_steps, orc_solve_stats* out) {
    int st = check_params(n, m, p);
    if (st) return st;
    if (m != flux_m(kind) || kind == ORC_FLUX_EULER2D) return ORC_EINVAL;
    return solve_any(u, n, 0, m, dx, 1.0, t_end, cfl, kind, bc, p, max_steps, out);
}

int orc_solve_2d(double* u, long nx, long ny, int m, double dx, double dy, double t_end, double cfl, int kind,
                 int bc, const orc_params* p, long max_steps, orc_solve_stats* out) {
    int st = check_2d(nx, ny, m, p);
    if (st) return st;
    if (m != ((kind == ORC_FLUX_EULER2D) ? 4 : 1) || kind == ORC_FLUX_EULER1D) return ORC_EINVAL;
    return solve_any(u, nx, ny, m, dx, dy, t_end, cfl, kind, bc, p, max_steps, out);
}
