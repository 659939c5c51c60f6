// npw_device.cuh -- per-face arithmetic of the non-polynomial ENO3 / WENO5 method on the GPU.
//
// R is the state type (double or float); D is the type in which the shape parameter, the
// monotone switch, the ENO choice and the smoothness indicators are evaluated (double).
// In the double instantiation every expression is written in a fixed evaluation order and
// the translation unit is compiled without multiply-add contraction, so that results are
// reproducible bit for bit from the cell averages.
//
// Paper passages: Sec. 2 (stencils S_r(i), v^{(r)-}_{i+1/2} = sum_j c_rj vbar_{i-r+j}, eq.
// weno_re with alpha_r = d_r / (eps + beta_r)^2), Sec. 3.5 Table k3 (coefficients and eta;
// row r = -1 uses 11/6), Sec. 3.3 (Gaussian recipe; k = 3 rows derived from the flat limit of
// the Gaussian interpolant of the primitive), Sec. 4 (eq. root_value, eq. adaptation),
// Sec. 5.1 (Lax-Friedrichs flux), Sec. 5.2 Ex. 4 (Euler, ideal gas).  k = 2: Sec. 3.2-3.5
// Table k2 with the shape parameter of eq. i+1/2_eps_approx (MQ) / i+1/2_eps_approx1
// (Gaussian), the Gaussian rows r = -1, 1 from the flat limit, and the switch of eq.
// root_value / eq. adaptation on the cell's three-cell stencil.
#pragma once
#include <cstdint>

#include "npw_internal.h"

namespace npw {

// ---------------------------------------------------------------------------------------
// Table k3.  row = r + 1 for r = -1..2; row r gives the value at face x_{i+1/2} from the
// cells i-r, i-r+1, i-r+2.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T poly_coef(int row, int j) {
    switch (row * 3 + j) {
        case 0: return T(11.0 / 6.0);
        case 1: return T(-7.0 / 6.0);
        case 2: return T(1.0 / 3.0);
        case 3: return T(1.0 / 3.0);
        case 4: return T(5.0 / 6.0);
        case 5: return T(-1.0 / 6.0);
        case 6: return T(-1.0 / 6.0);
        case 7: return T(5.0 / 6.0);
        case 8: return T(1.0 / 3.0);
        case 9: return T(1.0 / 3.0);
        case 10: return T(-7.0 / 6.0);
        default: return T(11.0 / 6.0);
    }
}

// coefficient of eta: multiquadric (Table k3, right) or Gaussian (Sec. 3.3 recipe, k = 3)
template <typename T>
__device__ __forceinline__ T pert_coef(int rbf, int row, int j) {
    if (rbf == NPW_RBF_GA_) {
        switch (row * 3 + j) {
            case 0: return T(-3.0);
            case 1: return T(3.0);
            case 2: return T(0.0);
            case 3: return T(2.0 / 3.0);
            case 4: return T(-1.0 / 3.0);
            case 5: return T(-1.0 / 3.0);
            case 6: return T(-1.0 / 3.0);
            case 7: return T(-1.0 / 3.0);
            case 8: return T(2.0 / 3.0);
            case 9: return T(0.0);
            case 10: return T(3.0);
            default: return T(-3.0);
        }
    }
    switch (row * 3 + j) {
        case 0: return T(-9.0 / 2.0);
        case 1: return T(6.0);
        case 2: return T(-3.0 / 2.0);
        case 3: return T(5.0 / 6.0);
        case 4: return T(-2.0 / 3.0);
        case 5: return T(-1.0 / 6.0);
        case 6: return T(-1.0 / 6.0);
        case 7: return T(-2.0 / 3.0);
        case 8: return T(5.0 / 6.0);
        case 9: return T(-3.0 / 2.0);
        case 10: return T(6.0);
        default: return T(-9.0 / 2.0);
    }
}

// linear weights for v^-_{i+1/2} (d_r, r = cells to the left) and mirrored for v^+_{i-1/2}
template <typename T>
__device__ __forceinline__ T lin_weight(int side, int r) {
    if (side == 0) return r == 0 ? T(3.0 / 10.0) : (r == 1 ? T(3.0 / 5.0) : T(1.0 / 10.0));
    return r == 0 ? T(1.0 / 10.0) : (r == 1 ? T(3.0 / 5.0) : T(3.0 / 10.0));
}

// ---------------------------------------------------------------------------------------
// Shape parameter (Table k3): eta = (w0 - 3 w1 + 3 w2 - w3) / (w0 - 15 w1 + 15 w2 - w3 + eps_M)
// with w = cells i-1..i+2 of face i+1/2.
// ---------------------------------------------------------------------------------------
template <typename D>
__device__ __forceinline__ D eta_num(D w0, D w1, D w2, D w3) {
    return w0 - D(3.0) * w1 + D(3.0) * w2 - w3;
}
template <typename D>
__device__ __forceinline__ D eta_den(D w0, D w1, D w2, D w3) {
    return w0 - D(15.0) * w1 + D(15.0) * w2 - w3;
}

// ---------------------------------------------------------------------------------------
// Monotone switch (Sec. 4).
// Variant 0: the cubic p with averages w0..w3 over the cells of the eta stencil, in
// s = (x - x_{i+1/2})/dx on -2 < s < 2; 12 p'(s) = A s^2 + B s + C with
//   A = 6 ((w3 - w0) + 3 (w1 - w2)),  B = 6 ((w0 - w1) + (w3 - w2)),
//   C = (w0 - w3) + 15 (w2 - w1).
// p is non-monotone iff 12 p' takes both signs on the open interval: min < 0 < max over
// 12p'(-2) = 4A - 2B + C, 12p'(2) = 4A + 2B + C and, when the vertex -B/(2A) is strictly
// inside (|B| < 4|A|), 12p'(vertex) = C - B^2/(4A).
// Variant 1: the k = 2 ratio of eq. root_value on cells (w0, w1, w2) and on (w1, w2, w3).
// ---------------------------------------------------------------------------------------
template <typename D>
__device__ __forceinline__ bool k2_ratio_fires(D a, D b, D c) {
    D num = D(-2.0) * a + D(3.0) * b - c;
    D den = -a + D(2.0) * b - c;
    if (den == D(0.0)) return false;
    D ratio = num / den;
    return ratio > D(0.0) && ratio < D(3.0);
}

template <typename D>
__device__ __forceinline__ bool switch_fires(D w0, D w1, D w2, D w3, int variant) {
    if (variant == 1) {
        bool f1 = k2_ratio_fires(w0, w1, w2);
        bool f2 = k2_ratio_fires(w1, w2, w3);
        return f1 || f2;
    }
    D A = D(6.0) * ((w3 - w0) + D(3.0) * (w1 - w2));
    D B = D(6.0) * ((w0 - w1) + (w3 - w2));
    D C = (w0 - w3) + D(15.0) * (w2 - w1);
    D vm = D(4.0) * A - D(2.0) * B + C;
    D vp = D(4.0) * A + D(2.0) * B + C;
    D mn = vm < vp ? vm : vp;
    D mx = vm < vp ? vp : vm;
    if (A != D(0.0) && fabs(B) < D(4.0) * fabs(A)) {
        D vv = C - B * B / (D(4.0) * A);
        mn = vv < mn ? vv : mn;
        mx = vv > mx ? vv : mx;
    }
    return mn < D(0.0) && mx > D(0.0);
}

// ---------------------------------------------------------------------------------------
// ENO stencil choice from Newton divided differences (Sec. 2, Sec. 3.1): c0..c4 = cells
// i-2..i+2; the left extension is taken only when strictly smaller.  Returns r.
// ---------------------------------------------------------------------------------------
template <typename D>
__device__ __forceinline__ int eno_choice(D c0, D c1, D c2, D c3, D c4) {
    D dl = fabs(c2 - c1);
    D dr = fabs(c3 - c2);
    if (dl < dr) {
        D ddl = fabs(c0 - D(2.0) * c1 + c2);
        D ddr = fabs(c1 - D(2.0) * c2 + c3);
        return (ddl < ddr) ? 2 : 1;
    }
    D ddl = fabs(c1 - D(2.0) * c2 + c3);
    D ddr = fabs(c2 - D(2.0) * c3 + c4);
    return (ddl < ddr) ? 1 : 0;
}

// Jiang-Shu smoothness indicators (cited in Sec. 2): beta[r] of stencil i-r..i-r+2.
template <typename D>
__device__ __forceinline__ void beta_k3(D c0, D c1, D c2, D c3, D c4, D beta[3]) {
    D a, b;
    a = c2 - D(2.0) * c3 + c4;
    b = D(3.0) * c2 - D(4.0) * c3 + c4;
    beta[0] = D(13.0 / 12.0) * a * a + D(0.25) * b * b;
    a = c1 - D(2.0) * c2 + c3;
    b = c1 - c3;
    beta[1] = D(13.0 / 12.0) * a * a + D(0.25) * b * b;
    a = c0 - D(2.0) * c1 + c2;
    b = c0 - D(4.0) * c1 + D(3.0) * c2;
    beta[2] = D(13.0 / 12.0) * a * a + D(0.25) * b * b;
}

// ---------------------------------------------------------------------------------------
// Value of cell i at its right face (side 0: v^-_{i+1/2}, rows r) or left face (side 1:
// v^+_{i-1/2}, rows r - 1).  c[0..4] = cells i-2..i+2; eta is the face's shape parameter
// (already rounded to R).  forced_r >= 0 replays a stencil choice.
// ---------------------------------------------------------------------------------------
template <typename R, typename D>
__device__ __forceinline__ R cell_face_value(const R* c, int side, R eta, const MethodParams& mp, int* r_out) {
    R cand[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int row = (side == 0) ? r : r - 1;
        R s = R(0.0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            R coef = poly_coef<R>(row + 1, j) + pert_coef<R>(mp.rbf, row + 1, j) * eta;
            s += coef * c[2 - r + j];
        }
        cand[r] = s;
    }
    if (mp.scheme == NPW_ENO_ || mp.scheme == NPW_RBF_ENO_) {
        int r = eno_choice<D>(D(c[0]), D(c[1]), D(c[2]), D(c[3]), D(c[4]));
        *r_out = r;
        return r == 0 ? cand[0] : (r == 1 ? cand[1] : cand[2]);
    }
    *r_out = 0;
    D beta[3];
    beta_k3<D>(D(c[0]), D(c[1]), D(c[2]), D(c[3]), D(c[4]), beta);
    R alpha[3];
    R asum = R(0.0);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        R den = R(D(mp.eps_weno) + beta[r]);
        alpha[r] = lin_weight<R>(side, r) / (den * den);
        asum += alpha[r];
    }
    R v = R(0.0);
#pragma unroll
    for (int r = 0; r < 3; ++r) v += (alpha[r] / asum) * cand[r];
    return v;
}

// ---------------------------------------------------------------------------------------
// k = 2.  Table k2: row = r + 1 for r = -1, 0, 1; row r gives the value at x_{i+1/2} from the
// cells i-r, i-r+1.  A cell i has the stencil c[0..2] = cells i-1, i, i+1; its two face
// values use their own shape parameters (side 0: v^-_{i+1/2}; side 1: v^+_{i-1/2}, the mirror).
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T poly2_coef(int row, int j) {
    switch (row * 2 + j) {
        case 0: return T(3.0 / 2.0);
        case 1: return T(-1.0 / 2.0);
        case 2: return T(1.0 / 2.0);
        case 3: return T(1.0 / 2.0);
        case 4: return T(-1.0 / 2.0);
        default: return T(3.0 / 2.0);
    }
}

// coefficient of eta: multiquadric (Table k2, right) or Gaussian (r = 0: eq. i+1/2_approx1;
// r = -1, 1: flat limit of the Gaussian interpolant)
template <typename T>
__device__ __forceinline__ T pert2_coef(int rbf, int row, int j) {
    if (rbf == NPW_RBF_GA_) {
        switch (row * 2 + j) {
            case 0: return T(-2.0);
            case 1: return T(0.0);
            case 2: return T(1.0 / 2.0);
            case 3: return T(1.0 / 2.0);
            case 4: return T(0.0);
            default: return T(-2.0);
        }
    }
    switch (row * 2 + j) {
        case 0: return T(-3.0 / 2.0);
        case 1: return T(1.0 / 2.0);
        case 2: return T(1.0 / 4.0);
        case 3: return T(1.0 / 4.0);
        case 4: return T(1.0 / 2.0);
        default: return T(-3.0 / 2.0);
    }
}

// WENO3 linear weights: v^-_{i+1/2} d = (2/3, 1/3) for r = 0 (cells i, i+1), r = 1 (i-1, i);
// v^+_{i-1/2} mirrored
template <typename T>
__device__ __forceinline__ T lin_weight2(int side, int r) {
    if (side == 0) return r == 0 ? T(2.0 / 3.0) : T(1.0 / 3.0);
    return r == 0 ? T(1.0 / 3.0) : T(2.0 / 3.0);
}

// shape parameter of a cell, side 0 / 1 (MQ: 2 num / (den + eps_M); Gaussian: half), with the
// optional guard and bound of the k = 3 path (magnitudes of the denominator's terms).  On the
// 5-cell cross of Sec. 6 (2D) the numerator also carries the transverse second difference
// trans of the cell, with weight -1/4 for the stencil of the two cells at the face (central)
// and 1/8 for the extrapolating one: the terms that cancel the transverse curvature of the
// cell averages at the face midpoint.
// *zr receives FL_ZERO_GUARD / FL_ZERO_BOUND where the guard / the bound set eta to 0
template <typename D>
__device__ __forceinline__ D eta_k2_cross(const D* c, int side, bool central, D trans, const MethodParams& mp,
                                          uint32_t* zr) {
    const D a = side == 0 ? c[0] : c[2];
    const D b = c[1];
    const D d = side == 0 ? c[2] : c[0];
    const D num = -a + D(2.0) * b - d + (central ? D(-0.25) : D(0.125)) * trans;
    const D den0 = -a + D(5.0) * b + D(2.0) * d;
    const D mag = fabs(a) + D(5.0) * fabs(b) + D(2.0) * fabs(d);
    if (mp.eta_guard > 0.0 && fabs(den0) <= D(mp.eta_guard) * mag) {
        *zr |= FL_ZERO_GUARD;
        return D(0.0);
    }
    const D e = (mp.rbf == NPW_RBF_GA_ ? D(1.0) : D(2.0)) * num / (den0 + D(mp.eps_M));
    if (mp.eta_max > 0.0 && fabs(e) > D(mp.eta_max)) {
        *zr |= FL_ZERO_BOUND;
        return D(0.0);
    }
    return e;
}

// value of cell i at its right (side 0) or left (side 1) face, k = 2; c[0..2] = cells i-1..i+1;
// eta_c: shape parameter of the central row (row 0), eta_x: of the extrapolating rows
// shift (points off the face midpoint, Sec. 6): the transverse term sigma sy, added to each
// candidate; the midpoint passes none
template <typename R, typename D>
__device__ __forceinline__ R cell_face_value_k2(const R* c, int side, R eta_c, R eta_x, const MethodParams& mp,
                                               int* r_out, R shift = R(0.0), bool shifted = false) {
    R cand[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = (side == 0) ? r : r - 1;
        const R eta = row == 0 ? eta_c : eta_x;
        R s = R(0.0);
#pragma unroll
        for (int j = 0; j < 2; ++j) s += (poly2_coef<R>(row + 1, j) + pert2_coef<R>(mp.rbf, row + 1, j) * eta) * c[1 - r + j];
        cand[r] = shifted ? s + shift : s;
    }
    if (mp.scheme == NPW_ENO_ || mp.scheme == NPW_RBF_ENO_) {
        const int r = fabs(D(c[1]) - D(c[0])) < fabs(D(c[2]) - D(c[1])) ? 1 : 0;
        *r_out = r;
        return cand[r];
    }
    *r_out = 0;
    const D b0 = (D(c[2]) - D(c[1])) * (D(c[2]) - D(c[1]));
    const D b1 = (D(c[1]) - D(c[0])) * (D(c[1]) - D(c[0]));
    const R den0 = R(D(mp.eps_weno) + b0), den1 = R(D(mp.eps_weno) + b1);
    const R a0 = lin_weight2<R>(side, 0) / (den0 * den0);
    const R a1 = lin_weight2<R>(side, 1) / (den1 * den1);
    R asum = R(0.0);
    asum += a0;
    asum += a1;
    R v = R(0.0);
    v += (a0 / asum) * cand[0];
    v += (a1 / asum) * cand[1];
    return v;
}

// One field at one face, k = 2.  w[0..5] = cells i-2..i+3 around face i+1/2; v^- from cell i
// (stencil w[1..3]), v^+ from cell i+1 (stencil w[2..4]); tl, tr: transverse second
// differences of cells i and i+1 (0 on a line).  Flag bits: 0 switch of cell i, 3 switch of
// cell i+1, 2 / 4 ENO r of cell i / i+1, 6 / 7 an eta of v^- zeroed by the guard / the bound,
// 8 / 9 the same for v^+.
template <typename R, typename D>
__device__ __forceinline__ uint32_t face_field_k2(const R* w, const MethodParams& mp, R* vm, R* vp, R tl, R tr,
                                                  R* eta_out) {
    uint32_t fl = 0;
    R el = R(0.0), er = R(0.0), elx = R(0.0), erx = R(0.0);
    if (mp.scheme == NPW_RBF_ENO_ || mp.scheme == NPW_RBF_WENO_) {
        const D cl[3] = {D(w[1]), D(w[2]), D(w[3])};
        const D cr[3] = {D(w[2]), D(w[3]), D(w[4])};
        if (mp.monotone_switch && k2_ratio_fires<D>(cl[0], cl[1], cl[2])) {
            fl |= FL_SWITCH;
        } else {
            el = R(eta_k2_cross<D>(cl, 0, true, D(tl), mp, &fl));
            elx = tl == R(0.0) ? el : R(eta_k2_cross<D>(cl, 0, false, D(tl), mp, &fl));
        }
        if (mp.monotone_switch && k2_ratio_fires<D>(cr[0], cr[1], cr[2])) {
            fl |= FL_SWITCH_R_K2;
        } else {
            uint32_t zr = 0;
            er = R(eta_k2_cross<D>(cr, 1, true, D(tr), mp, &zr));
            erx = tr == R(0.0) ? er : R(eta_k2_cross<D>(cr, 1, false, D(tr), mp, &zr));
            fl |= zr << 2;  // FL_ZERO_GUARD_R_K2, FL_ZERO_BOUND_R_K2
        }
    }
    int rl = 0, rr = 0;
    *vm = cell_face_value_k2<R, D>(w + 1, 0, el, elx, mp, &rl);
    *vp = cell_face_value_k2<R, D>(w + 2, 1, er, erx, mp, &rr);
    fl |= (uint32_t(rl & 1) << 2) | (uint32_t(rr & 1) << 4);
    if (eta_out) *eta_out = el;
    return fl;
}

// ---------------------------------------------------------------------------------------
// k = 2 on the 5-cell cross at a point of the face (Sec. 6; the two Gauss points of eq.
// 2DIntegral, Sec. 7): the 3-cell stencil of the two cells of the ENO row along the normal and
// the transverse neighbour that ENO picks, evaluated sigma cell widths from the face midpoint,
// is the Table k2 row plus sigma times the one-sided transverse difference sy toward that
// neighbour (side sg = +1 / -1).  Its Taylor error there is e v_xx dx^2 + (1/24 + sg sigma/2 -
// sigma^2/2) v_yy dy^2 - (sigma/2) v_xy dx dy (e = 1/6 for the two cells at the face, -1/3 for
// the extrapolating pair, whose perturbation weights sum to -2 times the central row's), and the
// shape parameter cancels it: numerator -a2 + t trans + x xy, central t = -1/4 + 3 sigma^2 -
// 3 sg sigma, x = 3 sigma; extrapolating t = 1/8 - 3/2 sigma^2 + 3/2 sg sigma, x = -3/2 sigma;
// xy is the mixed difference of the cell with the cell across the face on the sg side.
// ---------------------------------------------------------------------------------------
template <typename D>
struct CrossSide {
    D trans, sg, sy, xy;  // of one cell of the face: second difference, ENO side, one-sided difference, mixed
};

// transverse data of a cell from its column (lo, c, hi across the line) and, for xy, the cell
// across the face (alo, a, ahi) on the same rows
template <typename D>
__device__ __forceinline__ CrossSide<D> cross_side(D lo, D c, D hi, D alo, D a, D ahi) {
    CrossSide<D> cs;
    const D dn = c - lo, up = hi - c;
    cs.trans = (lo - D(2.0) * c) + hi;
    const bool lower = fabs(dn) < fabs(up);
    cs.sg = lower ? D(-1.0) : D(1.0);
    cs.sy = lower ? dn : up;
    cs.xy = lower ? -((alo - lo) - (a - c)) : ((ahi - hi) - (a - c));
    return cs;
}

template <typename D>
__device__ __forceinline__ D eta_k2_point(const D* c, int side, bool central, const CrossSide<D>& cs, D sigma,
                                          const MethodParams& mp, uint32_t* zr) {
    const D a = side == 0 ? c[0] : c[2];
    const D b = c[1];
    const D d = side == 0 ? c[2] : c[0];
    const D s = cs.sg;
    const D t_tr = central ? (D(-0.25) + D(3.0) * sigma * sigma) - D(3.0) * s * sigma
                           : (D(0.125) - D(1.5) * sigma * sigma) + D(1.5) * s * sigma;
    const D t_xy = central ? D(3.0) * sigma : D(-1.5) * sigma;
    const D num = ((-a + D(2.0) * b - d) + t_tr * cs.trans) + t_xy * cs.xy;
    const D den0 = -a + D(5.0) * b + D(2.0) * d;
    const D mag = fabs(a) + D(5.0) * fabs(b) + D(2.0) * fabs(d);
    if (mp.eta_guard > 0.0 && fabs(den0) <= D(mp.eta_guard) * mag) {
        *zr |= FL_ZERO_GUARD;
        return D(0.0);
    }
    const D e = (mp.rbf == NPW_RBF_GA_ ? D(1.0) : D(2.0)) * num / (den0 + D(mp.eps_M));
    if (mp.eta_max > 0.0 && fabs(e) > D(mp.eta_max)) {
        *zr |= FL_ZERO_BOUND;
        return D(0.0);
    }
    return e;
}

// One field at one point of a face (sigma from its midpoint), k = 2 on the cross: as
// face_field_k2, with l / r the transverse data of the cells behind v^- / v^+.
template <typename R, typename D>
__device__ __forceinline__ uint32_t face_point_k2(const R* w, const MethodParams& mp, R* vm, R* vp,
                                                  const CrossSide<D>& l, const CrossSide<D>& r, D sigma) {
    uint32_t fl = 0;
    R el = R(0.0), er = R(0.0), elx = R(0.0), erx = R(0.0);
    if (mp.scheme == NPW_RBF_ENO_ || mp.scheme == NPW_RBF_WENO_) {
        const D cl[3] = {D(w[1]), D(w[2]), D(w[3])};
        const D cr[3] = {D(w[2]), D(w[3]), D(w[4])};
        if (mp.monotone_switch && k2_ratio_fires<D>(cl[0], cl[1], cl[2])) {
            fl |= FL_SWITCH;
        } else {
            el = R(eta_k2_point<D>(cl, 0, true, l, sigma, mp, &fl));
            elx = R(eta_k2_point<D>(cl, 0, false, l, sigma, mp, &fl));
        }
        if (mp.monotone_switch && k2_ratio_fires<D>(cr[0], cr[1], cr[2])) {
            fl |= FL_SWITCH_R_K2;
        } else {
            uint32_t zr = 0;
            er = R(eta_k2_point<D>(cr, 1, true, r, sigma, mp, &zr));
            erx = R(eta_k2_point<D>(cr, 1, false, r, sigma, mp, &zr));
            fl |= zr << 2;  // FL_ZERO_GUARD_R_K2, FL_ZERO_BOUND_R_K2
        }
    }
    int rl = 0, rr = 0;
    *vm = cell_face_value_k2<R, D>(w + 1, 0, el, elx, mp, &rl, R(sigma * l.sy), true);
    *vp = cell_face_value_k2<R, D>(w + 2, 1, er, erx, mp, &rr, R(sigma * r.sy), true);
    fl |= (uint32_t(rl & 1) << 2) | (uint32_t(rr & 1) << 4);
    return fl;
}

// One field at one face.  w[0..5] = cells i-2..i+3 around face i+1/2.  Returns the flag
// byte (bit0 switch, bits 2-3 / 4-5 ENO r of the left / right cell, bit 6 / 7 the evaluated eta
// zeroed by the guard / the bound).
// eta_out (may be NULL): the face's shape parameter as used (k = 2: that of v^-, central row)
template <typename R, typename D>
__device__ __forceinline__ uint32_t face_field(const R* w, const MethodParams& mp, R* vm, R* vp, R tl = R(0.0),
                                               R tr = R(0.0), R* eta_out = nullptr) {
    if (mp.k == 2) return face_field_k2<R, D>(w, mp, vm, vp, tl, tr, eta_out);
    uint32_t fl = 0;
    R eta = R(0.0);
    if (mp.scheme == NPW_RBF_ENO_ || mp.scheme == NPW_RBF_WENO_) {
        const D w1 = D(w[1]), w2 = D(w[2]), w3 = D(w[3]), w4 = D(w[4]);
        bool fires = mp.monotone_switch ? switch_fires<D>(w1, w2, w3, w4, mp.switch_variant) : false;
        if (fires) {
            fl |= FL_SWITCH;
        } else {
            D den0 = eta_den<D>(w1, w2, w3, w4);
            bool unresolved = mp.eta_guard > 0.0 &&
                              fabs(den0) <= D(mp.eta_guard) * (fabs(w1) + D(15.0) * fabs(w2) + D(15.0) * fabs(w3) + fabs(w4));
            if (!unresolved) {
                D den = den0 + D(mp.eps_M);
                D e = eta_num<D>(w1, w2, w3, w4) / den;
                if (!(mp.eta_max > 0.0 && fabs(e) > D(mp.eta_max)))
                    eta = R(e);
                else
                    fl |= FL_ZERO_BOUND;
            } else {
                fl |= FL_ZERO_GUARD;
            }
        }
    }
    int rl = 0, rr = 0;
    *vm = cell_face_value<R, D>(w, 0, eta, mp, &rl);
    *vp = cell_face_value<R, D>(w + 1, 1, eta, mp, &rr);
    fl |= (uint32_t(rl & 3) << 2) | (uint32_t(rr & 3) << 4);
    if (eta_out) *eta_out = eta;
    return fl;
}

// ---------------------------------------------------------------------------------------
// Near ties of the threshold decisions at one face (the FL_NEAR_TIE bit of npweno_reconstruct):
// a quantity that decides the monotone switch, the guard or the bound lies within tol
// (relative) of its threshold, so that two correct evaluations in different forms (the
// switch's closed form here, an elimination elsewhere; the guard in float or in double) may
// decide differently.  The ENO choice is not among them: it compares two differences of the
// same cell averages, which every correct evaluation rounds alike, so it is expected to agree
// everywhere.  Margins (all in double, from the cell averages):
//   switch variant 0 (Sec. 4, the cubic on the eta stencil): 12 p' at either end or at an
//     inside vertex within 8 tol (|w0| + .. + |w3|) of 0 (times 12), or the vertex within
//     8 tol of an end of the stencil;  the ratio test (variant 1, k = 2): its denominator
//     within tol (|a| + |b| + |c|) of 0, or the ratio within 4 tol of 0 or 3;  a stencil of
//     equal averages is constant, hence monotone, and not a tie;
//   guard: |den| within tol of the guard threshold; bound: |eta| within tol of eta_max.
// w[0..5] = cells i-2..i+3 of face i+1/2.
// ---------------------------------------------------------------------------------------
// two exactly equal zeros (a plateau) compare the same way in any evaluation: not a tie
__device__ __forceinline__ bool tie_rel(double a, double b, double tol) {
    const double m = fmax(fabs(a), fabs(b));
    return m > 0.0 && fabs(a - b) <= tol * m;
}
__device__ __forceinline__ bool k2_ratio_near(double a, double b, double c, double tol) {
    if (a == b && b == c) return false;  // constant stencil: monotone, decided exactly
    const double num = -2.0 * a + 3.0 * b - c, den = -a + 2.0 * b - c;
    if (fabs(den) <= tol * (fabs(a) + fabs(b) + fabs(c))) return true;
    if (den == 0.0) return false;
    const double r = num / den;
    return fabs(r) <= 4.0 * tol || fabs(r - 3.0) <= 4.0 * tol;
}
__device__ __forceinline__ bool switch_v0_near(const double* w, double tol) {
    if (w[0] == w[1] && w[1] == w[2] && w[2] == w[3]) return false;  // constant stencil
    const double A = 6.0 * ((w[3] - w[0]) + 3.0 * (w[1] - w[2]));
    const double B = 6.0 * ((w[0] - w[1]) + (w[3] - w[2]));
    const double C = (w[0] - w[3]) + 15.0 * (w[2] - w[1]);
    const double lim = 12.0 * 8.0 * tol * (fabs(w[0]) + fabs(w[1]) + fabs(w[2]) + fabs(w[3]));
    bool near = fabs(4.0 * A - 2.0 * B + C) <= lim || fabs(4.0 * A + 2.0 * B + C) <= lim;
    if (A != 0.0) {
        const double sv = -B / (2.0 * A);
        near = near || fabs(fabs(sv) - 2.0) <= 8.0 * tol;
        if (fabs(sv) < 2.0) near = near || fabs(C - B * B / (4.0 * A)) <= lim;
    }
    return near;
}
template <typename R>
__device__ __forceinline__ bool face_near_tie(const R* wr, const MethodParams& mp, double tol) {
    double w[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) w[j] = (double)wr[j];
    const bool rbf = mp.scheme == NPW_RBF_ENO_ || mp.scheme == NPW_RBF_WENO_;
    bool near = false;
    if (mp.k == 2) {
        if (rbf && mp.monotone_switch) near = k2_ratio_near(w[1], w[2], w[3], tol) || k2_ratio_near(w[2], w[3], w[4], tol);
        if (rbf) {
            for (int side = 0; side < 2; ++side) {
                const double* c = w + 1 + side;  // cell i (side 0, v^-) or i + 1 (side 1, v^+)
                const double a = side == 0 ? c[0] : c[2], b = c[1], d = side == 0 ? c[2] : c[0];
                const double den0 = -a + 5.0 * b + 2.0 * d, mag = fabs(a) + 5.0 * fabs(b) + 2.0 * fabs(d);
                if (mp.eta_guard > 0.0) near = near || tie_rel(fabs(den0), mp.eta_guard * mag, tol);
                if (mp.eta_max > 0.0) {
                    const double e = (mp.rbf == NPW_RBF_GA_ ? 1.0 : 2.0) * (-a + 2.0 * b - d) / (den0 + mp.eps_M);
                    near = near || tie_rel(fabs(e), mp.eta_max, tol);
                }
            }
        }
        return near;
    }
    if (rbf && mp.monotone_switch)
        near = near || (mp.switch_variant == 1 ? (k2_ratio_near(w[1], w[2], w[3], tol) || k2_ratio_near(w[2], w[3], w[4], tol))
                                               : switch_v0_near(w + 1, tol));
    if (rbf) {
        const double den0 = eta_den<double>(w[1], w[2], w[3], w[4]);
        const double mag = fabs(w[1]) + 15.0 * fabs(w[2]) + 15.0 * fabs(w[3]) + fabs(w[4]);
        if (mp.eta_guard > 0.0) near = near || tie_rel(fabs(den0), mp.eta_guard * mag, tol);
        if (mp.eta_max > 0.0)
            near = near || tie_rel(fabs(eta_num<double>(w[1], w[2], w[3], w[4]) / (den0 + mp.eps_M)), mp.eta_max, tol);
    }
    return near;
}

// ---------------------------------------------------------------------------------------
// Physical fluxes and wave speeds (Sec. 5.2 examples).  dir 0 = x, 1 = y.
// ---------------------------------------------------------------------------------------
template <typename R, int KIND>
__device__ __forceinline__ void phys_flux(const R* U, const MethodParams& mp, int dir, R* F) {
    if (KIND == NPW_FLUX_ADVECTION_) {
        F[0] = (dir == 0 ? mp_val<R>(mp.adv_speed, mp.adv_speed_f) : mp_val<R>(mp.adv_speed_y, mp.adv_speed_y_f)) * U[0];
    } else if (KIND == NPW_FLUX_BURGERS_) {
        F[0] = R(0.5) * U[0] * U[0];
    } else if (KIND == NPW_FLUX_EULER1D_) {
        const R g = mp_val<R>(mp.gamma, mp.gamma_f);
        R rho = U[0], u = U[1] / rho, E = U[2];
        R P = (g - R(1.0)) * (E - R(0.5) * rho * u * u);
        F[0] = rho * u;
        F[1] = rho * u * u + P;
        F[2] = (E + P) * u;
    } else {
        const R g = mp_val<R>(mp.gamma, mp.gamma_f);
        R rho = U[0], u = U[1] / rho, v = U[2] / rho, E = U[3];
        R P = (g - R(1.0)) * (E - R(0.5) * rho * (u * u + v * v));
        R un = (dir == 0) ? u : v;
        F[0] = rho * un;
        F[1] = U[1] * un + ((dir == 0) ? P : R(0.0));
        F[2] = U[2] * un + ((dir == 0) ? R(0.0) : P);
        F[3] = (E + P) * un;
    }
}

template <typename R, int KIND>
__device__ __forceinline__ R wave_speed(const R* U, const MethodParams& mp, int dir) {
    if (KIND == NPW_FLUX_ADVECTION_)
        return fabs(dir == 0 ? mp_val<R>(mp.adv_speed, mp.adv_speed_f) : mp_val<R>(mp.adv_speed_y, mp.adv_speed_y_f));
    if (KIND == NPW_FLUX_BURGERS_) return fabs(U[0]);
    const R g = mp_val<R>(mp.gamma, mp.gamma_f);
    if (KIND == NPW_FLUX_EULER1D_) {
        R rho = U[0], u = U[1] / rho;
        R P = (g - R(1.0)) * (U[2] - R(0.5) * rho * u * u);
        return fabs(u) + sqrt(g * P / rho);
    }
    R rho = U[0], u = U[1] / rho, v = U[2] / rho;
    R P = (g - R(1.0)) * (U[3] - R(0.5) * rho * (u * u + v * v));
    return fabs(dir == 0 ? u : v) + sqrt(g * P / rho);
}

template <int KIND>
__host__ __device__ constexpr int kind_m() {
    return KIND == NPW_FLUX_EULER1D_ ? 3 : (KIND == NPW_FLUX_EULER2D_ ? 4 : 1);
}

// Lax-Friedrichs flux of one face, all M fields: h = 0.5 (f(a) + f(b) - alpha (b - a)).
template <typename R, int KIND, int M>
__device__ __forceinline__ void lf_flux(const R* a, const R* b, R alpha, const MethodParams& mp, int dir, R* h) {
    R fa[M], fb[M];
    phys_flux<R, KIND>(a, mp, dir, fa);
    phys_flux<R, KIND>(b, mp, dir, fb);
#pragma unroll
    for (int k = 0; k < M; ++k) h[k] = R(0.5) * (fa[k] + fb[k] - alpha * (b[k] - a[k]));
}

// ---------------------------------------------------------------------------------------
// Characteristic variant (1D Euler): Roe average of the two cells at the face, right
// eigenvectors R (columns) of dF/dU and their inverse in closed form,
//   L = [ (b2 + u/c)/2, -(b1 u + 1/c)/2, b1/2 ;  1 - b2, b1 u, -b1 ;  (b2 - u/c)/2, -(b1 u - 1/c)/2, b1/2 ]
// with b1 = (gamma - 1)/c^2, b2 = b1 u^2 / 2.
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ bool euler_eig(const R* UL, const R* UR, R gamma, R Rm[3][3], R Lm[3][3]) {
    R rl = UL[0], rr = UR[0];
    R ul = UL[1] / rl, ur = UR[1] / rr;
    R pl = (gamma - R(1.0)) * (UL[2] - R(0.5) * rl * ul * ul);
    R pr = (gamma - R(1.0)) * (UR[2] - R(0.5) * rr * ur * ur);
    R hl = (UL[2] + pl) / rl, hr = (UR[2] + pr) / rr;
    R sl = sqrt(rl), sr = sqrt(rr);
    R u = (sl * ul + sr * ur) / (sl + sr);
    R h = (sl * hl + sr * hr) / (sl + sr);
    R c2 = (gamma - R(1.0)) * (h - R(0.5) * u * u);
    if (!(c2 > R(0.0))) return false;
    R c = sqrt(c2);
    Rm[0][0] = R(1.0);
    Rm[0][1] = R(1.0);
    Rm[0][2] = R(1.0);
    Rm[1][0] = u - c;
    Rm[1][1] = u;
    Rm[1][2] = u + c;
    Rm[2][0] = h - u * c;
    Rm[2][1] = R(0.5) * u * u;
    Rm[2][2] = h + u * c;
    R b1 = (gamma - R(1.0)) / c2;
    R b2 = R(0.5) * b1 * u * u;
    R uc = u / c, ic = R(1.0) / c;
    Lm[0][0] = R(0.5) * (b2 + uc);
    Lm[0][1] = R(-0.5) * (b1 * u + ic);
    Lm[0][2] = R(0.5) * b1;
    Lm[1][0] = R(1.0) - b2;
    Lm[1][1] = b1 * u;
    Lm[1][2] = -b1;
    Lm[2][0] = R(0.5) * (b2 - uc);
    Lm[2][1] = R(-0.5) * (b1 * u - ic);
    Lm[2][2] = R(0.5) * b1;
    return true;
}

}  // namespace npw
