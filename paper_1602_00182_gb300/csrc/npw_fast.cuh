// npw_fast.cuh -- per-face / per-cell arithmetic of the mixed-precision path (NPW_FP32_MIXED).
//
// On GB300 a double-precision operation costs as much issue bandwidth as ~58 single-precision
// ones, so the mixed path keeps FP64 out of everything except the shape parameter:
//   * The monotone switch (Sec. 4) and the ENO stencil choice (Sec. 2) are decisions.  They are
//     taken from single-precision values with a rigorous forward error bound: a sign is used
//     only when |value| exceeds the bound, which makes it the sign of the exact quantity and
//     therefore the sign the double-precision evaluation gives; otherwise the decision is
//     recomputed in double precision.  The decisions are thus those of FP64 evaluation.
//   * The shape parameter eta of Table k3 (a ratio of two cancelling differences) is evaluated
//     either from the exactly computed differences as float pairs with a double-float quotient
//     (eta_eval 0, the default: within one float ulp plus ~2^-44 of the conditioning, no FP64
//     instruction) or in FP64 (eta_eval 1: FP64 numerator and denominator from the widened
//     averages, FP64 Newton quotient, within half an ulp plus 2^-52 of the conditioning).  Both
//     are rounded once to float for the perturbed coefficients c_rj + q_rj eta.  k = 2 (Table
//     k2) always takes the FP64 form.
//   * The WENO smoothness indicators beta_r (Jiang-Shu), the weights, candidates, flux and
//     update are single precision.
#pragma once
#include <cstdint>

#include "npw_device.cuh"
#include "npw_internal.h"

namespace npw {
namespace fast {

// float copies of the method parameters (rounded on the host)
struct FParams {
    float eps_weno, eps_M_f, eps_M_lo, eta_guard, eta_max;
    double eps_M, eta_guard_d;
    int scheme, rbf, monotone_switch, switch_variant, eta_eval;
};
__device__ __forceinline__ FParams fparams(const MethodParams& mp) {
    FParams f;
    f.eps_weno = mp.eps_weno_f;
    f.eps_M_f = mp.eps_M_f;
    f.eps_M_lo = mp.eps_M_lo_f;
    f.eta_guard = mp.eta_guard_f;
    f.eta_max = mp.eta_max_f;
    f.eps_M = mp.eps_M;
    f.eta_guard_d = mp.eta_guard;
    f.scheme = mp.scheme;
    f.rbf = mp.rbf;
    f.monotone_switch = mp.monotone_switch;
    f.switch_variant = mp.switch_variant;
    f.eta_eval = mp.eta_eval;
    return f;
}

constexpr float kU = 5.9604645e-08f;  // 2^-24, unit roundoff of float
constexpr float kE = 6.0f * kU;       // bound factor for short small-integer combinations
constexpr int kUncertain = 2;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// sign of the exact value v* given |v - v*| <= err: +1, -1, 0 (v == 0 exactly) or uncertain
__device__ __forceinline__ int csign(float v, float err) {
    if (v > err) return 1;
    if (v < -err) return -1;
    if (v == 0.0f && err == 0.0f) return 0;
    return kUncertain;
}

// Variant 0 of the switch from the neighbour differences d_j = w_{j+1} - w_j of the eta
// stencil.  In these terms 12 p'(-2) = 35 d0 - 34 d1 + 11 d2, 12 p'(2) = 11 d0 - 34 d1 + 35 d2,
// 12 p'(s) = 6 A s^2 + 6 B s + C with A = d0 - 2 d1 + d2, B = d2 - d0, C = -d0 + 14 d1 - d2; the
// vertex lies strictly inside iff 4|A| - |B| > 0, and sign(12 p'(vertex)) = sign(A) sign(2AC - 3B^2).
// Returns 1 (fires), 0 (does not) or -1 (not certain: decide in double precision).
__device__ __forceinline__ int switch_v0_cert(float d0, float d1, float d2) {
    const float a0 = fabsf(d0), a1 = fabsf(d1), a2 = fabsf(d2);
    const float A = fmaf(-2.f, d1, d0 + d2);
    const float eA = kE * fmaf(2.f, a1, a0 + a2);
    const float B = d2 - d0;
    const float eB = kE * (a0 + a2);
    const float C = fmaf(14.f, d1, -(d0 + d2));
    const float eC = kE * fmaf(14.f, a1, a0 + a2);
    const float aA = fabsf(A), aB = fabsf(B), aC = fabsf(C);
    // On the stencil (|s| <= 2), |6 A s^2 + 6 B s| <= 24 |A| + 12 |B|: where |C| reaches that,
    // p' never takes the sign opposite to C's (p' = 0 throughout when all three vanish), so it
    // cannot take both signs and the switch does not fire.  This decides most faces of smooth
    // data (|v'| above about 2 dx |v''|) and every constant stencil before the end values are
    // formed.
    if (aC - eC >= fmaf(24.f, aA + eA, 12.f * (aB + eB)) * (1.f + 4.f * kU)) return 0;
    const float Em = fmaf(35.f, d0, fmaf(-34.f, d1, 11.f * d2));
    const float Ep = fmaf(11.f, d0, fmaf(-34.f, d1, 35.f * d2));
    const int s1 = csign(Em, kE * fmaf(35.f, a0, fmaf(34.f, a1, 11.f * a2)));
    const int s2 = csign(Ep, kE * fmaf(11.f, a0, fmaf(34.f, a1, 35.f * a2)));
    if (s1 == kUncertain || s2 == kUncertain) return -1;
    // p' takes both signs at the two ends: non-monotone whatever the vertex does
    if ((s1 < 0 && s2 > 0) || (s1 > 0 && s2 < 0)) return 1;
    // With the vertex inside (|B| < 4|A|), |12 p'(vertex) - C| = 1.5 B^2 / |A| < 24 |A|.  If C
    // has the common sign of both ends and |C| exceeds that bound, p' keeps one sign on the
    // whole interval whether or not the vertex is inside (nearly linear data: A, B ~ 0).
    if (s1 == s2 && s1 != 0) {
        const int sC = csign(C, eC);
        if (sC == s1 && aC - eC > 24.f * (aA + eA) * (1.f + 4.f * kU)) return 0;
    }
    const int sD = csign(fmaf(4.f, aA, -aB), 4.f * eA + eB + kE * fmaf(4.f, aA, aB));
    if (sD == kUncertain) return -1;
    bool neg = s1 < 0 || s2 < 0, pos = s1 > 0 || s2 > 0;
    if (sD > 0) {
        const int sA = csign(A, eA);
        if (sA == kUncertain || sA == 0) return -1;
        const float G = fmaf(2.f * A, C, -3.f * B * B);
        const float eG = 2.f * (aA * eC + aC * eA + 3.f * eA * eC) + 3.f * (2.f * aB * eB + 3.f * eB * eB) +
                         kE * (2.f * aA * aC + 3.f * aB * aB);
        const int sG = csign(G, eG);
        if (sG == kUncertain) return -1;
        const int sV = sG * sA;
        neg = neg || sV < 0;
        pos = pos || sV > 0;
    }
    return (neg && pos) ? 1 : 0;
}

// eq. root_value on three cells with differences (da, db): ratio = (2 da - db) / (da - db);
// fires iff 0 < ratio < 3, i.e. sign(2da - db) = sign(da - db) = sign(da - 2db) != 0.
__device__ __forceinline__ int k2_cert(float da, float db) {
    const float a = fabsf(da), b = fabsf(db);
    const int sn = csign(fmaf(2.f, da, -db), kE * fmaf(2.f, a, b));
    const int st = csign(fmaf(-2.f, db, da), kE * fmaf(2.f, b, a));
    if (sn == kUncertain || st == kUncertain) return -1;
    if (sn == 0 || sn != st) return 0;  // the three signs cannot agree (nearly linear data)
    const int sd = csign(da - db, kE * (a + b));
    if (sd == kUncertain) return -1;
    return (sd != 0 && sn == sd) ? 1 : 0;
}

__device__ __forceinline__ bool switch_fires_f(float w0, float w1, float w2, float w3, int variant) {
    const float d0 = w1 - w0, d1 = w2 - w1, d2 = w3 - w2;
    int c;
    if (variant == 1) {
        const int c1 = k2_cert(d0, d1);
        const int c2 = k2_cert(d1, d2);
        c = (c1 == 1 || c2 == 1) ? 1 : ((c1 == 0 && c2 == 0) ? 0 : -1);
    } else {
        c = switch_v0_cert(d0, d1, d2);
    }
    if (c >= 0) return c == 1;
    return switch_fires<double>((double)w0, (double)w1, (double)w2, (double)w3, variant);
}

// a - 2 b + c = h + l + eg exactly, by error-free transformations (two-sum; 2 b is exact), with
// |l| <= u |h| and |eg| <= u^2 (|a| + 2|b| + |c|) roughly
__device__ __forceinline__ void sdiff_exact(float a, float b, float c, float& h, float& l, float& eg) {
    float s, e, t, f, g;
    two_sum(a, c, s, e);
    two_sum(s, -2.f * b, t, f);
    two_sum(f, e, g, eg);
    two_sum(t, g, h, l);
}
// sign of h + l + eg as above: +1 or -1, or 0 when not certain
__device__ __forceinline__ float sdiff_sign(float h, float eg) {
    if (h != 0.0f) return fabsf(h) * (1.0f - 2.0f * kU) > fabsf(eg) ? copysignf(1.0f, h) : 0.0f;
    return eg >= 0.0f ? 1.0f : -1.0f;  // l = 0 and the value is eg exactly
}
// The second step of the ENO choice on second differences X = a - 2b + c, Y = p - 2q + r whose
// difference in magnitude is a third difference below float resolution on fine smooth grids:
// 1 where |Y| > |X|, 0 where not, -1 where not certain.  |Y| - |X| = zh + zl + (em + ez +
// sY gY - sX gX) exactly, the bracket bounded by R; a decision is returned only where |zh + zl|
// exceeds R plus a bound on the FP64 evaluation's own error (2^-52 (|a| + 2|b| + |c| + |p| +
// 2|q| + |r|), doubled), so that it is the exact decision and also that of the FP64 evaluation.
// An exact tie (every term exact, zh + zl = 0) is decided as a tie (|X| < |Y| is false) where
// the magnitudes span at most 2^26, so that the FP64 evaluation is exact as well.
__device__ __forceinline__ int sdiff_abs_less(float a, float b, float c, float p, float q, float r) {
    float hx, lx, gx, hy, ly, gy;
    sdiff_exact(a, b, c, hx, lx, gx);
    sdiff_exact(p, q, r, hy, ly, gy);
    const float sx = sdiff_sign(hx, gx), sy = sdiff_sign(hy, gy);
    if (sx == 0.0f || sy == 0.0f) return -1;
    float zh, ze, m, em, zl, ez;
    two_sum(sy * hy, -sx * hx, zh, ze);
    two_sum(sy * ly, -sx * lx, m, em);
    two_sum(ze, m, zl, ez);
    const float w = zh + zl;
    const float R = (fabsf(em) + fabsf(ez)) + (fabsf(gx) + fabsf(gy));
    const float S = ((fabsf(a) + fabsf(c)) + 2.f * fabsf(b)) + ((fabsf(p) + fabsf(r)) + 2.f * fabsf(q));
    const float fp64 = S * 0x1p-50f;
    if (R == 0.0f) {  // |Y| - |X| = zh + zl exactly: w has its sign, and is 0 only at a tie
        if (w != 0.0f) return fabsf(w) * (1.0f - kU) > fp64 ? (w > 0.0f ? 1 : 0) : -1;
        const float t[6] = {fabsf(a), 2.f * fabsf(b), fabsf(c), fabsf(p), 2.f * fabsf(q), fabsf(r)};
        float mx = 0.0f, mn = INFINITY;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (t[k] != 0.0f) {
                mx = fmaxf(mx, t[k]);
                mn = fminf(mn, t[k]);
            }
        return (mx == 0.0f || mx <= mn * 0x1p26f) ? 0 : -1;
    }
    return fabsf(w) * (1.0f - kU) > (R * (1.0f + 8.0f * kU) + fp64) + 0x1p-140f ? (w > 0.0f ? 1 : 0) : -1;
}

// the ENO choice where the float test of its first (s1 = kUncertain) or second step is not
// certain, out of line: the second step from the second differences to a few units of u^2,
// else the FP64 evaluation
__device__ __forceinline__ int eno_choice_rest(float c0, float c1, float c2, float c3, float c4, int s1) {
    if (s1 != kUncertain) {
        const int x = s1 > 0 ? sdiff_abs_less(c0, c1, c2, c1, c2, c3) : sdiff_abs_less(c1, c2, c3, c2, c3, c4);
        if (x >= 0) {
            if (s1 > 0) return x ? 2 : 1;
            return x ? 1 : 0;
        }
    }
    return eno_choice<double>((double)c0, (double)c1, (double)c2, (double)c3, (double)c4);
}

// ENO stencil choice with the same certification (see eno_choice for the rule)
__device__ __forceinline__ int eno_choice_f(float c0, float c1, float c2, float c3, float c4) {
    const float dm = c1 - c0, dl = c2 - c1, dr = c3 - c2, dp = c4 - c3;
    const float al = fabsf(dl), ar = fabsf(dr);
    const int s1 = csign(ar - al, kE * (al + ar));
    if (s1 != kUncertain) {
        float ddl, ddr, e;
        if (s1 > 0) {  // left extension: cells {i-1, i}
            ddl = dl - dm;
            ddr = dr - dl;
            e = kE * (fabsf(dm) + 2.f * al + ar);
        } else {
            ddl = dr - dl;
            ddr = dp - dr;
            e = kE * (al + 2.f * ar + fabsf(dp));
        }
        const float adl = fabsf(ddl), adr = fabsf(ddr);
        const int s2 = csign(adr - adl, e + kE * (adl + adr));
        if (s2 != kUncertain) {
            if (s1 > 0) return s2 > 0 ? 2 : 1;
            return s2 > 0 ? 1 : 0;
        }
    }
    return eno_choice_rest(c0, c1, c2, c3, c4, s1);
}

// ---------------------------------------------------------------------------------------
// Shape parameter.  num = w0 - 3 w1 + 3 w2 - w3, den = w0 - 15 w1 + 15 w2 - w3 (Table k3).
// ---------------------------------------------------------------------------------------
// IEEE 754 format changes done with integer operations only, without a branch that could
// hold a hardware conversion, so that none of them occupies the FP64 pipe (on GB300 a
// float<->double conversion takes FP64-pipe slots like an FP64 add).
//
// widen: binary32 -> binary64, exact.  A normal number keeps sign and fraction (shifted left
// by 52 - 23 = 29 bits) and its exponent is rebiased by 1023 - 127 = 896.  A subnormal f 2^-149
// is normalised with a leading-zero count (its leading one at bit p = 31 - clz(f) gives the
// exponent p - 149, biased 905 - clz(f)); zero stays a signed zero (clz = 32 shifts f out);
// infinities and NaNs keep exponent 2047 and their fraction.
__device__ __forceinline__ double widen(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xFFu;
    uint32_t f = b & 0x7FFFFFu, E;
    if (e == 0u) {
        const int lz = __clz(f);
        E = f != 0u ? (uint32_t)(905 - lz) : 0u;
        f = (f << ((lz - 8) & 31)) & 0x7FFFFFu;
    } else {
        E = e == 255u ? 2047u : e + 896u;
    }
    return __hiloint2double((int)((b & 0x80000000u) | (E << 20) | (f >> 3)), (int)(f << 29));
}

// Zero or a normal number (neither subnormal, infinite nor NaN).
__device__ __forceinline__ bool zero_or_normal(float x) {
    const uint32_t t = __float_as_uint(x) & 0x7FFFFFFFu;
    return (t == 0u) | (t - 0x00800000u < 0x7F000000u);
}

// widen for a zero or normal x (the common case): the exponent field is rebiased in place.
__device__ __forceinline__ double widen_nz(float x) {
    const uint32_t b = __float_as_uint(x), t = b & 0x7FFFFFFFu;
    const uint32_t hi = t != 0u ? (t >> 3) + (896u << 20) : 0u;
    return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)(b << 29));
}
template <bool NZ>
__device__ __forceinline__ double widen_as(float x) {
    if constexpr (NZ)
        return widen_nz(x);
    else
        return widen(x);
}

// narrow: a finite binary64 value to the nearest binary32 (ties away from zero: the fraction
// is rounded by adding half a unit of bit 29 and truncating; a carry out of the fraction
// raises the exponent, which is the correct result).  Magnitudes below the float normal range
// (2^-126) give a signed zero and magnitudes beyond it a signed infinity.  Callers pass
// finite values only.
__device__ __forceinline__ float narrow(double v) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const uint64_t m = (b & 0x7FFFFFFFFFFFFFFFull) + (1ull << 28);
    const uint32_t E = (uint32_t)(m >> 52);
    // bits 29..60 of m: the 23 fraction bits and the low 9 exponent bits; subtracting 896 from
    // the exponent field modulo 2^9 leaves E - 896, exact for E in [897, 1150]
    uint32_t f = (uint32_t)(m >> 29) - (896u << 23);
    f = E < 897u ? 0u : (E > 1150u ? 0x7F800000u : f);
    return __uint_as_float(f | ((uint32_t)(b >> 32) & 0x80000000u));
}

// seed_f: a binary64 value whose magnitude lies in [2^-99, 2^99) truncated to binary32
// (relative error below 2^-23), for a reciprocal seed; false outside that range (zero,
// subnormal, huge, infinite or NaN), where the caller divides in double instead.
__device__ __forceinline__ bool seed_f(double v, float* out) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const uint32_t E = (uint32_t)(b >> 52) & 0x7FFu;
    *out = __uint_as_float(((uint32_t)(b >> 29) - (896u << 23)) | ((uint32_t)(b >> 32) & 0x80000000u));
    return E - 924u < 198u;
}


// every argument is +0 or -0: a stencil of zero cell averages (a field at rest, such as the
// momentum of a quiescent gas), whose denominator and guard threshold are both exactly 0, so the
// guard (|den| <= eta_guard * magnitudes) holds in any precision
__device__ __forceinline__ bool all_zero(float a, float b, float c, float d = 0.0f) {
    return ((__float_as_uint(a) | __float_as_uint(b) | __float_as_uint(c) | __float_as_uint(d)) & 0x7FFFFFFFu) == 0u;
}

// The rare branches below are kept out of line: a call is executed only when taken, while an
// inlined short branch may be turned into predicated instructions that take issue slots of
// the FP64 pipe on every evaluation.
static __device__ __noinline__ float div_rn_f(double num, double den) { return (float)(num / den); }

// Numerator a + 3b and denominator a + 15b (a = w0 - w3, b = w2 - w1) as unevaluated float
// pairs.  The differences are exact two_sum pairs, the products 3 bh and 15 bh are split
// exactly by fma and the leading terms are added with two_sum; the remaining small terms
// (each within 2^-23 of a leading term) are summed in float, so each pair is within ~2^-47 of
// its largest term.
__device__ __forceinline__ void eta_pairs(float w0, float w1, float w2, float w3, float& nh, float& nl, float& dh,
                                          float& dl) {
    float ah, al, bh, bl;
    two_sum(w0, -w3, ah, al);  // w0 - w3 = ah + al exactly
    two_sum(w2, -w1, bh, bl);  // w2 - w1 = bh + bl exactly
    const float p3 = 3.f * bh, p3e = fmaf(3.f, bh, -p3);
    const float p15 = 15.f * bh, p15e = fmaf(15.f, bh, -p15);
    float ne, de;
    two_sum(ah, p3, nh, ne);
    two_sum(ah, p15, dh, de);
    nl = ne + (al + (p3e + 3.f * bl));
    dl = de + (al + (p15e + 15.f * bl));
}

// FP64 evaluation of the Table k3 shape parameter from the float cell averages.  The four
// averages are widened exactly (integer format changes), a = w0 - w3 and b = w2 - w1 are FP64
// differences (exact unless the exponents differ by more than 29), and num = a + 3 b and
// den0 = a + 15 b are single-rounding multiply-adds, den = den0 + eps_M.  Numerator and
// denominator thus carry only the rounding of an FP64 evaluation of the undivided differences
// (2^-53 relative to |a| + 3|b| and |a| + 15|b|), however much they cancel.  The quotient is the
// Newton-Raphson reciprocal iteration in double: the seed r0 is the fast float reciprocal of den
// truncated to float (|1 - den r0| < 2^-21); with e = 1 - den r0 (one multiply-add) and
// q0 = num r0, num r0 (1 + e) = (num / den)(1 - e^2) is within 2^-41 of num / den before the
// rounding to float.  FP64-pipe instructions: 2 adds (a, b), 2 multiply-adds (num, den0), 1 add
// (eps_M), 1 multiply and 2 multiply-adds (the quotient).
// The guard compares |den0| with eta_guard (|w0| + 15|w1| + 15|w2| + |w3|): decided from the
// float product where it is more than 2^-20 away (the float value is within 6 u of the exact
// one), else by the FP64 path's own expression, out of line.
// NZ: the four averages are zero or normal (the cheaper widening applies); the other case
// (subnormal, infinite or NaN averages) takes the same arithmetic out of line.
static __device__ __noinline__ bool guard_exact(float w0, float w1, float w2, float w3, double eta_guard) {
    // (an all-zero stencil never gets here: see all_zero)
    const double v0 = widen(w0), v1 = widen(w1), v2 = widen(w2), v3 = widen(w3);
    const double den0 = v0 - 15.0 * v1 + 15.0 * v2 - v3;
    return fabs(den0) <= eta_guard * (fabs(v0) + 15.0 * fabs(v1) + 15.0 * fabs(v2) + fabs(v3));
}
template <bool NZ>
__device__ __forceinline__ float eta_quot(float w0, float w1, float w2, float w3, const FParams& fp, float guard,
                                          uint32_t* fl) {
    const double a = widen_as<NZ>(w0) - widen_as<NZ>(w3);
    const double b = widen_as<NZ>(w2) - widen_as<NZ>(w1);
    const double den0 = fma(15.0, b, a);
    if (fp.eta_guard > 0.0f) {
        // below 2^-100 the float threshold may have lost precision (subnormal products): exact path
        const double d0 = fabs(den0);
        bool zero;
        if (guard >= 0x1p-100f) {
            const double g = widen_nz(guard);
            zero = d0 <= g * (1.0 + 0x1p-20) && (d0 < g * (1.0 - 0x1p-20) || guard_exact(w0, w1, w2, w3, fp.eta_guard_d));
        } else {
            zero = all_zero(w0, w1, w2, w3) || guard_exact(w0, w1, w2, w3, fp.eta_guard_d);
        }
        if (zero) {
            *fl |= FL_ZERO_GUARD;
            return 0.0f;
        }
    }
    const double num = fma(3.0, b, a);
    const double den = den0 + fp.eps_M;
    float denf;
    if (!seed_f(den, &denf)) return div_rn_f(num, den);
    const double r0 = widen_nz(__fdividef(1.0f, denf));  // |r0| in (2^-99, 2^99]: normal
    const double q0 = num * r0;
    const double e = fma(-den, r0, 1.0);
    return narrow(fma(q0, e, q0));
}
static __device__ __noinline__ float eta_quot_any(float w0, float w1, float w2, float w3, const FParams& fp,
                                                  float guard, uint32_t* fl) {
    return eta_quot<false>(w0, w1, w2, w3, fp, guard, fl);
}
__device__ __forceinline__ float eta_fp64(float w0, float w1, float w2, float w3, const FParams& fp, float guard,
                                          uint32_t* fl) {
    if (!(zero_or_normal(w0) & zero_or_normal(w1) & zero_or_normal(w2) & zero_or_normal(w3)))
        return eta_quot_any(w0, w1, w2, w3, fp, guard, fl);
    return eta_quot<true>(w0, w1, w2, w3, fp, guard, fl);
}

// Double-float evaluation (eta_eval 0, no FP64 instruction): the pairs of eta_pairs, eps_M added
// by two_sum, renormalised, and the double-float quotient (one correction of the float
// quotient).  Its numerator and denominator are within ~2^-47 of the magnitudes of their terms
// (|a| + 3|b|, |a| + 15|b|), against 2^-53 for the FP64 evaluation: where they cancel strongly
// the quotient is correspondingly less accurate than eta_eval 1.
__device__ __forceinline__ float eta_doublefloat(float w0, float w1, float w2, float w3, const FParams& fp,
                                                 float guard, uint32_t* fl) {
    const float eps_M = fp.eps_M_f;
    float nh, nl, dh, dl;
    eta_pairs(w0, w1, w2, w3, nh, nl, dh, dl);
    if (fp.eta_guard > 0.0f) {  // certified as in eta_quot: exact where the float test is too close
        // the common case first: a denominator clearly above the threshold (then the averages
        // are not all zero, since an all-zero stencil has a zero threshold)
        const float d0 = fabsf(dh + dl);
        const bool clear = guard >= 0x1p-100f && d0 > guard * (1.0f + 0x1p-19f);
        const bool zero = !clear && (all_zero(w0, w1, w2, w3) ||
                                     (guard >= 0x1p-100f && d0 <= guard * (1.0f - 0x1p-19f)
                                          ? true
                                          : ((guard < 0x1p-100f || d0 <= guard * (1.0f + 0x1p-19f)) &&
                                             guard_exact(w0, w1, w2, w3, fp.eta_guard_d))));
        if (zero) {
            *fl |= FL_ZERO_GUARD;
            return 0.0f;
        }
    }
    float t;
    two_sum(dh, eps_M, dh, t);
    dl += t;
    // renormalise the pairs
    float s;
    two_sum(nh, nl, s, nl);
    nh = s;
    two_sum(dh, dl, s, dl);
    dh = s;
    if (dh == 0.0f) return nh / dh;  // same 0/0 or inf behaviour as the plain quotient
    // double-float quotient (nh + nl) / (dh + dl): q1 needs only a few ulps (the exact residual r
    // corrects it), so where |dh| lies in [2^-125, 2^125] the fast reciprocal division (within 2
    // ulp) serves for q1 and for the small correction q2; elsewhere the correctly rounded one
    const float adh = fabsf(dh);
    const bool fast_div = adh >= 0x1p-125f && adh <= 0x1p125f;
    const float q1 = fast_div ? __fdividef(nh, dh) : nh / dh;
    const float p = q1 * dh;
    const float pe = fmaf(q1, dh, -p);
    const float r = ((nh - p) - pe) + fmaf(-q1, dl, nl);
    const float q2 = fast_div ? __fdividef(r, dh) : r / dh;
    return q1 + q2;
}

// The guard sets eta = 0 where the denominator is below eta_guard times the sum of the
// magnitudes of its terms: such a denominator is round-off of the cell averages, and the
// quotient would be noise amplified by 1/eps_M.
__device__ __forceinline__ float eta_eval(float w0, float w1, float w2, float w3, const FParams& fp, uint32_t* fl) {
    const float guard = fp.eta_guard * (fabsf(w0) + 15.f * fabsf(w1) + 15.f * fabsf(w2) + fabsf(w3));
    return fp.eta_eval == 0 ? eta_doublefloat(w0, w1, w2, w3, fp, guard, fl)
                            : eta_fp64(w0, w1, w2, w3, fp, guard, fl);
}

// eta of the face whose eta stencil is (w0..w3), 0 where the switch fires; flag bits: FL_SWITCH,
// FL_ZERO_GUARD, FL_ZERO_BOUND
__device__ __forceinline__ float face_eta(float w0, float w1, float w2, float w3, const FParams& fp,
                                          uint32_t* flag) {
    if (fp.scheme != NPW_RBF_ENO_ && fp.scheme != NPW_RBF_WENO_) return 0.0f;
    if (fp.monotone_switch && switch_fires_f(w0, w1, w2, w3, fp.switch_variant)) {
        *flag |= FL_SWITCH;
        return 0.0f;
    }
    const float e = eta_eval(w0, w1, w2, w3, fp, flag);
    if (fp.eta_max > 0.0f && fabsf(e) > fp.eta_max) {
        *flag |= FL_ZERO_BOUND;
        return 0.0f;
    }
    return e;
}

// ---------------------------------------------------------------------------------------
// One cell: c[0..4] = cells i-2..i+2; eta_r = eta of face i+1/2, eta_l of face i-1/2.
// Writes v^-_{i+1/2} and v^+_{i-1/2}.  Returns the ENO stencil (0 for WENO).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int cell_recon(const float* c, float eta_r, float eta_l, const FParams& mp,
                                          float* vm, float* vp) {
    float cm[3], cp[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float sm = 0.0f, sp = 0.0f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float x = c[2 - r + j];
            sm = fmaf(fmaf(pert_coef<float>(mp.rbf, r + 1, j), eta_r, poly_coef<float>(r + 1, j)), x, sm);
            sp = fmaf(fmaf(pert_coef<float>(mp.rbf, r, j), eta_l, poly_coef<float>(r, j)), x, sp);
        }
        cm[r] = sm;
        cp[r] = sp;
    }
    if (mp.scheme == NPW_ENO_ || mp.scheme == NPW_RBF_ENO_) {
        const int r = eno_choice_f(c[0], c[1], c[2], c[3], c[4]);
        *vm = r == 0 ? cm[0] : (r == 1 ? cm[1] : cm[2]);
        *vp = r == 0 ? cp[0] : (r == 1 ? cp[1] : cp[2]);
        return r;
    }
    // Jiang-Shu indicators (single precision), shared by both faces of the cell.  The weights
    // use the fast float division (within 2 ulp for divisors in [2^-126, 2^126]): beta + eps is
    // at least eps_weno and is clamped at 1e18 (differences of the cell averages near 1e9, far
    // beyond any workload), so every divisor below stays inside that range.
    constexpr float kBeMax = 1e18f;
    float a, b, inv[3];
    const float eps = mp.eps_weno;
    a = c[2] - 2.f * c[3] + c[4];
    b = fmaf(3.f, c[2], fmaf(-4.f, c[3], c[4]));
    float be = fminf(fmaf(13.f / 12.f * a, a, 0.25f * b * b) + eps, kBeMax);
    inv[0] = __fdividef(1.0f, be * be);
    a = c[1] - 2.f * c[2] + c[3];
    b = c[1] - c[3];
    be = fminf(fmaf(13.f / 12.f * a, a, 0.25f * b * b) + eps, kBeMax);
    inv[1] = __fdividef(1.0f, be * be);
    a = c[0] - 2.f * c[1] + c[2];
    b = fmaf(-4.f, c[1], fmaf(3.f, c[2], c[0]));
    be = fminf(fmaf(13.f / 12.f * a, a, 0.25f * b * b) + eps, kBeMax);
    inv[2] = __fdividef(1.0f, be * be);
    // v^-: d = (3/10, 3/5, 1/10); v^+: d = (1/10, 3/5, 3/10)
    const float am0 = 0.3f * inv[0], am1 = 0.6f * inv[1], am2 = 0.1f * inv[2];
    const float ap0 = 0.1f * inv[0], ap1 = 0.6f * inv[1], ap2 = 0.3f * inv[2];
    *vm = __fdividef(fmaf(am0, cm[0], fmaf(am1, cm[1], am2 * cm[2])), am0 + am1 + am2);
    *vp = __fdividef(fmaf(ap0, cp[0], fmaf(ap1, cp[1], ap2 * cp[2])), ap0 + ap1 + ap2);
    return 0;
}

// Face form (used where the cells of a face see different data, as in the characteristic
// variant): w[0..5] = cells i-2..i+3 of face i+1/2.  The neighbouring faces' eta values are
// not needed: v^- uses this face's eta, v^+ of cell i+1 too.
// ---------------------------------------------------------------------------------------
// k = 2 in mixed precision.  The switch (eq. root_value on the cell's stencil) and the ENO2
// choice are certified from float differences with an FP64 fallback, as for k = 3; the shape
// parameter of each face value is evaluated in FP64 from the float cell averages (the
// literal formula of Table k2, identical to the FP64 path on the same data); candidates and
// WENO3 weights are float.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ bool switch_k2_f(float c0, float c1, float c2) {
    const int c = k2_cert(c1 - c0, c2 - c1);
    if (c >= 0) return c == 1;
    return k2_ratio_fires<double>((double)c0, (double)c1, (double)c2);
}

__device__ __forceinline__ int eno2_choice_f(float c0, float c1, float c2) {
    const float al = fabsf(c1 - c0), ar = fabsf(c2 - c1);
    const int s = csign(ar - al, kE * (al + ar));
    if (s != kUncertain) return s > 0 ? 1 : 0;
    return fabs((double)c1 - (double)c0) < fabs((double)c2 - (double)c1) ? 1 : 0;
}

// value of cell i (c[0..2] = cells i-1..i+1) at its right (side 0) or left (side 1) face;
// eta_c for the central row, eta_x for the extrapolating ones
__device__ __forceinline__ float cell_value_k2_f(const float* c, int side, float eta_c, float eta_x, const FParams& fp,
                                                 int* r_out) {
    float cand[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = (side == 0) ? r : r - 1;
        const float eta = row == 0 ? eta_c : eta_x;
        const float k0 = fmaf(pert2_coef<float>(fp.rbf, row + 1, 0), eta, poly2_coef<float>(row + 1, 0));
        const float k1 = fmaf(pert2_coef<float>(fp.rbf, row + 1, 1), eta, poly2_coef<float>(row + 1, 1));
        cand[r] = fmaf(k0, c[1 - r], k1 * c[2 - r]);
    }
    if (fp.scheme == NPW_ENO_ || fp.scheme == NPW_RBF_ENO_) {
        const int r = eno2_choice_f(c[0], c[1], c[2]);
        *r_out = r;
        return r == 0 ? cand[0] : cand[1];
    }
    *r_out = 0;
    constexpr float kBeMax = 1e18f;  // keeps the fast division in range (see cell_recon)
    const float g0 = c[2] - c[1], g1 = c[1] - c[0];
    const float be0 = fminf(fmaf(g0, g0, fp.eps_weno), kBeMax), be1 = fminf(fmaf(g1, g1, fp.eps_weno), kBeMax);
    const float a0 = __fdividef(side == 0 ? 2.f / 3.f : 1.f / 3.f, be0 * be0);
    const float a1 = __fdividef(side == 0 ? 1.f / 3.f : 2.f / 3.f, be1 * be1);
    return __fdividef(fmaf(a0, cand[0], a1 * cand[1]), a0 + a1);
}

// Both shape parameters of one face value of a k = 2 cell (the central row's and the
// extrapolating rows'), in FP64 from the float cell averages c[0..2] = cells i-1..i+1, with
// a, b, d the cells beside, at and across from the face (Table k2; the transverse term of the
// 5-cell cross of Sec. 6 enters the numerators).
//   * The guard of R12 compares |den0| with eta_guard (|a| + 5|b| + 2|d|).  It is first taken
//     in float with a bound on the rounding of both sides (each below 3u of the magnitude sum,
//     and the double evaluation within 2^-52 of it): only a float margin smaller than that
//     bound sends the test to double, where it is the FP64 path's expression, so the outcome
//     is the FP64 path's.
//   * The averages are widened exactly; the numerator -a + 2b - d is 2b - (a + d) by one add and
//     one multiply-add, the denominator -a + 5b + 2d by two multiply-adds plus eps_M: the
//     rounding of an FP64 evaluation of the undivided differences, however much they cancel.
//   * One reciprocal serves both quotients: r0, the fast float reciprocal of den truncated to
//     float (|1 - den r0| < 2^-21), and e = 1 - den r0; each quotient is q0 (1 + e) with
//     q0 = num r0, within 2^-41 of num / den.
//   * The factor 2 of the multiquadric row is applied to the rounded float value (exact).
// FP64-pipe instructions per face value: 5 for numerator and denominator, 1 for e and 2 per
// quotient (on the cross, 2 more for the two numerators and 2 for the second quotient).
template <bool NZ>
__device__ __forceinline__ void eta_k2_quot(float af, float bf, float df, double trans, const FParams& fp, float* ec,
                                            float* ex, uint32_t* fl) {
    const double a = widen_as<NZ>(af), b = widen_as<NZ>(bf), d = widen_as<NZ>(df);
    const double base = fma(2.0, b, -(a + d));
    const double den = fma(5.0, b, fma(2.0, d, -a)) + fp.eps_M;
    float denf, vc, vx;
    if (seed_f(den, &denf)) {
        const double r0 = widen_nz(__fdividef(1.0f, denf));
        const double e = fma(-den, r0, 1.0);
        const double nc = trans == 0.0 ? base : fma(-0.25, trans, base);
        const double qc = nc * r0;
        vc = narrow(fma(qc, e, qc));
        if (trans == 0.0) {
            vx = vc;
        } else {
            const double qx = fma(0.125, trans, base) * r0;
            vx = narrow(fma(qx, e, qx));
        }
    } else {
        vc = div_rn_f(fma(-0.25, trans, base), den);
        vx = trans == 0.0 ? vc : div_rn_f(fma(0.125, trans, base), den);
    }
    if (fp.rbf != NPW_RBF_GA_) {
        vc *= 2.0f;
        vx *= 2.0f;
    }
    const float bound = fp.eta_max;
    const bool zc = bound > 0.0f && fabsf(vc) > bound, zx = bound > 0.0f && fabsf(vx) > bound;
    *ec = zc ? 0.0f : vc;
    *ex = zx ? 0.0f : vx;
    if (zc | zx) *fl |= FL_ZERO_BOUND;
}
static __device__ __noinline__ void eta_k2_quot_any(float af, float bf, float df, double trans, const FParams& fp,
                                                    float* ec, float* ex, uint32_t* fl) {
    eta_k2_quot<false>(af, bf, df, trans, fp, ec, ex, fl);
}
// fl: FL_ZERO_GUARD / FL_ZERO_BOUND where the guard / the bound set a shape parameter to 0
__device__ __forceinline__ void eta_k2_pair(const float* cf, int side, double trans, const MethodParams& mp,
                                            const FParams& fp, float* ec, float* ex, uint32_t* fl) {
    const float af = side == 0 ? cf[0] : cf[2], bf = cf[1], df = side == 0 ? cf[2] : cf[0];
    *ec = *ex = 0.0f;
    if (fp.eta_guard > 0.0f) {
        const float magf = (fabsf(af) + 5.0f * fabsf(bf)) + 2.0f * fabsf(df);
        const float den0f = fmaf(2.0f, df, fmaf(5.0f, bf, -af));
        const float gm = fp.eta_guard * magf;
        if (all_zero(af, bf, df)) {
            *fl |= FL_ZERO_GUARD;
            return;
        }
        if (!(magf >= 0x1p-90f && fabsf(den0f) > gm + kE * magf * (1.0f + fp.eta_guard))) {
            const double a = widen(af), b = widen(bf), d = widen(df);
            if (fabs((-a + 5.0 * b) + 2.0 * d) <= mp.eta_guard * ((fabs(a) + 5.0 * fabs(b)) + 2.0 * fabs(d))) {
                *fl |= FL_ZERO_GUARD;
                return;
            }
        }
    }
    if (zero_or_normal(af) & zero_or_normal(bf) & zero_or_normal(df))
        eta_k2_quot<true>(af, bf, df, trans, fp, ec, ex, fl);
    else
        eta_k2_quot_any(af, bf, df, trans, fp, ec, ex, fl);
}

// Decisions of a k = 2 cell, as returned by cell_recon_k2: FL_SWITCH (the cell's switch fired:
// both its shape parameters are 0), FL_ZERO_GUARD / FL_ZERO_BOUND for the side-0 (v^-) value and
// the same bits shifted by K2_SIDE1 for the side-1 (v^+) value; 0 for schemes without eta.
constexpr int K2_SIDE1 = 8;
constexpr uint32_t K2_EVAL = 0x10000u;  // the cell's shape parameters were evaluated

// Both face values of one k = 2 cell (c3 = cells i-1..i+1, trans its transverse second
// difference or 0): v^- at its right face and v^+ at its left face, with the arithmetic that
// face_field_k2 gives them face by face.  Returns the cell's decision bits.
__device__ __forceinline__ uint32_t cell_recon_k2(const float* c3, double trans, const MethodParams& mp0,
                                                  const FParams& fp, float* vm, float* vp) {
    float e0c = 0.0f, e0x = 0.0f, e1c = 0.0f, e1x = 0.0f;
    uint32_t d = 0, f0 = 0, f1 = 0;
    if (fp.scheme == NPW_RBF_ENO_ || fp.scheme == NPW_RBF_WENO_) {
        if (fp.monotone_switch && switch_k2_f(c3[0], c3[1], c3[2])) {
            d = FL_SWITCH;
        } else {
            eta_k2_pair(c3, 0, trans, mp0, fp, &e0c, &e0x, &f0);
            eta_k2_pair(c3, 1, trans, mp0, fp, &e1c, &e1x, &f1);
            d = K2_EVAL | f0 | (f1 << K2_SIDE1);
        }
    }
    int r;
    *vm = cell_value_k2_f(c3, 0, e0c, e0x, fp, &r);
    *vp = cell_value_k2_f(c3, 1, e1c, e1x, fp, &r);
    return d;
}

// counts of one face value of a k = 2 cell from its decision bits (side 0: v^-, 1: v^+)
__device__ __forceinline__ void count_k2(EtaCount& c, uint32_t d, int side) {
    c.sw += d & FL_SWITCH;
    c.ev += d >> 16;
    const uint32_t z = side ? (d >> K2_SIDE1) : d;
    c.guard += (z >> 6) & 1u;
    c.bound += (z >> 7) & 1u;
}

// tl, tr: transverse second differences of the two cells (the 5-cell cross of Sec. 6; 0 on a
// line), taken in double from the float cell averages like the rest of the shape parameter
__device__ __forceinline__ uint32_t face_field_k2(const float* w, const MethodParams& mp0, float* vm, float* vp,
                                                  double tl, double tr, float* eta_out) {
    const FParams fp = fparams(mp0);
    uint32_t fl = 0;
    float el = 0.0f, er = 0.0f, elx = 0.0f, erx = 0.0f;
    if (fp.scheme == NPW_RBF_ENO_ || fp.scheme == NPW_RBF_WENO_) {
        if (fp.monotone_switch && switch_k2_f(w[1], w[2], w[3]))
            fl |= FL_SWITCH;
        else
            eta_k2_pair(w + 1, 0, tl, mp0, fp, &el, &elx, &fl);
        uint32_t zr = 0;
        if (fp.monotone_switch && switch_k2_f(w[2], w[3], w[4]))
            fl |= FL_SWITCH_R_K2;
        else
            eta_k2_pair(w + 2, 1, tr, mp0, fp, &er, &erx, &zr);
        fl |= zr << 2;  // FL_ZERO_GUARD_R_K2, FL_ZERO_BOUND_R_K2
    }
    int rl = 0, rr = 0;
    *vm = cell_value_k2_f(w + 1, 0, el, elx, fp, &rl);
    *vp = cell_value_k2_f(w + 2, 1, er, erx, fp, &rr);
    if (eta_out) *eta_out = el;
    return fl | (uint32_t(rl & 1) << 2) | (uint32_t(rr & 1) << 4);
}

// eta_out (may be NULL): the face's shape parameter as used (k = 2: that of v^-, central row)
__device__ __forceinline__ uint32_t face_field(const float* w, const MethodParams& mp0, float* vm, float* vp,
                                               double tl = 0.0, double tr = 0.0, float* eta_out = nullptr) {
    if (mp0.k == 2) return face_field_k2(w, mp0, vm, vp, tl, tr, eta_out);
    uint32_t fl = 0;
    const FParams mp = fparams(mp0);
    const float eta = face_eta(w[1], w[2], w[3], w[4], mp, &fl);
    float dummy;
    const int rl = cell_recon(w, eta, eta, mp, vm, &dummy);
    const int rr = cell_recon(w + 1, eta, eta, mp, &dummy, vp);
    if (eta_out) *eta_out = eta;
    return fl | (uint32_t(rl & 3) << 2) | (uint32_t(rr & 3) << 4);
}

}  // namespace fast

// the literal double-precision arithmetic for R = double, the mixed path for R = float
template <typename R, typename D>
__device__ __forceinline__ uint32_t face_field_any(const R* w, const MethodParams& mp, R* vm, R* vp, D tl = D(0.0),
                                                   D tr = D(0.0), R* eta_out = nullptr) {
    if constexpr (sizeof(R) == sizeof(float)) {
        return fast::face_field(w, mp, vm, vp, tl, tr, eta_out);
    } else {
        return face_field<R, D>(w, mp, vm, vp, R(tl), R(tr), eta_out);
    }
}

// All M fields at one face from the 6 x M stencil W[j*M + k] (cells i-2..i+3).  For the
// characteristic variant the fields are projected by L, reconstructed, and mapped back by R.
// T (optional, component-wise): transverse second differences [2][M] of the face's left and
// right cells, for the k = 2 shape parameter on the 5-cell cross (Sec. 6).  eta (optional):
// the M shape parameters of the face (characteristic: of the characteristic fields).
template <typename R, typename D, int KIND, int M, bool CHAR>
__device__ __forceinline__ bool face_all(const R* S, const MethodParams& mp, R* vm, R* vp, uint32_t* flags,
                                         const D* T = nullptr, R* eta = nullptr) {
    if (CHAR) {
        R Rm[3][3], Lm[3][3];
        if (!euler_eig<R>(S + 2 * M, S + 3 * M, mp_val<R>(mp.gamma, mp.gamma_f), Rm, Lm)) return false;
        R wm[3], wp[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R line[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                R s = R(0.0);
#pragma unroll
                for (int k = 0; k < 3; ++k) s += Lm[a][k] * S[j * M + k];
                line[j] = s;
            }
            flags[a] = face_field_any<R, D>(line, mp, &wm[a], &wp[a], D(0.0), D(0.0), eta ? eta + a : nullptr);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R sm = R(0.0), sp = R(0.0);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                sm += Rm[k][a] * wm[a];
                sp += Rm[k][a] * wp[a];
            }
            vm[k] = sm;
            vp[k] = sp;
        }
        return true;
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        R line[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) line[j] = S[j * M + k];
        flags[k] = T ? face_field_any<R, D>(line, mp, &vm[k], &vp[k], T[k], T[M + k], eta ? eta + k : nullptr)
                     : face_field_any<R, D>(line, mp, &vm[k], &vp[k], D(0.0), D(0.0), eta ? eta + k : nullptr);
    }
    return true;
}

}  // namespace npw
