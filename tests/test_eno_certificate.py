"""The certificate behind the mixed path's ENO choice (Sec. 2), checked on the host.

Where the float test of the second ENO step is not certain, the kernels compare |p - 2q + r|
with |a - 2b + c| from the second differences written as error-free float sums (two-sum chains)
and return a decision only where it is both the exact one and the one the FP64 evaluation gives
(the oracle's arithmetic).  This test runs the same sequence of float operations in numpy
float32 (no contraction: the kernels are compiled with --fmad=false) on smooth fine-grid,
random, near-tie, plateau, multi-scale and zero-crossing stencils, and checks every decision it
returns against exact rational arithmetic and against the FP64 evaluation.  The GPU tests then
compare the kernels' ENO bits with the oracle's.
"""
from fractions import Fraction

import numpy as np

f32 = np.float32
U = f32(2.0 ** -24)


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def sdiff_exact(a, b, c):
    """a - 2b + c = h + l + eg exactly."""
    s, e = two_sum(a, c)
    t, f = two_sum(s, f32(f32(-2.0) * b))
    g, eg = two_sum(f, e)
    h, l = two_sum(t, g)
    return h, l, eg


def sdiff_sign(h, eg):
    if h != 0:
        return (f32(1.0) if h > 0 else f32(-1.0)) if f32(abs(h) * f32(1 - 2 * U)) > abs(eg) else f32(0.0)
    return f32(1.0) if eg >= 0 else f32(-1.0)


def sdiff_abs_less(a, b, c, p, q, r):
    """1 where |p - 2q + r| > |a - 2b + c|, 0 where not, -1 where not certain."""
    hx, lx, gx = sdiff_exact(a, b, c)
    hy, ly, gy = sdiff_exact(p, q, r)
    sx, sy = sdiff_sign(hx, gx), sdiff_sign(hy, gy)
    if sx == 0 or sy == 0:
        return -1
    zh, ze = two_sum(f32(sy * hy), f32(-sx * hx))
    m, em = two_sum(f32(sy * ly), f32(-sx * lx))
    zl, ez = two_sum(ze, m)
    w = f32(zh + zl)
    R = f32(f32(abs(em) + abs(ez)) + f32(abs(gx) + abs(gy)))
    S = f32(f32(f32(abs(a) + abs(c)) + f32(2 * abs(b))) + f32(f32(abs(p) + abs(r)) + f32(2 * abs(q))))
    fp64 = f32(S * f32(2.0 ** -50))
    if R == 0:
        if w != 0:
            return (1 if w > 0 else 0) if f32(abs(w) * f32(1 - U)) > fp64 else -1
        t = [abs(x) for x in (a, f32(2 * b), c, p, f32(2 * q), r) if x != 0]
        return 0 if (not t or max(t) <= min(t) * f32(2.0 ** 26)) else -1
    bound = f32(f32(f32(R * f32(1 + 8 * U)) + fp64) + f32(2.0 ** -140))
    return (1 if w > 0 else 0) if f32(abs(w) * f32(1 - U)) > bound else -1


def _stencils(rng, kind, count):
    for _ in range(count):
        if kind == "smooth":
            n = rng.choice([1024, 8192, 65536])
            x0, h = rng.uniform(0, 6.28), 6.28 / n
            yield [f32(1 + 0.5 * np.sin(x0 + k * h) + 0.3 * np.cos(3 * (x0 + k * h))) for k in range(5)]
        elif kind == "random":
            yield [f32(v) for v in rng.normal(size=5)]
        elif kind == "near_tie":
            base, d = rng.uniform(0.5, 2), rng.uniform(-1e-3, 1e-3)
            yield [f32(base + d * (k - 2) ** 2 + rng.normal() * 1e-9) for k in range(5)]
        elif kind == "plateau":
            yield [f32(rng.choice([0.0, 1.0, -1.0, 1e-20, 3.5, 1e30])) for _ in range(5)]
        elif kind == "multiscale":
            yield [f32(rng.normal() * 10.0 ** rng.integers(-30, 30)) for _ in range(5)]
        else:  # through a zero crossing
            n = rng.choice([256, 4096, 65536])
            x0, h = rng.uniform(0, 1), 1.0 / n
            yield [f32(0.3 * np.sin(20 * (x0 + k * h))) for k in range(5)]


def test_eno_second_step_certificate():
    rng = np.random.default_rng(1602)
    undecided = {}
    for kind in ("smooth", "random", "near_tie", "plateau", "multiscale", "zero_crossing"):
        n = und = 0
        for c in _stencils(rng, kind, 2500):
            for (a, b, cc, p, q, r) in ((c[0], c[1], c[2], c[1], c[2], c[3]), (c[1], c[2], c[3], c[2], c[3], c[4])):
                n += 1
                got = sdiff_abs_less(a, b, cc, p, q, r)
                if got < 0:
                    und += 1
                    continue
                X = Fraction(float(a)) - 2 * Fraction(float(b)) + Fraction(float(cc))
                Y = Fraction(float(p)) - 2 * Fraction(float(q)) + Fraction(float(r))
                exact = 1 if abs(Y) > abs(X) else 0
                x64 = abs(float(a) - 2.0 * float(b) + float(cc))
                y64 = abs(float(p) - 2.0 * float(q) + float(r))
                assert got == exact == (1 if x64 < y64 else 0), (kind, [float(v) for v in c])
        undecided[kind] = und / n
    # the certificate decides every smooth, random, near-tie and zero-crossing stencil here
    for kind in ("smooth", "random", "near_tie", "zero_crossing"):
        assert undecided[kind] < 0.01, undecided
