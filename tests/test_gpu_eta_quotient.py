"""Direct pin of the mixed-precision shape parameter (NPW_FP32_MIXED) against the correctly
rounded quotient.

The mixed path does not divide in the obvious way.  With eta_eval 1 (and always for k = 2) it
widens the float cell averages, forms the Table k3 (k = 3) or Table k2 (k = 2) numerator and
denominator in FP64 by differences and single-rounding multiply-adds, and takes a Newton-Raphson
quotient seeded by a fast float reciprocal; with eta_eval 0 (the default, k = 3) it keeps
numerator and denominator as float pairs and takes a double-float quotient.  The claim: the result is the exact quotient rounded once to
float, up to the rounding an FP64 evaluation of the undivided differences carries -- u (|a| +
3|b|) / |num| + u (|a| + 15|b|) / |den| relative for k = 3 (u = 2^-53; a = w0 - w3,
b = w2 - w1), which is below one float ulp unless the differences cancel strongly -- plus
2^-41 for the quotient; the float pairs of eta_eval 0 carry ~2^-47 instead of u.  Results below the float
normal range are flushed to zero.  The reference is exact rational arithmetic (fractions) on
the same float data: no part of it comes from the library.

Cases: random stencils, cancelling denominators, denominators near zero relative to the data,
cell averages below 2^-100 (subnormal pair components), and denominators outside the reciprocal
seed's range [2^-99, 2^99) (the double-division path).  Which faces the guard and the bound
set to zero must agree exactly with the FP64 oracle on the same data.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from tests.parity_util import GPU_ZERO_BOUND, GPU_ZERO_GUARD

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS_M = 1e-12
MIXED_GUARD = 8.0 * 2.0 ** -24
F32_MIN_NORMAL = 2.0 ** -126


@pytest.fixture(scope="module")
def npw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_00182_gb300 import build as b
    b.build()
    import paper_1602_00182_gb300.npweno as m
    m.load()
    return m


def _blocks(seed):
    """A periodic line of float32 cell averages made of 8-cell blocks, one case each."""
    g = np.random.default_rng(seed)
    out = []
    for _ in range(60):
        out.append(g.normal(size=8))                                  # random
    for _ in range(60):                                               # cancelling denominator
        w = g.normal(size=8)
        for j in range(3, 8):
            w[j] = w[j - 3] - 15.0 * w[j - 2] + 15.0 * w[j - 1] + g.normal() * 1e-5
        out.append(w / max(np.abs(w).max(), 1.0))
    for _ in range(40):                                               # den tiny vs the data
        w = 1.0 + g.normal(size=8) * 1e-3
        for j in range(3, 8):
            w[j] = w[j - 3] - 15.0 * w[j - 2] + 15.0 * w[j - 1] + g.normal() * 1e-7
        out.append(w)
    for _ in range(40):                                               # k = 2: -a + 5 b + 2 d ~ 0
        w = 1.0 + g.normal(size=8) * 0.1
        for j in range(2, 8):
            w[j] = (w[j - 2] - 5.0 * w[j - 1]) / 2.0 + g.normal() * 1e-7
        out.append(w / np.abs(w).max())
    for s in (1e-33, 1e-36, 3e-38):                                   # pair components below 2^-100
        for _ in range(20):
            out.append(g.normal(size=8) * s)
    for s in (1e-31, 2e-32, 1e31, 1e33):                              # den outside the seed range
        for _ in range(20):
            out.append(g.normal(size=8) * s)
    u = np.concatenate(out).astype(np.float32)
    return u


def _exact_eta(u32, k, rbf):
    """Exact-rational quotient of each face (face f between cells f-1 and f, periodic), rounded
    once to double, and the conditioning kappa = S_num / |num| + S_den / |den| of an FP64
    evaluation.  k = 3: (w0 - 3 w1 + 3 w2 - w3) / (w0 - 15 w1 + 15 w2 - w3 + eps_M) on cells
    f-2..f+1, S_num = |a| + 3|b|, S_den = |a| + 15|b| + eps_M (a = w0 - w3, b = w2 - w1);
    k = 2 (v^- of cell f-1, cells f-2, f-1, f = a, b, d): F (-a + 2 b - d) / (-a + 5 b + 2 d +
    eps_M), F = 2 (MQ) or 1 (Gaussian), S_num = |a| + 2|b| + |d|, S_den = |a| + 5|b| + 2|d| + eps_M."""
    n = u32.size
    fr = [Fraction(float(x)) for x in u32]
    em = Fraction(EPS_M)
    out = np.zeros(n + 1)
    kap = np.zeros(n + 1)
    for f in range(n + 1):
        c = lambda j: fr[(f + j) % n]
        if k == 3:
            a, b = c(-2) - c(1), c(0) - c(-1)
            num, den = a + 3 * b, a + 15 * b + em
            sn, sd = abs(a) + 3 * abs(b), abs(a) + 15 * abs(b) + em
            fac = 1
        else:
            a, b, d = c(-2), c(-1), c(0)
            num, den = -a + 2 * b - d, -a + 5 * b + 2 * d + em
            sn, sd = abs(a) + 2 * abs(b) + abs(d), abs(a) + 5 * abs(b) + 2 * abs(d) + em
            fac = 2 if rbf == O.MQ else 1
        if den == 0:
            out[f], kap[f] = np.nan, np.inf
            continue
        out[f] = float(fac * num / den)
        kap[f] = float(sn / abs(num)) + float(sd / abs(den)) if num != 0 else np.inf
    return out, kap


def _ulp32(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


@pytest.mark.parametrize("k", [3, 2])
@pytest.mark.parametrize("eta_eval", [0, 1])
@pytest.mark.parametrize("rbf", [O.MQ, O.GA])
def test_mixed_eta_is_the_rounded_exact_quotient(npw, k, eta_eval, rbf):
    u = _blocks(10 * k + eta_eval)
    p = npw.Params(k=k, rbf=rbf, monotone_switch=0, precision=npw.NPW_FP32_MIXED, eta_eval=eta_eval,
                   eps_M=EPS_M, eta_guard=-1.0, eta_max=-1.0)
    _, _, gfl, geta = npw.npweno_reconstruct(torch.tensor(u, device="cuda"), O.PERIODIC, p, with_eta=True)
    geta = geta.cpu().numpy().astype(np.float64)
    assert not (gfl.cpu().numpy() & (GPU_ZERO_GUARD | GPU_ZERO_BOUND)).any()
    q, kap = _exact_eta(u, k, rbf)
    fin = np.isfinite(q) & np.isfinite(kap)
    normal = fin & (np.abs(q) >= F32_MIN_NORMAL) & (np.abs(q) < 3e38)
    err = np.abs(geta[normal] - q[normal])
    ulp = _ulp32(q[normal])
    # the FP64 evaluation (eta_eval 1; k = 2 always), rounded once: 0.5 ulp; float pairs and a
    # double-float quotient (eta_eval 0, k = 3): within one ulp (not correctly rounded)
    fp64_form = eta_eval == 1 or k == 2
    unit, last = (2.0 ** -52, 0.5) if fp64_form else (2.0 ** -44, 1.0)
    bound = last * ulp + np.abs(q[normal]) * (unit * (kap[normal] + 5.0) + 2.0 ** -40)
    worst = float((err / bound).max())
    well = kap[normal] < 2.0 ** 20  # no strong cancellation: the bound is below one ulp
    exact = float(np.mean(err[well] <= 0.5 * ulp[well] * (1 + 2.0 ** -20)))
    print(f"k={k} eta_eval={eta_eval} rbf={rbf}: {normal.sum()} faces ({well.sum()} well conditioned, "
          f"{exact:.4f} of them rounded to nearest), worst err / bound {worst:.3f}")
    assert np.all(err <= bound), worst
    assert np.all(err[well] <= ulp[well])
    # below the float normal range: flushed to a (signed) zero or within the smallest normal
    tiny = fin & (np.abs(q) < F32_MIN_NORMAL)
    assert np.all(np.abs(geta[tiny]) <= F32_MIN_NORMAL)
    assert normal.sum() > 0.9 * fin.sum() and well.sum() > 0.5 * normal.sum()


@pytest.mark.parametrize("k", [3, 2])
@pytest.mark.parametrize("eta_eval", [0, 1])
def test_mixed_guard_and_bound_zero_the_oracles_faces(npw, k, eta_eval):
    """The automatic round-off guard of the float state and a bound zero exactly the faces the
    FP64 oracle zeroes on the same float data (the guard is decided in float only where its
    rounding cannot change the outcome, else in double)."""
    u = _blocks(3 + k)
    for eta_max in (0.0, 0.5):
        p = npw.Params(k=k, monotone_switch=0, precision=npw.NPW_FP32_MIXED, eta_eval=eta_eval, eps_M=EPS_M,
                       eta_guard=0.0, eta_max=eta_max if eta_max > 0 else -1.0)
        _, _, gfl, _ = npw.npweno_reconstruct(torch.tensor(u, device="cuda"), O.PERIODIC, p, with_eta=True)
        gfl = gfl.cpu().numpy()
        op = O.Params(k=k, monotone_switch=0, eps_M=EPS_M, eta_guard=MIXED_GUARD, eta_max=eta_max)
        _, _, _, _, zr, cnt = O.reconstruct(u.astype(np.float64), O.PERIODIC, op, with_reason=True)
        o_guard = (zr & (O.ZERO_GUARD_L | O.ZERO_GUARD_R)) != 0
        o_bound = (zr & (O.ZERO_BOUND_L | O.ZERO_BOUND_R)) != 0
        assert o_guard.any()
        assert np.array_equal((gfl & GPU_ZERO_GUARD) != 0, o_guard)
        assert np.array_equal((gfl & GPU_ZERO_BOUND) != 0, o_bound)
        if eta_max > 0:
            assert o_bound.any()
