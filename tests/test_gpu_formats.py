"""The integer float<->double format changes of the mixed-precision shape parameter
(fast::widen, widen_nz, narrow, seed_f in csrc/npw_fast.cuh) against the GPU's own
conversions and numpy's IEEE conversions, through npw_format_check.

They replace hardware conversions (which occupy the FP64 pipe on this GPU) in every shape
parameter evaluation of NPW_FP32_MIXED, so each documented property is checked here on every
float class: exact widening, round to nearest with ties away from zero, the flush below 2^-126,
the seed's truncation bound and range.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_00182_gb300 import build as b
    b.build()
    import paper_1602_00182_gb300.npweno as m
    m.load()
    return m


def _floats(rng, n):
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-126, 128, n).astype(np.float64)
    sign = rng.choice([-1.0, 1.0], n)
    x = (sign * mant * np.exp2(expo)).astype(np.float32)
    sub = (rng.integers(1, 1 << 23, 200) * np.float32(2.0 ** -149)).astype(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, np.finfo(np.float32).max, np.finfo(np.float32).tiny,
                        -np.finfo(np.float32).tiny, 2.0 ** -149, -(2.0 ** -149), 1.0, -1.0], dtype=np.float32)
    return np.concatenate([x, sub, -sub, special])


def _doubles(rng, n):
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-160, 140, n).astype(np.float64)
    sign = rng.choice([-1.0, 1.0], n)
    d = sign * mant * np.exp2(expo)
    special = np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** -99, 2.0 ** 99, 2.0 ** -100, np.nextafter(2.0 ** 99, 0.0),
                        float(np.finfo(np.float32).max), 3.5e38, -3.5e38, 2.0 ** -126, 1.0e-39])
    return np.concatenate([d, special])


def _run(npw, f, d):
    m = max(len(f), len(d))
    f = np.resize(f, m)
    d = np.resize(d, m)
    out = npw.npw_format_check(torch.tensor(f, device="cuda"), torch.tensor(d, device="cuda"))
    torch.cuda.synchronize()
    return f, d, {k: v.cpu().numpy() for k, v in out.items()}


def test_widen_is_exact_on_every_float_class(npw):
    f, _, o = _run(npw, _floats(np.random.default_rng(1), 200000), np.zeros(1))
    ref = f.astype(np.float64)
    fin = ~np.isnan(f)
    # bit for bit, signed zeros and infinities included; NaN stays NaN
    assert np.array_equal(o["widen"][fin].view(np.uint64), ref[fin].view(np.uint64))
    assert np.all(np.isnan(o["widen"][~fin]))
    assert np.array_equal(o["hw_widen"][fin].view(np.uint64), ref[fin].view(np.uint64))
    zn = (f == 0) | ((np.abs(f) >= np.finfo(np.float32).tiny) & np.isfinite(f))
    assert np.array_equal((o["flags"] & 1) == 1, zn)
    assert np.array_equal(o["widen_nz"][zn].view(np.uint64), ref[zn].view(np.uint64))


def test_narrow_rounds_to_nearest_with_the_documented_edges(npw):
    _, d, o = _run(npw, np.zeros(1, np.float32), _doubles(np.random.default_rng(2), 200000))
    hw = o["hw_narrow"]
    with np.errstate(over="ignore"):
        assert np.array_equal(hw.view(np.uint32), d.astype(np.float32).view(np.uint32))  # GPU = IEEE
    tiny = np.abs(hw) < np.finfo(np.float32).tiny  # the hardware result is subnormal or zero
    got = o["narrow"]
    assert np.array_equal(got[~tiny].view(np.uint32), hw[~tiny].view(np.uint32))
    assert np.all(got[tiny] == 0.0)
    assert np.array_equal(np.signbit(got[tiny]), np.signbit(d[tiny]))


def test_narrow_ties_go_away_from_zero(npw):
    f32 = np.array([1.0, 3.0, 1.5, 2.0 ** 100, 7.0], dtype=np.float32)
    half_ulp = np.spacing(f32).astype(np.float64) / 2.0
    d = np.concatenate([f32.astype(np.float64) + half_ulp, -(f32.astype(np.float64) + half_ulp)])
    _, _, o = _run(npw, np.zeros(1, np.float32), d)
    up = np.nextafter(f32, np.float32(np.inf))
    assert np.array_equal(o["narrow"], np.concatenate([up, -up]))


def test_seed_truncates_within_its_range(npw):
    _, d, o = _run(npw, np.zeros(1, np.float32), _doubles(np.random.default_rng(3), 200000))
    a = np.abs(d)
    in_range = (a >= 2.0 ** -99) & (a < 2.0 ** 99)
    assert np.array_equal((o["flags"] & 2) == 2, in_range)
    s = o["seed"][in_range].astype(np.float64)
    dd = d[in_range]
    assert np.all(np.abs(s) <= np.abs(dd))  # truncation toward zero
    assert np.all(np.abs(s - dd) <= np.abs(dd) * 2.0 ** -23)
    assert np.array_equal(np.signbit(s), np.signbit(dd))
