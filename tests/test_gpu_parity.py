"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (each derived from the arithmetic it bounds):
  * NPW_FP64 vs oracle: relative L_inf <= 1e-12 on every face (both sides evaluate the same IEEE
    operations in the same order, without contraction); ENO stencil choices identical on
    every face, switch flags identical except at faces either side marks as switch near ties
    (closed form on the GPU, a 4x4 elimination in the oracle), whose share is bounded per data
    set; at those faces the oracle replays the GPU's decisions (tests/parity_util.py).
  * NPW_FP32_MIXED vs oracle: the per-config L1 / L_inf bounds stated in each test.
Sizes span several 1024-cell tiles and a ragged last tile; edge cases: the minimum n = 6,
tile boundaries, invalid arguments and non-finite states.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_00182_gb300 import inputs as I
from tests.parity_util import compare_faces

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_GUARD = 8.0 * 2.0 ** -24  # the mixed path's automatic eta guard, given to the oracle
SCHEMES = [(O.ENO, 0), (O.WENO_JS, 1), (O.RBF_ENO, 2), (O.RBF_WENO, 3)]


@pytest.fixture(scope="module")
def npw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_00182_gb300 import build as b
    b.build()
    import paper_1602_00182_gb300.npweno as m
    m.load()
    return m


def _dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _gparams(npw, o: "O.Params", precision=0):
    return npw.Params(k=o.k, cross_2d=o.cross_2d, scheme=o.scheme, rbf=o.rbf, monotone_switch=o.monotone_switch,
                      switch_variant=o.switch_variant,
                      characteristic=o.characteristic, precision=precision, eps_M=o.eps_M, eps_weno=o.eps_weno,
                      gamma=o.gamma, adv_speed=o.adv_speed, adv_speed_y=o.adv_speed_y, inflow=o.inflow,
                      eta_guard=o.eta_guard if o.eta_guard > 0 else 0.0, eta_max=o.eta_max if o.eta_max > 0 else -1.0)


def _mixed_data(n, seed):
    """Smooth waves, a jump, a flat stretch and a linear ramp (exercises every branch)."""
    g = np.random.default_rng(seed)
    x = np.linspace(0, 1, n, endpoint=False)
    u = 1.0 + 0.3 * np.sin(2 * np.pi * 3 * x + g.uniform(0, 6)) + 0.1 * np.cos(2 * np.pi * 7 * x)
    u[x > 0.6] += 0.5
    u[(x > 0.2) & (x < 0.3)] = 1.1
    u[(x > 0.75) & (x < 0.8)] = np.linspace(0, 1, ((x > 0.75) & (x < 0.8)).sum())
    return u


def _generic_data(n, seed):
    """Smooth waves and two jumps at irrational positions, no plateaus: decisions near their
    thresholds only by chance."""
    g = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    u = 1.0 + 0.4 * np.sin(2 * np.pi * 2 * x + g.uniform(0, 6)) + 0.15 * np.cos(2 * np.pi * 9 * x + g.uniform(0, 6))
    u += 0.6 * (x > 1 / np.sqrt(5)) - 0.3 * (x > 1 / np.sqrt(2))
    return u


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# shares of faces where a switch decision may be a near tie: the generic data have none by
# construction; _mixed_data has a linear ramp over 5% of its cells, where the ratio test of
# switch variant 1 divides rounding noise by rounding noise
TIE_FRAC_GENERIC = 0.005
TIE_FRAC_MIXED = 0.06
TIE_FRAC_NEAR = 0.05




# ------------------------------------------------------------------------------ reconstruct
@pytest.mark.parametrize("scheme", [s for s, _ in SCHEMES])
@pytest.mark.parametrize("rbf", [O.MQ, O.GA])
@pytest.mark.parametrize("switch,variant", [(0, 0), (1, 0), (1, 1)])
@pytest.mark.parametrize("bc", [O.PERIODIC, O.TRANSMISSIVE, O.INFLOW])
def test_reconstruct_fp64(npw, scheme, rbf, switch, variant, bc):
    op = O.Params(scheme=scheme, rbf=rbf, monotone_switch=switch, switch_variant=variant, inflow=(0.7, 0, 0, 0))
    for data, frac in ((_mixed_data, TIE_FRAC_MIXED), (_generic_data, TIE_FRAC_GENERIC)):
        for n in (6, 37, 1025, 3001):
            u = data(n, n)
            gvm, gvp, gfl, geta = npw.npweno_reconstruct(_dev(u), bc, _gparams(npw, op), with_eta=True)
            compare_faces(u, bc, op, gvm.cpu().numpy(), gvp.cpu().numpy(), gfl.cpu().numpy(), FP64_TOL,
                          1.0 if n < 64 else frac, geta=geta.cpu().numpy(), eta_exact=True,
                          label=f"{data.__name__} n={n}")


@pytest.mark.parametrize("eta_max,eta_guard", [(0.05, 0.0), (0.0, 1e-3), (0.02, 1e-3)])
def test_reconstruct_fp64_guard_and_bound(npw, eta_max, eta_guard):
    """The optional guard and bound (not in the paper) zero the same faces on both sides, and the
    GPU flags them (bits 6 / 7).  Switch off, so that the extrema of the data give large
    shape parameters and small denominators."""
    op = O.Params(eta_max=eta_max, eta_guard=eta_guard, monotone_switch=0)
    u = _generic_data(3001, 5)
    gvm, gvp, gfl, geta = npw.npweno_reconstruct(_dev(u), O.PERIODIC, _gparams(npw, op), with_eta=True)
    gfl = gfl.cpu().numpy()
    assert ((gfl & 0xC0) != 0).any()
    compare_faces(u, O.PERIODIC, op, gvm.cpu().numpy(), gvp.cpu().numpy(), gfl, FP64_TOL, TIE_FRAC_GENERIC,
                  geta=geta.cpu().numpy(), eta_exact=True, label="guard/bound")


@pytest.mark.parametrize("char", [0, 1])
def test_reconstruct_euler_fp64(npw, char):
    """Riemann and Shu-Osher-type Euler data, component- and characteristic-wise.  Piecewise
    constant states are decided exactly (a constant stencil is monotone), so near ties are rare
    even here."""
    for inst in I.euler_batch(count=4, nmin=64, nmax=2500):
        op = O.Params(characteristic=char)
        gvm, gvp, gfl, geta = npw.npweno_reconstruct(_dev(inst.u0), O.TRANSMISSIVE, _gparams(npw, op), with_eta=True)
        compare_faces(inst.u0, O.TRANSMISSIVE, op, gvm.cpu().numpy(), gvp.cpu().numpy(), gfl.cpu().numpy(),
                      FP64_TOL, 0.02, geta=geta.cpu().numpy(), eta_exact=not char, label=f"euler {inst.kind}")


def test_flux_fp64(npw):
    g = np.random.default_rng(1)
    for kind, m in ((O.ADVECTION, 1), (O.BURGERS, 1), (O.EULER1D, 3)):
        if m == 1:
            a, b = g.normal(size=(1, 777)), g.normal(size=(1, 777))
        else:
            a = I.prim_to_cons(g.uniform(0.2, 1, 777), g.uniform(-1, 1, 777), g.uniform(0.2, 1, 777))
            b = I.prim_to_cons(g.uniform(0.2, 1, 777), g.uniform(-1, 1, 777), g.uniform(0.2, 1, 777))
        h = O.flux(a, b, kind, 1.7, O.Params())
        gh = npw.npweno_flux(_dev(a), _dev(b), kind, 1.7, npw.Params()).cpu().numpy()
        assert np.array_equal(gh, h), kind


# ------------------------------------------------------------------------------ time stepping
@pytest.mark.parametrize("scheme", [s for s, _ in SCHEMES])
def test_rk3_step_fp64(npw, scheme):
    for n in (6, 1023, 1024, 1025, 2500):
        u = _mixed_data(n, 3 * n)
        op = O.Params(scheme=scheme)
        ref, a_ref = O.rk3_step(u, 1.0 / n, 0.3 / n, O.BURGERS, O.PERIODIC, op)
        gu = _dev(u)
        a = npw.npweno_rk3_step(gu, 1.0 / n, 0.3 / n, O.BURGERS, O.PERIODIC, _gparams(npw, op), want_alpha=True)
        assert a == a_ref
        assert _rel(gu.cpu().numpy(), ref) <= FP64_TOL, n


@pytest.mark.parametrize("n", [25, 50, 100, 200, 400])
@pytest.mark.parametrize("switch", [0, 1])
def test_advection_solve_fp64(npw, n, switch):
    """Linear advection of sin(pi x) on [-1, 1], periodic, RBF-WENO5 (MQ), LF, TVD-RK3 at
    CFL 0.5 to T = 2 (400 steps at N = 200)."""
    u0, dx = I.advection_sin(n)
    op = O.Params(monotone_switch=switch)
    ref, rst = O.solve(u0, dx, 2.0, 0.5, O.ADVECTION, O.PERIODIC, op)
    gu = _dev(u0)
    st = npw.npweno_solve(gu, dx, 2.0, 0.5, O.ADVECTION, O.PERIODIC, _gparams(npw, op))
    assert st["steps"] == rst["steps"] and st["t"] == 2.0 and st["status"] == 0
    assert _rel(gu.cpu().numpy(), ref) <= FP64_TOL


@pytest.mark.parametrize("scheme", [s for s, _ in SCHEMES])
def test_burgers_solve_fp64_through_shock(npw, scheme):
    inst = I.burgers_batch(count=1, nmin=1500, nmax=1600)[0]
    op = O.Params(scheme=scheme, rbf=O.GA)
    ref, rst = O.solve(inst.u0[0], inst.dx, 0.6, 0.5, O.BURGERS, O.PERIODIC, op)
    gu = _dev(inst.u0[0])
    st = npw.npweno_solve(gu, inst.dx, 0.6, 0.5, O.BURGERS, O.PERIODIC, _gparams(npw, op))
    assert st["steps"] == rst["steps"]
    assert _rel(gu.cpu().numpy(), ref) <= 1e-11


def test_batch_fp64_matches_oracle(npw):
    """Uneven batch: each instance keeps its own dt and stops at its own t_end."""
    inst = I.burgers_batch(count=12, nmin=64, nmax=2600)
    tends = [0.1 + 0.05 * i for i in range(len(inst))]
    table, total = npw.make_instances([it.n for it in inst], [it.dx for it in inst], tends, [0.5] * len(inst),
                                      [O.PERIODIC] * len(inst))
    arena = _dev(np.concatenate([it.u0[0] for it in inst]))
    op = O.Params(rbf=O.GA)
    status, stats = npw.npweno_batch_solve(arena, table, 1, O.BURGERS, _gparams(npw, op))
    assert status == 0
    a = arena.cpu().numpy()
    off = 0
    for it, te, s in zip(inst, tends, stats):
        ref, rst = O.solve(it.u0[0], it.dx, te, 0.5, O.BURGERS, O.PERIODIC, op)
        assert s["steps"] == rst["steps"] and s["t"] == te
        assert _rel(a[off:off + it.n], ref) <= 1e-11
        off += it.n


@pytest.mark.parametrize("char", [0, 1])
def test_euler_batch_fp64(npw, char):
    inst = I.euler_batch(count=4, nmin=300, nmax=1200)
    op = O.Params(characteristic=char)
    table, total = npw.make_instances([it.n for it in inst], [it.dx for it in inst], [min(it.t_end, 0.05) for it in inst],
                                      [0.5] * 4, [O.TRANSMISSIVE] * 4, m=3)
    arena = _dev(np.concatenate([it.u0.ravel() for it in inst]))
    status, stats = npw.npweno_batch_solve(arena, table, 3, O.EULER1D, _gparams(npw, op))
    assert status == 0
    a = arena.cpu().numpy()
    off = 0
    for it, s in zip(inst, stats):
        ref, rst = O.solve(it.u0, it.dx, min(it.t_end, 0.05), 0.5, O.EULER1D, O.TRANSMISSIVE, op)
        got = a[off:off + 3 * it.n].reshape(3, it.n)
        assert s["steps"] == rst["steps"]
        assert _rel(got, ref) <= 1e-11
        off += 3 * it.n


# ------------------------------------------------------------------------------ decision counts
@pytest.mark.parametrize("k", [3, 2])
@pytest.mark.parametrize("scheme", [O.RBF_ENO, O.RBF_WENO])
def test_solve_decision_counts_match_oracle_fp64(npw, k, scheme):
    """npw_solve_stats counts the shape-parameter decisions of every stage (switch fired, eta
    evaluated, zeroed by the guard, zeroed by the bound); in FP64 they equal the oracle's counts
    over the same run.  A bound and a guard are set so that both fire."""
    u0, dx = I.advection_sin(201)
    u0 = u0 + 0.3 * (np.arange(201) > 120)
    op = O.Params(k=k, scheme=scheme, eta_max=0.05, eta_guard=1e-3)
    ref, rst = O.solve(u0, dx, 0.3, 0.5, O.ADVECTION, O.PERIODIC, op)
    gu = _dev(u0)
    st = npw.npweno_solve(gu, dx, 0.3, 0.5, O.ADVECTION, O.PERIODIC, _gparams(npw, op))
    assert st["steps"] == rst["steps"]
    assert _rel(gu.cpu().numpy(), ref) <= FP64_TOL
    print(f"k={k}: oracle {rst['eta']}, GPU {st['eta']}")
    assert st["eta"] == rst["eta"]
    assert rst["eta"]["bound"] > 0 and rst["eta"]["guard"] > 0 and rst["eta"]["switch"] > 0
    per_step = (2 if k == 2 else 1) * 3 * 202  # faces (k = 2: face values) per step
    assert sum(st["eta"][x] for x in ("switch", "eval")) == per_step * st["steps"]


def test_batch_and_2d_decision_counts_match_oracle_fp64(npw):
    inst = I.burgers_batch(count=5, nmin=64, nmax=2600, seed_index=4)
    op = O.Params(rbf=O.GA, eta_max=0.2)
    table, total = npw.make_instances([it.n for it in inst], [it.dx for it in inst], [0.4] * 5, [0.5] * 5, [0] * 5)
    arena = _dev(np.concatenate([it.u0[0] for it in inst]))
    status, stats = npw.npweno_batch_solve(arena, table, 1, O.BURGERS, _gparams(npw, op))
    assert status == 0
    for it, s in zip(inst, stats):
        _, rst = O.solve(it.u0[0], it.dx, 0.4, 0.5, O.BURGERS, O.PERIODIC, op)
        assert s["eta"] == rst["eta"], (it.n, s["eta"], rst["eta"])
    U, d = I.four_quadrant(40, np.random.default_rng(4))
    U = np.ascontiguousarray(U[:, :, :37])
    op = O.Params(eta_max=0.3)
    _, rst = O.solve_2d(U, d, d, 0.02, 0.5, O.EULER2D, O.PERIODIC, op)
    st = npw.npweno_solve_2d(_dev(U), d, d, 0.02, 0.5, O.EULER2D, O.PERIODIC, _gparams(npw, op))
    assert st["steps"] == rst["steps"]
    assert st["eta"] == rst["eta"], (st["eta"], rst["eta"])


# ------------------------------------------------------------------------------ 2D
@pytest.mark.parametrize("shape", [(32, 32), (40, 24), (70, 9)])
def test_2d_euler_fp64(npw, shape):
    nx, ny = shape
    U, d = I.isentropic_vortex(max(nx, ny), 4.0, 5.0, 5.0)
    U = np.ascontiguousarray(U[:, :ny, :nx])
    op = O.Params()
    gu = _dev(U)
    ref1 = O.rk3_step_2d(U, d, d, 0.01, O.EULER2D, O.PERIODIC, op)
    npw.npweno_rk3_step_2d(gu, d, d, 0.01, O.EULER2D, O.PERIODIC, _gparams(npw, op))
    assert _rel(gu.cpu().numpy(), ref1) <= FP64_TOL


def test_2d_solve_fp64(npw):
    U, d = I.four_quadrant(48, np.random.default_rng(4))
    op = O.Params()
    ref, rst = O.solve_2d(U, d, d, 0.05, 0.5, O.EULER2D, O.PERIODIC, op)
    gu = _dev(U)
    st = npw.npweno_solve_2d(gu, d, d, 0.05, 0.5, O.EULER2D, O.PERIODIC, _gparams(npw, op))
    assert st["steps"] == rst["steps"]
    assert _rel(gu.cpu().numpy(), ref) <= 1e-11


# ------------------------------------------------------------------------------ mixed precision
def test_burgers_batch_mixed_precision_accuracy(npw):
    """Config family of the benchmark (periodic Burgers on [0, 2 pi], Gaussian perturbation,
    CFL 0.5) run past shock formation to T = 1.5 in NPW_FP32_MIXED, against the FP64 oracle
    started from the same float-rounded data.  Bound from the arithmetic: each of the
    3 S stage updates rounds the state to 2^-24 relative (|u| <= 2.5, S <= 1100 steps here),
    so smooth regions drift by at most ~3 S 2^-24 |u| ~ 5e-4 (L_inf) and far less on average;
    a shock displaced by a fraction of a cell adds jump x fraction to one cell.  Stated bars:
    L1 <= 5e-6, L_inf <= 2e-3 per instance (observed worst: 2.5e-7 and 4.6e-6; the L_inf bar
    leaves room for a shock cell)."""
    inst = I.burgers_batch(count=16, nmin=64, nmax=1024)
    table, total = npw.make_instances([it.n for it in inst], [it.dx for it in inst], [1.5] * 16, [0.5] * 16,
                                      [O.PERIODIC] * 16)
    arena = _dev(np.concatenate([it.u0[0] for it in inst]), torch.float32)
    op = O.Params(rbf=O.GA, eta_guard=MIXED_GUARD)
    status, stats = npw.npweno_batch_solve(arena, table, 1, O.BURGERS, _gparams(npw, op, precision=1))
    assert status == 0
    a = arena.cpu().numpy().astype(np.float64)
    off = 0
    worst_l1 = worst_linf = 0.0
    for it in inst:
        ref, _ = O.solve(it.u0[0].astype(np.float32).astype(np.float64), it.dx, 1.5, 0.5, O.BURGERS, O.PERIODIC, op)
        e = np.abs(a[off:off + it.n] - ref)
        worst_l1, worst_linf = max(worst_l1, e.mean()), max(worst_linf, e.max())
        off += it.n
    print(f"mixed precision Burgers T=1.5: worst L1 {worst_l1:.3e}, worst Linf {worst_linf:.3e}")
    assert worst_l1 <= 5e-6 and worst_linf <= 2e-3


def test_mixed_precision_single_stage(npw):
    """One RK3 step from float-representable data: FP32 arithmetic bound ~ 1e-6 relative."""
    u = _mixed_data(3000, 9).astype(np.float32).astype(np.float64)
    op = O.Params(eta_guard=MIXED_GUARD)
    ref, _ = O.rk3_step(u, 1.0 / 3000, 0.3 / 3000, O.BURGERS, O.PERIODIC, op)
    gu = _dev(u, torch.float32)
    npw.npweno_rk3_step(gu, 1.0 / 3000, 0.3 / 3000, O.BURGERS, O.PERIODIC, _gparams(npw, op, precision=1))
    assert _rel(gu.cpu().numpy().astype(np.float64), ref) <= 2e-6


# ------------------------------------------------------------------------------ properties / edges
def test_conservation_fp64_periodic(npw):
    inst = I.burgers_batch(count=1, nmin=3000, nmax=3100)[0]
    gu = _dev(inst.u0[0])
    s0 = gu.sum().item()
    npw.npweno_solve(gu, inst.dx, 1.0, 0.5, O.BURGERS, O.PERIODIC, npw.Params(rbf=npw.NPW_RBF_GA))
    assert abs(gu.sum().item() - s0) <= 1e-11 * abs(s0)


def test_invalid_arguments(npw):
    u = _dev(np.ones(5))
    with pytest.raises(npw.NpwError) as e:
        npw.npweno_reconstruct(u, 0, npw.Params())
    assert e.value.status == npw.NPW_EINVAL
    u = _dev(np.ones((2, 50)))
    with pytest.raises(npw.NpwError):
        npw.npweno_solve(u, 0.1, 1.0, 0.5, npw.NPW_FLUX_BURGERS, 0, npw.Params())
    with pytest.raises(npw.NpwError):
        npw.npweno_solve(_dev(np.ones(50)), -0.1, 1.0, 0.5, npw.NPW_FLUX_BURGERS, 0, npw.Params())
    with pytest.raises(ValueError):  # dtype must match the precision
        npw.npweno_solve(_dev(np.ones(50), torch.float32), 0.1, 1.0, 0.5, npw.NPW_FLUX_BURGERS, 0, npw.Params())


def test_nonfinite_state_is_reported(npw):
    u = np.ones(2000)
    u[1234] = np.nan
    with pytest.raises(npw.NpwError) as e:
        npw.npweno_solve(_dev(u), 0.01, 1.0, 0.5, npw.NPW_FLUX_BURGERS, 0, npw.Params())
    assert e.value.status == npw.NPW_ENONFINITE
    # in a batch only the broken instance fails; the others finish
    table, total = npw.make_instances([500, 700], [0.01, 0.01], [0.2, 0.2], [0.5, 0.5], [0, 0])
    a = np.ones(1200)
    a[100] = np.inf
    arena = _dev(a)
    st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, npw.Params())
    assert st == npw.NPW_ENONFINITE
    assert stats[0]["status"] == npw.NPW_ENONFINITE and stats[1]["status"] == 0 and stats[1]["t"] == 0.2


def test_zero_time_and_minimum_size(npw):
    u0, dx = I.advection_sin(6)
    gu = _dev(u0)
    st = npw.npweno_solve(gu, dx, 0.0, 0.5, npw.NPW_FLUX_ADVECTION, 0, npw.Params())
    assert st["steps"] == 0 and np.array_equal(gu.cpu().numpy(), u0)
    ref, rst = O.solve(u0, dx, 0.7, 0.5, O.ADVECTION, O.PERIODIC, O.Params())
    st = npw.npweno_solve(gu, dx, 0.7, 0.5, npw.NPW_FLUX_ADVECTION, 0, npw.Params())
    assert st["steps"] == rst["steps"] and _rel(gu.cpu().numpy(), ref) <= FP64_TOL


# ------------------------------------------------------------------------------ mixed-precision decisions
def _near_tie_data(n, seed):
    """Data that puts the switch and ENO decisions close to their thresholds: smooth waves
    with extrema on and near faces, constant and linear stretches, tiny oscillations."""
    g = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    u = 1.0 + 0.5 * np.sin(4 * np.pi * x)
    u[n // 5: n // 5 + 20] = 0.75
    u[n // 3: n // 3 + 30] = np.linspace(0.2, 0.4, 30)
    u[n // 2: n // 2 + 40] += 1e-6 * g.normal(size=40)
    u[2 * n // 3:] = np.round(u[2 * n // 3:] * 64) / 64  # plateaus with exact steps
    return u.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("scheme", [s for s, _ in SCHEMES])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("eta_eval", [0, 1])
def test_reconstruct_mixed_decisions_match_fp64(npw, scheme, variant, eta_eval):
    """NPW_FP32_MIXED: switch flags and ENO choices equal the double-precision decisions of the
    oracle on the same float data (except oracle-marked near ties); values within float
    arithmetic of the oracle."""
    for n in (64, 1500, 4097):
        u = _near_tie_data(n, n) if n != 64 else _mixed_data(n, 5).astype(np.float32).astype(np.float64)
        op = O.Params(scheme=scheme, switch_variant=variant, eta_guard=MIXED_GUARD)
        gp = _gparams(npw, op, precision=1)
        gp.eta_eval = eta_eval
        gvm, gvp, gfl, geta = npw.npweno_reconstruct(_dev(u, torch.float32), O.PERIODIC, gp, with_eta=True)
        compare_faces(u, O.PERIODIC, op, gvm.cpu().numpy(), gvp.cpu().numpy(), gfl.cpu().numpy(), 2e-6,
                      1.0 if n < 100 else TIE_FRAC_NEAR, geta=geta.cpu().numpy(), label=f"mixed n={n}")


def test_mixed_precision_full_burgers_instance_stays_finite(npw):
    """The instance of the 4096-instance batch (N = 5612) whose float-state plateau noise made
    the eta denominator exactly zero: with the round-off guard it finishes, and it stays within
    the mixed-precision bars of the FP64 oracle."""
    inst = I.burgers_batch(count=4096, seed_index=1)
    it = max((x for x in inst if x.n == 5612), key=lambda x: x.n)
    u = _dev(it.u0[0], torch.float32)
    st = npw.npweno_solve(u, it.dx, 1.5, 0.5, O.BURGERS, O.PERIODIC, npw.Params(rbf=npw.NPW_RBF_GA, precision=1))
    assert st["status"] == 0 and st["t"] == 1.5
    assert np.all(np.isfinite(u.cpu().numpy()))


# ------------------------------------------------------------------------------ resident whole-solve kernel
@pytest.mark.parametrize("family", ["burgers", "euler", "inflow"])
@pytest.mark.parametrize("k", [3, 2])
def test_resident_matches_per_stage_kernels(npw, family, k):
    """Instances that fit in shared memory are solved whole by one CTA (batch_mode 0); the
    per-stage kernels (batch_mode 1) run the same arithmetic, so both give identical bits
    (k = 3 and k = 2)."""
    if family == "burgers":
        inst = I.burgers_batch(count=24, nmin=64, nmax=9000)
        m, kind, bc = 1, O.BURGERS, O.PERIODIC
        tends = [0.4] * len(inst)
        u0s = [it.u0.ravel() for it in inst]
        ns, dxs = [it.n for it in inst], [it.dx for it in inst]
        inflow = (0.0, 0, 0, 0)
    elif family == "euler":
        inst = I.euler_batch(count=6, nmin=300, nmax=3300)
        m, kind, bc = 3, O.EULER1D, O.TRANSMISSIVE
        tends = [min(it.t_end, 0.05) for it in inst]
        u0s = [it.u0.ravel() for it in inst]
        ns, dxs = [it.n for it in inst], [it.dx for it in inst]
        inflow = (0.0, 0, 0, 0)
    else:
        ns = [200, 1500, 5000]
        dxs = [2.0 / n for n in ns]
        u0s = [np.where(np.linspace(-1, 1, n, endpoint=False) <= 0, 1.0, -1.0) for n in ns]
        m, kind, bc = 1, O.ADVECTION, O.INFLOW
        tends = [0.5] * 3
        inflow = (1.0, 0, 0, 0)
    table, total = npw.make_instances(ns, dxs, tends, [0.5] * len(ns), [bc] * len(ns), m=m)
    outs = []
    for mode in (0, 1):
        arena = _dev(np.concatenate(u0s), torch.float32)
        p = npw.Params(k=k, rbf=npw.NPW_RBF_GA, precision=1, batch_mode=mode, inflow=inflow)
        st, stats = npw.npweno_batch_solve(arena, table, m, kind, p)
        assert st == 0
        outs.append((arena.cpu().numpy(), stats))
    assert np.array_equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1], outs[1][1]):
        assert a["steps"] == b["steps"] and a["t"] == b["t"] and a["alpha_max"] == b["alpha_max"]
        assert a["eta"] == b["eta"]


def test_per_stage_mixed_burgers_accuracy(npw):
    """The per-stage mixed kernels (batch_mode 1) against the oracle on a multi-tile batch."""
    inst = I.burgers_batch(count=6, nmin=1000, nmax=5000)
    table, total = npw.make_instances([it.n for it in inst], [it.dx for it in inst], [0.5] * 6, [0.5] * 6,
                                      [O.PERIODIC] * 6)
    arena = _dev(np.concatenate([it.u0[0] for it in inst]), torch.float32)
    op = O.Params(rbf=O.GA, eta_guard=MIXED_GUARD)
    p = _gparams(npw, op, precision=1)
    p.batch_mode = 1
    status, stats = npw.npweno_batch_solve(arena, table, 1, O.BURGERS, p)
    assert status == 0
    a = arena.cpu().numpy().astype(np.float64)
    off = 0
    for it in inst:
        ref, _ = O.solve(it.u0[0].astype(np.float32).astype(np.float64), it.dx, 0.5, 0.5, O.BURGERS, O.PERIODIC, op)
        e = np.abs(a[off:off + it.n] - ref)
        print(f"per-stage mixed Burgers T=0.5, n={it.n}: L1 {e.mean():.3e}, Linf {e.max():.3e}")
        assert e.mean() <= 5e-6 and e.max() <= 2e-3  # observed worst: 5.6e-7, 2.3e-4 (a shock cell)
        off += it.n


@pytest.mark.parametrize("mode", [0, 1])
def test_mixed_precision_conserves_with_compensation(npw, mode):
    """Float state with the compensated (increment-form, Kahan-carried) RK3 update: the periodic
    sum drifts only by the float rounding of the final per-cell values, not by swallowed small
    increments (without compensation it drifted by ~1e-4 relative over 7000 steps)."""
    inst = I.burgers_batch(count=3, nmin=5000, nmax=8000, seed_index=21)
    table, total = npw.make_instances([it.n for it in inst], [it.dx for it in inst], [1.5] * 3, [0.5] * 3, [0] * 3)
    host0 = np.concatenate([it.u0[0] for it in inst]).astype(np.float32)
    arena = _dev(host0, torch.float32)
    p = npw.Params(rbf=npw.NPW_RBF_GA, precision=1, batch_mode=mode)
    st, stats = npw.npweno_batch_solve(arena, table, 1, O.BURGERS, p)
    assert st == 0
    a = arena.cpu().numpy().astype(np.float64)
    off = 0
    for it, s in zip(inst, stats):
        s0 = host0[off:off + it.n].astype(np.float64).sum()
        s1 = a[off:off + it.n].sum()
        assert abs(s1 - s0) <= 2e-7 * abs(s0) + 2.0 ** -24 * np.sqrt(it.n) * 4, (it.n, s["steps"], s1 - s0)
        off += it.n


@pytest.mark.parametrize("switch", [0, 1])
@pytest.mark.parametrize("kind", [O.ADVECTION, O.BURGERS, O.EULER2D])
def test_2d_mixed_step_matches_oracle(npw, switch, kind):
    """NPW_FP32_MIXED 2D (the phased tile kernel: eta per face, one reconstruction per cell and
    direction): one RK3 step against the oracle from the same float data on a ragged grid (tiles
    cut at both edges).  Without the switch the bar is float rounding (2e-6 relative); with it,
    decisions of stages 2 and 3 taken on float stage values may differ at near ties (mean 1e-6,
    max 3e-5 relative).  Both sides bound |eta| by 1: without the switch the printed eta is
    unbounded at the extrema of the data (num / eps_M where the denominator vanishes), and a
    float candidate with a coefficient of 1e6 is not within float rounding of the FP64 one."""
    nx, ny = 70, 45
    if kind == O.EULER2D:
        nx = ny = 70  # the whole periodic vortex (a cropped one would have a jump at the wrap)
        U, d = I.isentropic_vortex(nx, 4.0, 5.0, 5.0, npts=2)
    else:
        g = np.random.default_rng(kind)
        x = (np.arange(nx) + 0.5) / nx
        y = (np.arange(ny) + 0.5) / ny
        U = (1.0 + 0.5 * np.sin(2 * np.pi * x)[None, :] * np.cos(2 * np.pi * y)[:, None])[None]
        U[0, ny // 3:, nx // 2:] += 0.3 * g.uniform()
        d = 1.0 / nx
    U = U.astype(np.float32).astype(np.float64)
    op = O.Params(monotone_switch=switch, eta_guard=MIXED_GUARD, adv_speed=1.0, adv_speed_y=0.5, eta_max=1.0)
    dt = 0.2 * d
    ref = O.rk3_step_2d(U, d, d, dt, kind, O.PERIODIC, op)
    gu = _dev(U, torch.float32)
    npw.npweno_rk3_step_2d(gu, d, d, dt, kind, O.PERIODIC, _gparams(npw, op, precision=1))
    got = gu.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max()
    e = np.abs(got - ref)
    if not switch:
        assert e.max() <= 2e-6 * scale, e.max() / scale
    else:
        assert e.mean() <= 1e-6 * scale and e.max() <= 3e-5 * scale, (e.mean() / scale, e.max() / scale)
