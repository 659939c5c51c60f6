"""Parity of the k = 2 schemes (Table k2: ENO2, WENO3, RBF-ENO2, RBF-WENO3; one shape parameter
per face value and the per-cell switch of eq. root_value) on the GPU with the FP64 oracle.

Bars as for k = 3: NPW_FP64 relative L_inf <= 1e-12 with switch and ENO flags identical away
from near ties; NPW_FP32_MIXED decisions identical to the oracle's on the same float data and
values within float arithmetic (one stage 2e-6 relative, full runs L1 <= 1e-4 and
L_inf <= 2e-2).  Flag bits for k = 2: 0 / 3 switch of the left / right cell of the face,
2 / 4 their ENO stencil.
"""
import numpy as np
import pytest

import oracle as O
from paper_1602_00182_gb300 import inputs as I
from tests.parity_util import compare_faces

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_GUARD = 8.0 * 2.0 ** -24


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


def _gp(npw, o, precision=0):
    return npw.Params(k=2, scheme=o.scheme, rbf=o.rbf, monotone_switch=o.monotone_switch,
                      characteristic=o.characteristic, precision=precision, eps_M=o.eps_M, eps_weno=o.eps_weno,
                      gamma=o.gamma, adv_speed=o.adv_speed, inflow=o.inflow,
                      eta_guard=o.eta_guard if o.eta_guard > 0 else 0.0, eta_max=o.eta_max if o.eta_max > 0 else -1.0)


def _data(n, seed):
    g = np.random.default_rng(seed)
    x = np.linspace(0, 1, n, endpoint=False)
    u = 1.0 + 0.3 * np.sin(2 * np.pi * 3 * x + g.uniform(0, 6)) + 0.1 * np.cos(2 * np.pi * 7 * x)
    u[x > 0.6] += 0.5
    u[(x > 0.2) & (x < 0.3)] = 1.1
    u[(x > 0.75) & (x < 0.8)] = np.linspace(0, 1, ((x > 0.75) & (x < 0.8)).sum())
    return u


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("scheme", [O.ENO, O.WENO_JS, O.RBF_ENO, O.RBF_WENO])
@pytest.mark.parametrize("rbf", [O.MQ, O.GA])
@pytest.mark.parametrize("switch", [0, 1])
@pytest.mark.parametrize("bc", [O.PERIODIC, O.TRANSMISSIVE, O.INFLOW])
def test_k2_reconstruct_fp64(npw, scheme, rbf, switch, bc):
    op = O.Params(k=2, scheme=scheme, rbf=rbf, monotone_switch=switch, inflow=(0.7, 0, 0, 0))
    for n in (6, 37, 1025, 3001):
        u = _data(n, n)
        gvm, gvp, gfl, geta = npw.npweno_reconstruct(_dev(u), bc, _gp(npw, op), with_eta=True)
        # the linear ramp of _data (5% of the cells) makes the ratio test's denominator rounding
        # noise: those faces are switch near ties
        compare_faces(u, bc, op, gvm.cpu().numpy(), gvp.cpu().numpy(), gfl.cpu().numpy(), FP64_TOL,
                      1.0 if n < 64 else 0.06, geta=geta.cpu().numpy(), eta_exact=True, label=f"k2 n={n}")


def _guard_data():
    """Zero-mean data (the face values cross zero, where the k = 2 denominator, about 6 v, is
    small) with 8-cell blocks whose denominator -a + 5 b + 2 d of v^- cancels to ~1e-6 of its
    terms, so that both the guard and the bound have faces to act on."""
    g = np.random.default_rng(3)
    x = (np.arange(2000) + 0.5) / 2000
    u = 0.4 * np.sin(2 * np.pi * 3 * x + g.uniform(0, 6)) + 0.5 * (x > 1 / np.sqrt(3)) - 0.25
    for s in range(100, 1900, 150):
        for j in range(2, 8):
            u[s + j] = (u[s + j - 2] - 5.0 * u[s + j - 1]) / 2.0 + g.normal() * 1e-6
        u[s:s + 8] /= max(1.0, np.abs(u[s:s + 8]).max())
    return u


@pytest.mark.parametrize("eta_max,eta_guard", [(0.05, 0.0), (0.0, 1e-3)])
def test_k2_reconstruct_guard_and_bound(npw, eta_max, eta_guard):
    op = O.Params(k=2, eta_max=eta_max, eta_guard=eta_guard, monotone_switch=0)
    u = _guard_data()
    gvm, gvp, gfl, geta = npw.npweno_reconstruct(_dev(u), O.PERIODIC, _gp(npw, op), with_eta=True)
    gfl = gfl.cpu().numpy()
    assert ((gfl & 0xC0) != 0).any()
    compare_faces(u, O.PERIODIC, op, gvm.cpu().numpy(), gvp.cpu().numpy(), gfl, FP64_TOL, 0.005,
                  geta=geta.cpu().numpy(), eta_exact=True, label="k2 guard/bound")


@pytest.mark.parametrize("char", [0, 1])
def test_k2_reconstruct_euler_fp64(npw, char):
    for inst in I.euler_batch(count=4, nmin=64, nmax=2500):
        op = O.Params(k=2, characteristic=char)
        gvm, gvp, gfl, geta = npw.npweno_reconstruct(_dev(inst.u0), O.TRANSMISSIVE, _gp(npw, op), with_eta=True)
        compare_faces(inst.u0, O.TRANSMISSIVE, op, gvm.cpu().numpy(), gvp.cpu().numpy(), gfl.cpu().numpy(),
                      FP64_TOL, 0.02, geta=geta.cpu().numpy(), eta_exact=not char, label=f"k2 euler {inst.kind}")


@pytest.mark.parametrize("scheme", [O.ENO, O.WENO_JS, O.RBF_ENO, O.RBF_WENO])
def test_k2_rk3_step_fp64(npw, scheme):
    for n in (6, 1023, 1025, 2500):
        u = _data(n, 3 * n)
        op = O.Params(k=2, scheme=scheme)
        ref, a_ref = O.rk3_step(u, 1.0 / n, 0.3 / n, O.BURGERS, O.PERIODIC, op)
        gu = _dev(u)
        a = npw.npweno_rk3_step(gu, 1.0 / n, 0.3 / n, O.BURGERS, O.PERIODIC, _gp(npw, op), want_alpha=True)
        assert a == a_ref
        assert _rel(gu.cpu().numpy(), ref) <= FP64_TOL, n


@pytest.mark.parametrize("n", [25, 50, 100, 200, 400])
@pytest.mark.parametrize("scheme", [O.RBF_ENO, O.RBF_WENO])
def test_k2_advection_solve_fp64(npw, n, scheme):
    """sin(pi x) advected to T = 2 at CFL 0.5 with RBF-ENO2 / RBF-WENO3 (MQ), switch on."""
    u0, dx = I.advection_sin(n)
    op = O.Params(k=2, scheme=scheme)
    ref, rst = O.solve(u0, dx, 2.0, 0.5, O.ADVECTION, O.PERIODIC, op)
    gu = _dev(u0)
    st = npw.npweno_solve(gu, dx, 2.0, 0.5, O.ADVECTION, O.PERIODIC, _gp(npw, op))
    assert st["steps"] == rst["steps"] and st["t"] == 2.0 and st["status"] == 0
    assert _rel(gu.cpu().numpy(), ref) <= FP64_TOL


def test_k2_burgers_through_shock_fp64(npw):
    u0 = -np.sin(np.pi * np.linspace(-1, 1, 201)[:-1])
    op = O.Params(k=2, scheme=O.RBF_ENO, rbf=O.GA)
    ref, rst = O.solve(u0, 0.01, 0.6, 0.5, O.BURGERS, O.PERIODIC, op)
    gu = _dev(u0)
    st = npw.npweno_solve(gu, 0.01, 0.6, 0.5, O.BURGERS, O.PERIODIC, _gp(npw, op))
    assert st["steps"] == rst["steps"]
    assert _rel(gu.cpu().numpy(), ref) <= 1e-11


@pytest.mark.parametrize("scheme", [O.ENO, O.WENO_JS, O.RBF_ENO, O.RBF_WENO])
def test_k2_mixed_decisions_match_fp64(npw, scheme):
    """NPW_FP32_MIXED, k = 2: switch and ENO flags equal the oracle's double-precision
    decisions on the same float data; values within float arithmetic."""
    for n in (64, 1500, 4097):
        u = _data(n, n).astype(np.float32).astype(np.float64)
        u[n // 2: n // 2 + 40] = np.round(u[n // 2: n // 2 + 40] * 64) / 64  # plateaus and exact steps
        op = O.Params(k=2, scheme=scheme, eta_guard=MIXED_GUARD)
        gvm, gvp, gfl, geta = npw.npweno_reconstruct(_dev(u, torch.float32), O.PERIODIC, _gp(npw, op, precision=1),
                                                     with_eta=True)
        compare_faces(u, O.PERIODIC, op, gvm.cpu().numpy(), gvp.cpu().numpy(), gfl.cpu().numpy(), 2e-6,
                      1.0 if n < 100 else 0.06, geta=geta.cpu().numpy(), label=f"k2 mixed n={n}")


def test_k2_mixed_burgers_batch(npw):
    """Mixed-precision batch of periodic Burgers instances (ragged sizes) to T = 0.5 with
    RBF-WENO3 (Gaussian) against the oracle from the same float data."""
    inst = I.burgers_batch(count=12, nmin=64, nmax=1500, t_end=0.5, seed_index=31)
    ns = [it.n for it in inst]
    table, total = npw.make_instances(ns, [it.dx for it in inst], [0.5] * len(ns), [0.5] * len(ns), [0] * len(ns))
    host0 = np.concatenate([it.u0[0] for it in inst]).astype(np.float32)
    arena = _dev(host0, torch.float32)
    p = npw.Params(k=2, rbf=npw.NPW_RBF_GA, precision=npw.NPW_FP32_MIXED)
    st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, p)
    assert st == 0
    a = arena.cpu().numpy().astype(np.float64)
    off = 0
    op = O.Params(k=2, rbf=O.GA, eta_guard=MIXED_GUARD)
    for k, it in enumerate(inst):
        u0 = host0[off:off + it.n].astype(np.float64)
        ref, rst = O.solve(u0, it.dx, 0.5, 0.5, O.BURGERS, O.PERIODIC, op)
        assert stats[k]["status"] == 0 and stats[k]["t"] == 0.5
        e = np.abs(a[off:off + it.n] - ref)
        assert e.mean() <= 1e-4 and e.max() <= 2e-2, (k, it.n, e.mean(), e.max())
        off += it.n


@pytest.mark.parametrize("precision,switch", [(0, 1), (1, 0), (1, 1)])
def test_k2_2d_euler_step(npw, precision, switch):
    """One RK3 step of the isentropic vortex, 2D dimension by dimension, k = 2.  FP64: the
    oracle's bits (1e-12).  Mixed without the switch: float rounding (2e-6 relative).  Mixed
    with the switch: the decisions of stages 2 and 3 are taken on the float stage values, which
    differ from the oracle's double stage values by rounding, so a switch at a near tie may go
    the other way there (measured: the maximum error grows from 9e-7 to 3e-5 on this data while
    the mean stays at rounding level): mean error <= 1e-6 and max <= 3e-5 relative."""
    U, d = I.isentropic_vortex(64, 4.0, 5.0, 5.0, npts=2)
    if precision:
        U = U.astype(np.float32).astype(np.float64)
    op = O.Params(k=2, monotone_switch=switch, eta_guard=MIXED_GUARD if precision else 0.0)
    ref = O.rk3_step_2d(U, d, d, 0.2 * d, O.EULER2D, O.PERIODIC, op)
    gu = _dev(U, torch.float32 if precision else torch.float64)
    npw.npweno_rk3_step_2d(gu, d, d, 0.2 * d, O.EULER2D, O.PERIODIC, _gp(npw, op, precision=precision))
    got = gu.cpu().numpy().astype(np.float64)
    if not precision:
        assert _rel(got, ref) <= FP64_TOL
    elif not switch:
        assert _rel(got, ref) <= 2e-6
    else:
        scale = np.abs(ref).max()
        e = np.abs(got - ref)
        assert e.mean() <= 1e-6 * scale and e.max() <= 3e-5 * scale, (e.mean() / scale, e.max() / scale)


def test_k2_server_matches_batch_solve(npw):
    """The request server runs k = 2 requests (face-based float kernels, uncompensated); each
    result equals the batch solve of the same instance."""
    p = npw.Params(k=2, precision=1, batch_mode=1)
    srv = npw.Server(heap_cells=20000, max_slots=4, params=p)
    reqs = I.burgers_batch(count=3, nmin=300, nmax=900, seed_index=33)
    for j, it in enumerate(reqs):
        srv.submit(it.u0[0], npw.NPW_FLUX_BURGERS, 0, it.dx, 0.3, 0.5, tag=j)
    got = {}
    for _ in range(1000):
        act, q = srv.step(16)
        for r in srv.poll():
            got[r["tag"]] = r
        if act == 0 and q == 0:
            break
    srv.close()
    assert len(got) == 3
    for j, it in enumerate(reqs):
        table, _ = npw.make_instances([it.n], [it.dx], [0.3], [0.5], [0])
        arena = _dev(it.u0[0], torch.float32)
        st, stats = npw.npweno_batch_solve(arena, table, 1, npw.NPW_FLUX_BURGERS, p)
        assert st == 0 and got[j]["status"] == 0 and got[j]["steps"] == stats[0]["steps"]
        assert np.array_equal(got[j]["u"], arena.cpu().numpy())


def _cross_params(npw, op, precision):
    p = _gp(npw, op, precision=precision)
    p.cross_2d = 1
    return p


@pytest.mark.parametrize("shape", [(40, 24), (70, 45)])
@pytest.mark.parametrize("bc", [O.PERIODIC, O.TRANSMISSIVE, O.INFLOW])
@pytest.mark.parametrize("scheme", [O.RBF_ENO, O.RBF_WENO])
def test_k2_cross_2d_step_fp64(npw, shape, bc, scheme):
    """Sec. 6 shape parameter on the 5-cell cross (k = 2, 2D), FP64: one RK3 step of Burgers on
    a ragged grid equals the oracle to 1e-12, for every boundary condition."""
    nx, ny = shape
    g = np.random.default_rng(nx * ny + bc)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    U = 1.0 + 0.4 * np.sin(2 * np.pi * (x[None, :] + 0.7 * y[:, None])) + 0.1 * np.cos(6 * np.pi * y)[:, None]
    U[ny // 2:, nx // 3:] += 0.3 * g.uniform()
    d = 1.0 / nx
    op = O.Params(k=2, scheme=scheme, cross_2d=1, inflow=(1.2, 0, 0, 0))
    ref = O.rk3_step_2d(U, d, d, 0.2 * d, O.BURGERS, bc, op)
    gu = _dev(U)
    npw.npweno_rk3_step_2d(gu, d, d, 0.2 * d, O.BURGERS, bc, _cross_params(npw, op, 0))
    assert _rel(gu.cpu().numpy(), ref) <= FP64_TOL
    # the line form differs from the cross form on this data
    line = O.rk3_step_2d(U, d, d, 0.2 * d, O.BURGERS, bc, O.Params(k=2, scheme=scheme, inflow=(1.2, 0, 0, 0)))
    assert _rel(line, ref) > 1e-8


def test_k2_cross_2d_euler_fp64_and_mixed(npw):
    U, d = I.isentropic_vortex(48, 4.0, 5.0, 5.0, npts=2)
    op = O.Params(k=2, cross_2d=1)
    ref = O.rk3_step_2d(U, d, d, 0.2 * d, O.EULER2D, O.PERIODIC, op)
    gu = _dev(U)
    npw.npweno_rk3_step_2d(gu, d, d, 0.2 * d, O.EULER2D, O.PERIODIC, _cross_params(npw, op, 0))
    assert _rel(gu.cpu().numpy(), ref) <= FP64_TOL
    # mixed precision without the switch: float rounding of one step
    U32 = U.astype(np.float32).astype(np.float64)
    opm = O.Params(k=2, cross_2d=1, monotone_switch=0, eta_guard=MIXED_GUARD)
    refm = O.rk3_step_2d(U32, d, d, 0.2 * d, O.EULER2D, O.PERIODIC, opm)
    gm = _dev(U32, torch.float32)
    npw.npweno_rk3_step_2d(gm, d, d, 0.2 * d, O.EULER2D, O.PERIODIC, _cross_params(npw, opm, 1))
    assert _rel(gm.cpu().numpy().astype(np.float64), refm) <= 2e-6


def test_k2_cross_2d_solve_fp64(npw):
    """Advection of sin(2 pi (x + y)) for 40 steps with the cross form, FP64, against the oracle."""
    n = 32
    e = np.linspace(0.0, 1.0, n + 1)
    F = lambda x, y: -np.sin(2 * np.pi * (x + y)) / (4 * np.pi ** 2)  # noqa: E731
    U = (F(e[1:][None, :], e[1:][:, None]) - F(e[:-1][None, :], e[1:][:, None]) - F(e[1:][None, :], e[:-1][:, None]) +
         F(e[:-1][None, :], e[:-1][:, None])) * n * n
    d = 1.0 / n
    op = O.Params(k=2, scheme=O.RBF_ENO, monotone_switch=0, cross_2d=1)
    ref, rst = O.solve_2d(U, d, d, 40 * 0.1 * d, 0.2, O.ADVECTION, O.PERIODIC, op)
    gu = _dev(U)
    st = npw.npweno_solve_2d(gu, d, d, 40 * 0.1 * d, 0.2, O.ADVECTION, O.PERIODIC, _cross_params(npw, op, 0))
    assert st["status"] == 0 and st["steps"] == rst["steps"]
    assert _rel(gu.cpu().numpy(), ref) <= 1e-11
