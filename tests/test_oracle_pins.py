"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets a part of the oracle so that a plausible mistake (a dropped term, a wrong
sign, a transposed row, a wrong weight) fails at least one of them:
  * P1  eta -> 0 limit: ENO/WENO-JS equal the exact-rational reconstruction built from the
        definition (polynomial interpolation of the primitive), Sec. 2 / Table k3 (left);
  * P2  exactness on cell averages of quadratics for every scheme (eta = 0 there, Table k3);
  * P3  Taylor order of every perturbed row with the table's eta: 4 (poly rows: 3);
  * P4  the perturbation rows are the flat limit of the MQ / Gaussian RBF interpolant;
  * P6  the monotone switch on hand cases of eq. root_value and against exact root location;
  * P11 whole-grid brute force (fractions) for every scheme, with and without the switch;
  * the WENO pieces (d_r, beta_r) against their definitions.
"""
import numpy as np
import pytest
from fractions import Fraction as F

import oracle as O
from paper_1602_00182_gb300 import inputs as I
from tests import bruteforce as B


def _smooth_avgs(edges):
    # averages of f(x) = sin(x + 0.3) + 2 (exact antiderivative)
    a, b = edges[:-1], edges[1:]
    return (-np.cos(b + 0.3) + np.cos(a + 0.3)) / (b - a) + 2.0


# --------------------------------------------------------------------------------------- P1
def test_linear_weights_match_definition():
    assert B.linear_weights(0) == [F(3, 10), F(3, 5), F(1, 10)]
    assert B.linear_weights(1) == [F(1, 10), F(3, 5), F(3, 10)]


@pytest.mark.parametrize("r", [-1, 0, 1, 2])
def test_poly_rows_are_primitive_interpolation(r):
    # Table k3 (left) with 11/6 in row r = -1: the eta = 0 coefficient of the oracle equals the
    # derivative of the interpolant of the primitive (right face of cell 0, stencil with r
    # cells to the left; row -1 = left face of the r = 0 stencil shifted by one cell).
    if r >= 0:
        exact = B.poly_row(r, 0)
    else:
        exact = B.poly_row(0, 1)
    for j in range(3):
        assert O.table_coef(O.MQ, r, j, 0.0) == pytest.approx(float(exact[j]), abs=1e-15)
        assert O.table_coef(O.GA, r, j, 0.0) == pytest.approx(float(exact[j]), abs=1e-15)


def test_beta_matches_integral_definition():
    g = np.random.default_rng(5)
    for _ in range(20):
        c = [F(int(x), 97) for x in g.integers(-300, 300, size=5)]
        v = {k - 2: c[k] for k in range(5)}
        got = O.beta_k3([float(x) for x in c])
        for r in range(3):
            assert got[r] == pytest.approx(float(B.beta(v, 0, r)), rel=1e-13, abs=1e-15)


def test_eno_choice_matches_divided_differences():
    g = np.random.default_rng(6)
    for _ in range(300):
        c = [F(int(x), 13) for x in g.integers(-40, 40, size=5)]
        v = {k - 2: c[k] for k in range(5)}
        r, _near = O.eno_choice([float(x) for x in c], tol=0.0)
        assert r == B.eno_r(v, 0)


# --------------------------------------------------------------------------------------- P2
@pytest.mark.parametrize("scheme", [O.ENO, O.WENO_JS, O.RBF_ENO, O.RBF_WENO])
@pytest.mark.parametrize("rbf", [O.MQ, O.GA])
@pytest.mark.parametrize("switch", [0, 1])
def test_quadratics_reconstructed_exactly(scheme, rbf, switch):
    g = np.random.default_rng(7)
    n = 24
    edges = np.linspace(0.0, 3.0, n + 1)
    for _ in range(4):
        c0, c1, c2 = g.normal(size=3)
        P = lambda x: c0 * x + c1 * x ** 2 / 2 + c2 * x ** 3 / 3  # antiderivative
        avg = (P(edges[1:]) - P(edges[:-1])) / np.diff(edges)
        vm, vp, fl, eta = O.reconstruct(avg, O.TRANSMISSIVE, O.Params(scheme=scheme, rbf=rbf, monotone_switch=switch))
        exact = c0 + c1 * edges + c2 * edges ** 2
        # faces whose stencil stays inside the domain (the transmissive ghosts are not quadratic)
        inner = slice(3, n - 2)
        np.testing.assert_allclose(vm[inner], exact[inner], rtol=0, atol=1e-12 * (1 + np.abs(exact).max()))
        np.testing.assert_allclose(vp[inner], exact[inner], rtol=0, atol=1e-12 * (1 + np.abs(exact).max()))
        assert np.all(np.abs(eta[inner]) < 1e-9)


# --------------------------------------------------------------------------------------- P3
@pytest.mark.parametrize("rbf", [O.MQ, O.GA])
@pytest.mark.parametrize("r", [0, 1, 2])
def test_perturbed_rows_are_fourth_order(rbf, r):
    """RBF-ENO with the stencil forced to r (replay flags): v^- and v^+ converge at order 4
    with the table's eta; ENO (eta = 0) at order 3.  A wrong coefficient, a wrong row for v^+
    or a wrong eta formula drops the order to 3."""
    def errs(scheme):
        out_m, out_p = [], []
        for n in (40, 80, 160):
            edges = np.linspace(0.0, 2.0, n + 1)
            avg = _smooth_avgs(edges)
            replay = np.full(n + 1, (r << 2) | (r << 4), dtype=np.uint8)
            vm, vp, _, _ = O.reconstruct(avg, O.TRANSMISSIVE, O.Params(scheme=scheme, rbf=rbf, monotone_switch=0),
                                         replay=replay)
            ex = np.sin(edges + 0.3) + 2.0
            inner = slice(4, n - 3)
            out_m.append(np.abs(vm[inner] - ex[inner]).max())
            out_p.append(np.abs(vp[inner] - ex[inner]).max())
        return np.array(out_m), np.array(out_p)

    em, ep = errs(O.RBF_ENO)
    for e in (em, ep):
        orders = np.log2(e[:-1] / e[1:])
        assert np.all(orders > 3.8), orders
    pm, pp = errs(O.ENO)
    for e in (pm, pp):
        orders = np.log2(e[:-1] / e[1:])
        assert np.all(np.abs(orders - 3.0) < 0.2), orders


# --------------------------------------------------------------------------------------- P4
@pytest.mark.parametrize("kind,rbf", [("mq", O.MQ), ("ga", O.GA)])
def test_perturbation_rows_are_rbf_flat_limit(kind, rbf):
    pytest.importorskip("mpmath")
    rows = B.rbf_rows(kind)
    for r in (-1, 0, 1, 2):
        for j in range(3):
            q = O.table_coef(rbf, r, j, 1.0) - O.table_coef(rbf, r, j, 0.0)
            assert q == pytest.approx(float(rows[r][j]), abs=1e-12), (kind, r, j)


# --------------------------------------------------------------------------------------- P6
def test_switch_k2_hand_cases():
    # eq. root_value on three cells (variant 1 tests both 3-cell halves of the 4-cell stencil)
    assert O.switch_k3([0, 1, 0, -1], variant=1)[0]  # (0,1,0): extremum inside
    assert not O.switch_k3([0, 1, 2, 3], variant=1)[0]  # linear: zero denominator, monotone
    assert O.switch_k3([0, 0, 1, 2], variant=1)[0]  # (0,0,1): ratio 1 -> non-monotone
    assert not O.switch_k3([1, 2, 4, 8], variant=1)[0]  # convex increasing: ratio outside (0,3)


def test_switch_cubic_against_exact_roots():
    g = np.random.default_rng(11)
    fired = 0
    for k in range(400):
        ints = g.integers(-30, 30, size=4)
        if k % 2:
            ints = np.sort(ints)  # increasing data: both outcomes common
        w = [F(int(x), 7) for x in ints]
        fires, near = O.switch_k3([float(x) for x in w], variant=0, tol=1e-9)
        if near:
            continue
        assert fires == B.switch_fires(w), w
        fired += fires
    assert 40 < fired < 340  # both outcomes exercised


def test_switch_monotone_smooth_data_does_not_fire():
    # cubic x^3 + x: p' > 0 everywhere
    edges = np.arange(-2.0, 3.0)
    P = lambda x: x ** 4 / 4 + x ** 2 / 2
    w = (P(edges[1:]) - P(edges[:-1]))
    assert not O.switch_k3(w)[0]


# --------------------------------------------------------------------------------------- P11
@pytest.mark.parametrize("scheme", ["eno", "weno_js", "rbf_eno", "rbf_weno"])
@pytest.mark.parametrize("rbf", ["mq", "ga"])
@pytest.mark.parametrize("switch", [False, True])
def test_bruteforce_tiny_grid(scheme, rbf, switch):
    pytest.importorskip("mpmath")
    g = np.random.default_rng([len(scheme), ord(scheme[0]), ord(rbf[0]), int(switch)])
    checked = 0
    for trial in range(6):
        n = 8
        vals = [F(int(x), 16) for x in g.integers(-32, 33, size=n)]
        vmx, vpx = B.reconstruct_periodic(vals, scheme, rbf=rbf, monotone_switch=switch)
        # random data can give |eta| > 1: compare the paper's formula without the eta bound
        p = O.Params(scheme=O.SCHEMES[scheme], rbf=O.MQ if rbf == "mq" else O.GA, monotone_switch=int(switch),
                     tie_tol=1e-9, eta_max=0.0)
        vm, vp, fl, eta = O.reconstruct(np.array([float(x) for x in vals]), O.PERIODIC, p)
        ties = (fl & (O.FLAG_SWITCH_TIE | O.FLAG_ENO_TIE_L | O.FLAG_ENO_TIE_R)) != 0
        for f in range(n + 1):
            if ties[f]:
                continue
            assert vm[f] == pytest.approx(float(vmx[f]), rel=1e-11, abs=1e-11), (trial, f)
            assert vp[f] == pytest.approx(float(vpx[f]), rel=1e-11, abs=1e-11), (trial, f)
            checked += 1
    assert checked > 20


def test_periodic_faces_coincide():
    g = np.random.default_rng(3)
    u = g.normal(size=37)
    vm, vp, fl, eta = O.reconstruct(u, O.PERIODIC, O.Params())
    assert vm[0] == vm[-1] and vp[0] == vp[-1] and eta[0] == eta[-1]


def test_eta_guard_on_unresolved_denominator():
    """Cell averages of x^3 around a face: the cubic is monotone with zero slope at the face, so
    the eta denominator is exactly 0 and eta = num / eps_M.  The optional guard (a reading for
    float states, off by default) sets eta = 0 there and leaves resolved faces alone."""
    edges = np.arange(-5.0, 6.0)
    P = lambda x: x ** 4 / 4
    avg = P(edges[1:]) - P(edges[:-1])  # exact averages of x^3 on unit cells
    face = 5  # face x = 0 between cell 4 and cell 5
    p0 = O.Params(scheme=O.RBF_WENO, monotone_switch=1, eta_max=0.0)
    _, _, _, eta0 = O.reconstruct(avg, O.TRANSMISSIVE, p0)
    assert abs(eta0[face]) > 1e10  # num / eps_M
    p1 = O.Params(scheme=O.RBF_WENO, monotone_switch=1, eta_guard=8 * 2.0 ** -24, eta_max=0.0)
    _, _, _, eta1 = O.reconstruct(avg, O.TRANSMISSIVE, p1)
    assert eta1[face] == 0.0
    other = [f for f in range(3, 9) if f != face]
    np.testing.assert_array_equal(eta1[other], eta0[other])


def test_eta_bound_on_monotone_zero_slope_stencil():
    """A monotone stencil with nearly zero slope at the face, (-1, -1/15 - 1e-3, 1/15 + 1e-3, 1):
    12 p'(s) = 9.56 s^2 + 0.03 > 0 (the switch does not fire) while the Table k3 denominator is
    only 0.03, so eta = -53 (at (-1, -1/15, 1/15, 1) it would be num / eps_M ~ 1e12).  The
    optional bound eta_max (a reading, off by default) returns the polynomial reconstruction
    there and marks the face; the smooth data of the paper's tests have |eta| < 0.05 and are
    untouched."""
    w = np.array([3.0, 3.0, -1.0, -1.0 / 15.0 - 1e-3, 1.0 / 15.0 + 1e-3, 1.0, 1.0, 1.0])
    fires, near = O.switch_k3(w[2:6], tol=1e-9)
    assert not fires and not near
    _, _, _, eta_off, z_off, c_off = O.reconstruct(w, O.TRANSMISSIVE, O.Params(), with_reason=True)
    _, _, _, eta_on, z_on, c_on = O.reconstruct(w, O.TRANSMISSIVE, O.Params(eta_max=1.0), with_reason=True)
    face = 4  # between cells 3 and 4: stencil cells 2..5
    assert eta_off[face] == pytest.approx(-1.594 / 0.03, rel=1e-6) and eta_on[face] == 0.0
    assert z_on[face] == O.ZERO_BOUND_L and c_on["bound"] == np.count_nonzero(z_on) >= 1
    assert not z_off.any() and c_off["bound"] == 0 and c_off["guard"] == 0
    u, dx = I.advection_sin(40)
    _, _, _, e1 = O.reconstruct(u, O.PERIODIC, O.Params(eta_max=1.0))
    _, _, _, e0 = O.reconstruct(u, O.PERIODIC, O.Params())
    np.testing.assert_array_equal(e1, e0)


def test_decision_counters_add_up():
    """The counters of a reconstruction: every face of an RBF scheme either has its eta zeroed by
    the switch or evaluated (k = 3: one per face; k = 2: one per face value); the guard and the
    bound count among the evaluated ones, and agree with the zero-reason bytes."""
    g = np.random.default_rng(7)
    u = np.concatenate([np.linspace(0.0, 1.0, 30) ** 3, np.full(10, 1.0), 1.0 + 0.1 * np.sin(np.arange(40)),
                        np.cumsum(g.uniform(0.0, 1.0, 40))])
    for k, per_face in ((3, 1), (2, 2)):
        p = O.Params(k=k, eta_guard=1e-3, eta_max=0.02)
        _, _, fl, _, z, c = O.reconstruct(u, O.TRANSMISSIVE, p, with_reason=True)
        assert c["switch"] + c["eval"] == per_face * u.size + per_face
        gl, bl = O.ZERO_GUARD_L, O.ZERO_BOUND_L
        assert c["guard"] == np.count_nonzero(z & gl) + np.count_nonzero(z & (gl << 2))
        assert c["bound"] == np.count_nonzero(z & bl) + np.count_nonzero(z & (bl << 2))
        assert c["guard"] > 0 and c["bound"] > 0
        sw = np.count_nonzero(fl & O.FLAG_SWITCH) + (np.count_nonzero(fl & O.FLAG_SWITCH_R_K2) if k == 2 else 0)
        assert c["switch"] == sw


# --------------------------------------------------------------------------------------- k = 2
# Table k2 and its shape parameter (Sec. 3.2-3.5), the k = 2 switch as printed (Sec. 4), ENO2
# and WENO3.  Same pins as for k = 3: rows from the definition, flat limit, eta from its
# derivation, Taylor order, exactness, and the whole-grid brute force.
@pytest.mark.parametrize("rbf", [O.MQ, O.GA])
def test_k2_poly_rows_are_primitive_interpolation(rbf):
    # row r (face i+1/2 from cells i-r, i-r+1): r = 0, 1 are cell i's right-face candidates,
    # r = -1 is cell i+1's left-face candidate with its own stencil r = 0
    expect = {0: B.poly_row_k2(0, 0), 1: B.poly_row_k2(1, 0), -1: B.poly_row_k2(0, 1)}
    for r, row in expect.items():
        for j in range(2):
            assert O.table_coef_k2(rbf, r, j, 0.0) == float(row[j]), (r, j)


def test_k2_linear_weights_are_the_three_cell_candidate():
    assert B.linear_weights_k2(0) == [F(2, 3), F(1, 3)]
    assert B.linear_weights_k2(1) == [F(1, 3), F(2, 3)]


@pytest.mark.parametrize("kind,rbf", [("mq", O.MQ), ("ga", O.GA)])
def test_k2_perturbation_rows_are_rbf_flat_limit(kind, rbf):
    """MQ: Table k2 (right) as printed; Gaussian: eq. i+1/2_approx1 for r = 0 and the flat
    limit for r = -1, 1."""
    pytest.importorskip("mpmath")
    rows = B.rbf_rows_k2(kind)
    for r in (-1, 0, 1):
        for j in range(2):
            q = O.table_coef_k2(rbf, r, j, 1.0) - O.table_coef_k2(rbf, r, j, 0.0)
            assert q == pytest.approx(float(rows[r][j]), abs=1e-12), (kind, r, j)


@pytest.mark.parametrize("rbf,kind", [(O.MQ, "mq"), (O.GA, "ga")])
def test_k2_eta_is_the_error_cancelling_shape_parameter(rbf, kind):
    """eta of eq. i+1/2_eps_approx / i+1/2_eps_approx1 equals -v''/(3v) (MQ) or -v''/(6v)
    (Gaussian) with v, v'' at the face from the cubic interpolant of the primitive (the paper's
    derivation, done here in exact rationals), for both faces of the cell."""
    g = np.random.default_rng(21)
    p = O.Params(k=2, rbf=rbf, eps_M=0.0, eta_max=0.0)
    checked = 0
    for _ in range(200):
        c3 = [F(int(x), 8) for x in g.integers(-40, 41, size=3)]
        for side in (0, 1):
            try:
                ex = B.eta_k2_from_derivation(c3, side, kind)
            except ZeroDivisionError:
                continue
            got = O.eta_k2([float(x) for x in c3], side, p)
            assert got == pytest.approx(float(ex), rel=1e-13, abs=1e-13), (c3, side)
            checked += 1
    assert checked > 300


def test_k2_switch_is_the_vertex_test():
    """eq. root_value / eq. adaptation: fires exactly when the vertex of p lies strictly inside
    the stencil (exact rational location), and never on linear data."""
    g = np.random.default_rng(22)
    checked = 0
    for _ in range(400):
        c3 = [F(int(x), 4) for x in g.integers(-20, 21, size=3)]
        fires, near = O.switch_k2([float(x) for x in c3], tol=1e-12)
        if near:
            continue
        assert fires == B.switch_fires_k2(c3), c3
        checked += 1
    assert checked > 300
    assert not O.switch_k2([1.0, 2.0, 3.0])[0]
    assert O.switch_k2([0.0, 1.0, 0.0])[0]


@pytest.mark.parametrize("rbf", [O.MQ, O.GA])
@pytest.mark.parametrize("r", [0, 1])
def test_k2_perturbed_rows_are_third_order(rbf, r):
    """RBF-ENO2 with the stencil forced to r: v^- and v^+ converge at order 3 with the table's
    eta (one above ENO2, Sec. 3.2); ENO2 at order 2."""
    def errs(scheme):
        out_m, out_p = [], []
        for n in (80, 160, 320):
            edges = np.linspace(0.0, 2.0, n + 1)
            avg = _smooth_avgs(edges)
            replay = np.full(n + 1, (r << 2) | (r << 4), dtype=np.uint8)
            vm, vp, _, _ = O.reconstruct(avg, O.TRANSMISSIVE,
                                         O.Params(k=2, scheme=scheme, rbf=rbf, monotone_switch=0), replay=replay)
            ex = np.sin(edges + 0.3) + 2.0
            inner = slice(4, n - 3)
            out_m.append(np.abs(vm[inner] - ex[inner]).max())
            out_p.append(np.abs(vp[inner] - ex[inner]).max())
        return np.array(out_m), np.array(out_p)

    for e in errs(O.RBF_ENO):
        orders = np.log2(e[:-1] / e[1:])
        assert np.all(orders > 2.8), orders
    for e in errs(O.ENO):
        orders = np.log2(e[:-1] / e[1:])
        assert np.all(np.abs(orders - 2.0) < 0.2), orders


@pytest.mark.parametrize("scheme", [O.ENO, O.WENO_JS, O.RBF_ENO, O.RBF_WENO])
@pytest.mark.parametrize("rbf", [O.MQ, O.GA])
def test_k2_linear_data_reconstructed_exactly(scheme, rbf):
    n = 24
    edges = np.linspace(-1.0, 2.0, n + 1)
    avg = 0.5 * (edges[:-1] + edges[1:]) * 3.0 - 1.0  # averages of 3x - 1
    vm, vp, fl, eta = O.reconstruct(avg, O.TRANSMISSIVE, O.Params(k=2, scheme=scheme, rbf=rbf))
    ex = 3.0 * edges - 1.0
    inner = slice(3, n - 2)
    np.testing.assert_allclose(vm[inner], ex[inner], atol=1e-12)
    np.testing.assert_allclose(vp[inner], ex[inner], atol=1e-12)


@pytest.mark.parametrize("scheme", ["eno", "weno_js", "rbf_eno", "rbf_weno"])
@pytest.mark.parametrize("rbf", ["mq", "ga"])
@pytest.mark.parametrize("switch", [False, True])
def test_k2_bruteforce_tiny_grid(scheme, rbf, switch):
    pytest.importorskip("mpmath")
    g = np.random.default_rng([2, len(scheme), ord(scheme[0]), ord(rbf[0]), int(switch)])
    checked = 0
    for trial in range(6):
        n = 8
        vals = [F(int(x), 16) for x in g.integers(-32, 33, size=n)]
        try:
            vmx, vpx = B.reconstruct_periodic_k2(vals, scheme, rbf=rbf, monotone_switch=switch)
        except ZeroDivisionError:
            continue
        p = O.Params(k=2, scheme=O.SCHEMES[scheme], rbf=O.MQ if rbf == "mq" else O.GA,
                     monotone_switch=int(switch), tie_tol=1e-9, eps_M=0.0, eta_max=0.0)
        vm, vp, fl, eta = O.reconstruct(np.array([float(x) for x in vals]), O.PERIODIC, p)
        ties = (fl & (O.FLAG_SWITCH_TIE | O.FLAG_ENO_TIE_L | O.FLAG_ENO_TIE_R)) != 0
        for f in range(n + 1):
            if ties[f]:
                continue
            assert vm[f] == pytest.approx(float(vmx[f]), rel=1e-11, abs=1e-11), (trial, f)
            assert vp[f] == pytest.approx(float(vpx[f]), rel=1e-11, abs=1e-11), (trial, f)
            checked += 1
    assert checked > 20


# --------------------------------------------------------------------------------------- 2D cross
def _avg_sin2d(n, shift=0.0):
    """Exact cell averages of sin(2 pi (x + y - shift)) on n x n cells of [0, 1]^2."""
    e = np.linspace(0.0, 1.0, n + 1)

    def F(x, y):  # d2F/dxdy = sin(2 pi (x + y - shift))
        return -np.sin(2 * np.pi * (x + y - shift)) / (4 * np.pi ** 2)
    X0, X1 = e[:-1][None, :], e[1:][None, :]
    Y0, Y1 = e[:-1][:, None], e[1:][:, None]
    return (F(X1, Y1) - F(X0, Y1) - F(X1, Y0) + F(X0, Y0)) * n * n, e


@pytest.mark.parametrize("scheme", [O.RBF_ENO, O.RBF_WENO])
@pytest.mark.parametrize("rbf", [O.MQ, O.GA])
def test_cross_2d_face_values_are_third_order(scheme, rbf):
    """Sec. 6: with the shape parameter on the 5-cell cross, the k = 2 face values at the x-face
    midpoints of sin(2 pi (x + y)) converge at order 3 (the paper's reconstruction test); the
    line form, whose eta ignores the transverse term v_yy dy^2 / 24 of the cell averages, stays
    at order 2, as does ENO2.  A wrong transverse coefficient or a wrong denominator drops the
    cross form to order 2."""
    def errs(cross, sch):
        out = []
        for n in (40, 80, 160, 320):
            U, e = _avg_sin2d(n)
            vmx, vpx, vmy, vpy = O.reconstruct_2d(U, O.PERIODIC,
                                                 O.Params(k=2, scheme=sch, rbf=rbf, monotone_switch=0, cross_2d=cross))
            c = (e[:-1] + e[1:]) / 2
            ex_x = np.sin(2 * np.pi * (e[None, :] + c[:, None]))
            ex_y = np.sin(2 * np.pi * (c[None, :] + e[:, None]))
            out.append(max(np.abs(vmx - ex_x).max(), np.abs(vpx - ex_x).max(),
                           np.abs(vmy - ex_y).max(), np.abs(vpy - ex_y).max()))
        return np.log2(np.array(out[:-1]) / np.array(out[1:]))
    assert np.all(errs(1, scheme) > 2.9)
    assert np.all(np.abs(errs(0, scheme) - 2.0) < 0.3)
    assert np.all(np.abs(errs(1, O.ENO) - 2.0) < 0.1)


def test_cross_2d_reduces_to_line_without_transverse_variation():
    """On data constant along y the transverse second differences of the x faces vanish, and the
    cross form of Sec. 6 gives exactly the line values of Table k2 there.  (Its y faces do
    change: a cell average differs from the value at a y-face midpoint by the x curvature.)"""
    g = np.random.default_rng(23)
    row = g.uniform(0.5, 1.5, size=37)
    U = np.tile(row, (12, 1))
    for sch in (O.RBF_ENO, O.RBF_WENO):
        a = O.reconstruct_2d(U, O.PERIODIC, O.Params(k=2, scheme=sch, cross_2d=1))
        b = O.reconstruct_2d(U, O.PERIODIC, O.Params(k=2, scheme=sch, cross_2d=0))
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert not np.array_equal(a[2], b[2])
        vm, vp, _, _ = O.reconstruct(row, O.PERIODIC, O.Params(k=2, scheme=sch))
        assert np.array_equal(a[0][5], vm) and np.array_equal(a[1][5], vp)
