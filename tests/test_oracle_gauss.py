"""Pins of the oracle's reconstruction at a point of a face (Sec. 6, k = 2 on the 5-cell cross)
and of the two-point Gauss rule for eq. 2DIntegral (Sec. 7).

Sec. 7 states that the third-order reconstruction needs two quadrature points per face for a
third-order scheme, and uses one (the midpoint) in its experiments.  The oracle evaluates the
3-cell stencil of eq. poly_recon2d, perturbed as in eq. rbf_recon_2d, at the point sigma cell
widths from the midpoint along the face and cancels the Taylor error at that point.  The pins:

* linear fields are reproduced exactly at every point (every scheme);
* the unperturbed stencil (ENO) on quadratic fields misses the exact value by the closed-form
  Taylor error e v_xx dx^2 + (1/24 + s sigma/2 - sigma^2/2) v_yy dy^2 -+ (sigma/2) v_xy dx dy,
  with e and s the stencil choices (a dropped transverse term or a wrong sign fails it);
* RBF-ENO point values converge at third order at the Gauss points and elsewhere on a field with
  v_xx != v_yy and v_xy != 0 (ENO: second order);
* the finite-volume solve of Sec. 7 Example 1 with the Gauss rule converges at third order,
  the midpoint rule at second (the paper's table0_2d).
"""
import numpy as np
import pytest

import oracle as O

G = O.GAUSS2


def test_gauss_abscissa():
    # the two-point Gauss-Legendre rule on [-1/2, 1/2] integrates cubics exactly
    for p in range(4):
        exact = (0.5 ** (p + 1) - (-0.5) ** (p + 1)) / (p + 1)
        assert abs(0.5 * (G ** p + (-G) ** p) - exact) < 1e-16


def _avg_poly(nx, ny, c):
    """Exact cell averages of v = c0 + c1 x + c2 y + c3 x^2 + c4 y^2 + c5 x y on [0,1]^2."""
    hx, hy = 1.0 / nx, 1.0 / ny
    x0 = np.arange(nx) * hx
    y0 = np.arange(ny) * hy
    xc, yc = x0 + hx / 2, y0 + hy / 2
    x2 = ((x0 + hx) ** 3 - x0 ** 3) / (3 * hx)
    y2 = ((y0 + hy) ** 3 - y0 ** 3) / (3 * hy)
    X, Y = xc[None, :], yc[:, None]
    return (c[0] + c[1] * X + c[2] * Y + c[3] * x2[None, :] + c[4] * y2[:, None] + c[5] * X * Y)


def _poly(c, x, y):
    return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * y * y + c[5] * x * y


SCHEMES_K2 = [("eno", dict(scheme=O.ENO)), ("weno3", dict(scheme=O.WENO_JS)),
              ("rbf_eno_mq", dict(scheme=O.RBF_ENO, cross_2d=1)), ("rbf_eno_ga", dict(scheme=O.RBF_ENO, cross_2d=1, rbf=O.GA)),
              ("rbf_weno_mq", dict(scheme=O.RBF_WENO, cross_2d=1))]


@pytest.mark.parametrize("name,kw", SCHEMES_K2)
@pytest.mark.parametrize("sigma", [-0.5, -G, 0.0, G, 0.37])
def test_linear_fields_are_exact_at_every_point(name, kw, sigma):
    nx, ny = 23, 17
    c = (0.3, 1.7, -2.2, 0.0, 0.0, 0.0)
    u = _avg_poly(nx, ny, c)
    p = O.Params(k=2, **kw)
    vmx, vpx, vmy, vpy = O.reconstruct_2d(u, O.TRANSMISSIVE, p, sigma=sigma)
    hx, hy = 1.0 / nx, 1.0 / ny
    xf, yc = np.arange(nx + 1) * hx, (np.arange(ny) + 0.5) * hy
    ex = _poly(c, xf[None, :], yc[:, None] + sigma * hy)
    xc, yf = (np.arange(nx) + 0.5) * hx, np.arange(ny + 1) * hy
    ey = _poly(c, xc[None, :] + sigma * hx, yf[:, None])
    # interior faces: the stencil (2 cells along the normal, 1 across, the diagonal) stays inside
    sx = (slice(2, ny - 2), slice(3, nx - 2))
    sy = (slice(3, ny - 2), slice(2, nx - 2))
    for got, ref, s in ((vmx, ex, sx), (vpx, ex, sx), (vmy, ey, sy), (vpy, ey, sy)):
        assert np.abs(got[s] - ref[s]).max() < 1e-13


def _eno_side(dn, up):
    """ENO pick of the transverse neighbour (Sec. 6 with Newton's divided differences as in 1D):
    the lower one (-1) only where its difference is strictly smaller in magnitude."""
    return np.where(np.abs(dn) < np.abs(up), -1.0, 1.0)


@pytest.mark.parametrize("sigma", [-G, G, 0.41, -0.23])
@pytest.mark.parametrize("c", [(0.0, 0.4, -0.3, 1.3, -0.7, 2.1), (1.0, -1.0, 0.5, -2.0, 3.0, -1.5)])
def test_eno_point_error_on_quadratics_is_the_taylor_closed_form(sigma, c):
    """Unperturbed 3-cell stencil at a point of an x face, v^- from cell i (half a cell behind
    the face): error e v_xx dx^2 + (1/24 + s sigma/2 - sigma^2/2) v_yy dy^2 - (sigma/2) v_xy dx dy
    (v^+: + (sigma/2) v_xy dx dy), e = 1/6 for the two cells at the face and -1/3 for the
    extrapolating pair, s = the ENO side of the transverse neighbour; y faces with x and y
    exchanged.  Exact for quadratics (the Taylor series ends)."""
    nx, ny = 19, 26
    hx, hy = 1.0 / nx, 1.0 / ny
    u = _avg_poly(nx, ny, c)
    vxx, vyy, vxy = 2 * c[3], 2 * c[4], c[5]
    vmx, vpx, vmy, vpy = O.reconstruct_2d(u, O.TRANSMISSIVE, O.Params(k=2, scheme=O.ENO), sigma=sigma)
    # x faces f = 3..nx-3 of rows 2..ny-3
    for j in range(2, ny - 2):
        for f in range(3, nx - 2):
            yq = (j + 0.5) * hy + sigma * hy
            exact = _poly(c, f * hx, yq)
            for side, cell, nb in ((0, f - 1, f), (1, f, f - 1)):
                # ENO pair along x: the extrapolating pair where the far difference is smaller
                far = cell - 1 if side == 0 else cell + 1
                ext = abs(u[j, cell] - u[j, far]) < abs(u[j, nb] - u[j, cell])
                e = -1.0 / 3.0 if ext else 1.0 / 6.0
                s = _eno_side(u[j, cell] - u[j - 1, cell], u[j + 1, cell] - u[j, cell])
                sgn = -1.0 if side == 0 else 1.0
                err = e * vxx * hx ** 2 + (1 / 24 + s * sigma / 2 - sigma ** 2 / 2) * vyy * hy ** 2 \
                    + sgn * (sigma / 2) * vxy * hx * hy
                got = vmx[j, f] if side == 0 else vpx[j, f]
                assert abs(got - (exact + err)) < 1e-12, (j, f, side)
    # y faces f = 3..ny-3 of columns 2..nx-3
    for i in range(2, nx - 2):
        for f in range(3, ny - 2):
            xq = (i + 0.5) * hx + sigma * hx
            exact = _poly(c, xq, f * hy)
            for side, cell, nb in ((0, f - 1, f), (1, f, f - 1)):
                far = cell - 1 if side == 0 else cell + 1
                ext = abs(u[cell, i] - u[far, i]) < abs(u[nb, i] - u[cell, i])
                e = -1.0 / 3.0 if ext else 1.0 / 6.0
                s = _eno_side(u[cell, i] - u[cell, i - 1], u[cell, i + 1] - u[cell, i])
                sgn = -1.0 if side == 0 else 1.0
                err = e * vyy * hy ** 2 + (1 / 24 + s * sigma / 2 - sigma ** 2 / 2) * vxx * hx ** 2 \
                    + sgn * (sigma / 2) * vxy * hx * hy
                got = vmy[f, i] if side == 0 else vpy[f, i]
                assert abs(got - (exact + err)) < 1e-12, (i, f, side)


def _avg_sin(n, kx, ky):
    """Exact cell averages of sin(2 pi (kx x + ky y)) on the periodic unit square."""
    h = 1.0 / n
    x0 = np.arange(n) * h
    a, b = 2 * np.pi * kx, 2 * np.pi * ky
    fx = (np.exp(1j * a * (x0 + h)) - np.exp(1j * a * x0)) / (1j * a * h)
    fy = (np.exp(1j * b * (x0 + h)) - np.exp(1j * b * x0)) / (1j * b * h)
    return np.imag(fy[:, None] * fx[None, :])


def _point_errors(n, sigma, p, kx=1, ky=2):
    u = _avg_sin(n, kx, ky)
    vmx, vpx, vmy, vpy = O.reconstruct_2d(u, O.PERIODIC, p, sigma=sigma)
    h = 1.0 / n
    f = lambda x, y: np.sin(2 * np.pi * (kx * x + ky * y))
    ex = f(np.arange(n + 1)[None, :] * h, ((np.arange(n) + 0.5)[:, None] + sigma) * h)
    ey = f(((np.arange(n) + 0.5)[None, :] + sigma) * h, np.arange(n + 1)[:, None] * h)
    e = np.concatenate([np.abs(vmx - ex).ravel(), np.abs(vpx - ex).ravel(),
                        np.abs(vmy - ey).ravel(), np.abs(vpy - ey).ravel()])
    return e.mean(), e.max()


@pytest.mark.parametrize("sigma", [-G, G, 0.4])
def test_point_values_third_order_rbf_eno_second_order_eno(sigma):
    """sin(2 pi (x + 2 y)) (v_xx != v_yy, v_xy != 0), switch off: RBF-ENO (MQ) point values at
    third order in L1 and Linf, the ENO stencil at second."""
    ns = (16, 32, 64)
    rbf = [_point_errors(n, sigma, O.Params(k=2, scheme=O.RBF_ENO, cross_2d=1, monotone_switch=0)) for n in ns]
    eno = [_point_errors(n, sigma, O.Params(k=2, scheme=O.ENO)) for n in ns]
    o_rbf = [np.log2(rbf[i][q] / rbf[i + 1][q]) for i in range(2) for q in range(2)]
    o_eno = [np.log2(eno[i][q] / eno[i + 1][q]) for i in range(2) for q in range(2)]
    assert min(o_rbf[2:]) > 2.85, o_rbf
    assert max(o_eno[2:]) < 2.2, o_eno
    assert rbf[-1][0] < eno[-1][0] / 10


def test_example1_gauss_rule_third_order_midpoint_second():
    """Sec. 7 Example 1 (v_t + v_x + v_y = 0, sin(2 pi (x + y)), periodic, T = 0.5, dt = 0.1 dx),
    RBF-ENO k = 2 (MQ) on the cross, switch off, with |eta| <= 1 (the printed k = 2 eta is
    singular where v crosses zero; the bound drops ~0.2% of the evaluations): the Gauss rule
    converges at third order (L1 and Linf), the midpoint rule at second."""
    pg = O.Params(k=2, scheme=O.RBF_ENO, cross_2d=1, gauss_2d=1, monotone_switch=0, eta_max=1.0)
    pm = O.Params(k=2, scheme=O.RBF_ENO, cross_2d=1, monotone_switch=0, eta_max=1.0)
    eg, em = [], []
    for n in (20, 40, 80):
        u0 = _avg_sin(n, 1, 1)  # the exact solution at T = 0.5 (shift 2T = 1) is u0 itself
        for p, out in ((pg, eg), (pm, em)):
            uT, st = O.solve_2d(u0, 1.0 / n, 1.0 / n, 0.5, 0.2, O.ADVECTION, O.PERIODIC, p)
            assert st["eta"]["bound"] <= 0.01 * st["eta"]["eval"]
            e = np.abs(uT - u0)
            out.append((e.mean(), e.max()))
    og = [np.log2(eg[1][q] / eg[2][q]) for q in range(2)]
    om = [np.log2(em[1][q] / em[2][q]) for q in range(2)]
    assert min(og) > 2.8, og
    assert max(om) < 2.2, om
    assert eg[-1][0] < em[-1][0] / 4


def test_gauss_rule_reduces_to_1d_on_x_invariant_data():
    """Data constant along y: the transverse differences vanish, both Gauss points carry the
    midpoint value, and the 2D solve is the 1D solve row by row."""
    n = 24
    x = (np.arange(n) + 0.5) / n
    u1 = np.sin(2 * np.pi * x) + 0.3 * (x > 0.5)
    u2 = np.repeat(u1[None, :], 8, axis=0)
    p1 = O.Params(k=2, scheme=O.RBF_ENO)
    r1, _ = O.solve(u1, 1.0 / n, 0.3, 0.4, O.ADVECTION, O.PERIODIC, p1, max_steps=5)
    p2 = O.Params(k=2, scheme=O.RBF_ENO, cross_2d=1, gauss_2d=1, adv_speed_y=0.0)
    r2, _ = O.solve_2d(u2, 1.0 / n, 1.0 / n, 0.3, 0.4, O.ADVECTION, O.PERIODIC, p2, max_steps=5)
    np.testing.assert_allclose(r2, np.repeat(r1[None, :], 8, axis=0), rtol=0, atol=1e-15)


def test_gauss_rule_needs_k2_and_the_cross():
    u = _avg_sin(12, 1, 1)
    for p in (O.Params(k=3, gauss_2d=1), O.Params(k=2, scheme=O.RBF_ENO, gauss_2d=1, cross_2d=0)):
        with pytest.raises(Exception):
            O.solve_2d(u, 1 / 12, 1 / 12, 0.1, 0.2, O.ADVECTION, O.PERIODIC, p, max_steps=1)
    with pytest.raises(Exception):
        O.reconstruct_2d(u, O.PERIODIC, O.Params(k=3), sigma=0.2)
