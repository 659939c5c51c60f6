"""The paper's discontinuous-advection experiments through the CUDA path, k = 2 and k = 3:
Sec. 5.2 Example 2 (-sgn(x) on [-1, 1], inflow value 1 at x = -1, N = 200, T = 0.5) and Sec. 7
Example 2 (a jump across y = 0.5 on [0, 1]^2, inflow value 1 at y = 0, periodic in x, N = 100).

  * NPW_FP64 against the oracle: relative L_inf <= 1e-12.
  * NPW_FP32_MIXED: near the oracle (mean difference per cell <= 1e-4, largest <= 5e-3: decisions
    at the jump are near ties, see MIXED_MEAN), and ENO / RBF-ENO stay non-oscillatory (within
    [-1, 1] up to float rounding, no new variation), as the paper states.  These runs drop the
    face values where the printed k = 2 eta is singular (its denominator crosses zero inside the
    jump from 1 to -1) with the optional bound on both sides, the setting under which the oracle
    reproduces the paper's statements about this example: |eta| <= 100 in 2D, |eta| <= 1 in 1D
    (with coefficients up to 600 the float candidates are not within 1e-4 of the FP64 ones).
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHEMES = [O.ENO, O.WENO_JS, O.RBF_ENO, O.RBF_WENO]


@pytest.fixture(scope="module")
def npw():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_00182_gb300 import build as b
    b.build()
    import paper_1602_00182_gb300.npweno as m
    m.load()
    return m


def _example2(n=200):
    edges = np.linspace(-1, 1, n + 1)
    return np.where(edges[1:] <= 0, 1.0, -1.0), 2.0 / n


def _gpu_solve(npw, u0, dx, k, scheme, precision, eta_max=0.0):
    dtype = torch.float64 if precision == 0 else torch.float32
    u = torch.tensor(u0, dtype=dtype, device="cuda")
    p = npw.Params(k=k, scheme=scheme, precision=precision, inflow=(1.0, 0, 0, 0), eta_max=eta_max)
    st = npw.npweno_solve(u, dx, 0.5, 0.1, npw.NPW_FLUX_ADVECTION, npw.NPW_BC_INFLOW, p)
    assert st["status"] == 0
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64), st


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_example2_fp64_matches_oracle(npw, k, scheme):
    u0, dx = _example2()
    ref, ost = O.solve(u0, dx, 0.5, 0.1, O.ADVECTION, O.INFLOW, O.Params(k=k, scheme=scheme, inflow=(1.0, 0, 0, 0)))
    got, st = _gpu_solve(npw, u0, dx, k, scheme, 0)
    assert st["steps"] == ost["steps"]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


# At the jump the ENO-choice and switch decisions are near ties: moving the initial data by
# 2^-24 relative (the float rounding of a state) changes the oracle's own FP64 result by up to
# 1.1e-3 for RBF-ENO2 and 1.3e-4 for RBF-ENO3 (measured, seeds 0-4), on a few cells at the
# front.  A float run differs from the FP64 run in the same way, so its bar is on the mean
# difference per cell, with a loose bound on the largest one.
MIXED_MEAN, MIXED_MAX = 1e-4, 5e-3


def _close(got, ref):
    diff = np.abs(got - ref)
    assert diff.mean() <= MIXED_MEAN and diff.max() <= MIXED_MAX, (diff.mean(), diff.max())
    return True


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_example2_mixed_matches_oracle_and_eno_stays_monotone(npw, k, scheme):
    u0, dx = _example2()
    p = O.Params(k=k, scheme=scheme, inflow=(1.0, 0, 0, 0), eta_guard=8.0 * 2.0 ** -24, eta_max=1.0)
    ref, _ = O.solve(u0, dx, 0.5, 0.1, O.ADVECTION, O.INFLOW, p)
    got, _ = _gpu_solve(npw, u0, dx, k, scheme, 1, eta_max=1.0)
    assert _close(got, ref)
    if scheme in (O.ENO, O.RBF_ENO):
        tol = 4 * 2.0 ** -24
        assert got.max() <= 1.0 + tol and got.min() >= -1.0 - tol
        assert np.sum(np.abs(np.diff(got))) <= 2.0 + 200 * tol


# ------------------------------------------------------------------------------------ 2D
def _example2_2d(n=100):
    """Sec. 7 Example 2: v = 1 for y <= 0.5, -1 above, on [0, 1]^2; bottom inflow v = 1, periodic
    in x (bc = periodic, bc_y = inflow), transmissive top."""
    edges = np.linspace(0, 1, n + 1)
    return np.repeat(np.where(edges[1:] <= 0.5, 1.0, -1.0)[:, None], n, axis=1), 1.0 / n


@pytest.mark.parametrize("k,scheme,cross", [(2, O.ENO, 0), (2, O.RBF_ENO, 0), (2, O.RBF_ENO, 1), (2, O.RBF_WENO, 1),
                                            (3, O.RBF_ENO, 0), (3, O.RBF_WENO, 0)])
def test_example2_2d_fp64_matches_oracle(npw, k, scheme, cross):
    u0, d = _example2_2d(100)
    ref, ost = O.solve_2d(u0, d, d, 0.25, 0.1, O.ADVECTION, O.PERIODIC,
                          O.Params(k=k, scheme=scheme, cross_2d=cross, inflow=(1.0, 0, 0, 0), bc_y=O.INFLOW))
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    p = npw.Params(k=k, scheme=scheme, cross_2d=cross, inflow=(1.0, 0, 0, 0), bc_y=npw.NPW_BC_INFLOW)
    st = npw.npweno_solve_2d(u, d, d, 0.25, 0.1, npw.NPW_FLUX_ADVECTION, npw.NPW_BC_PERIODIC, p)
    torch.cuda.synchronize()
    assert st["status"] == 0 and st["steps"] == ost["steps"]
    got = u.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("scheme,cross", [(O.ENO, 0), (O.RBF_ENO, 0), (O.RBF_ENO, 1)])
def test_example2_2d_mixed_stays_monotone(npw, scheme, cross):
    """k = 2 as in the paper's figure: the float path stays within [-1, 1] (up to float rounding)
    with no new variation along y, and near the oracle (the bar of the 1D test)."""
    u0, d = _example2_2d(100)
    op = O.Params(k=2, scheme=scheme, cross_2d=cross, inflow=(1.0, 0, 0, 0), bc_y=O.INFLOW, eta_guard=8.0 * 2.0 ** -24,
                  eta_max=100.0)
    ref, _ = O.solve_2d(u0, d, d, 0.25, 0.1, O.ADVECTION, O.PERIODIC, op)
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    p = npw.Params(k=2, scheme=scheme, cross_2d=cross, precision=1, inflow=(1.0, 0, 0, 0), bc_y=npw.NPW_BC_INFLOW,
                   eta_max=100.0)
    st = npw.npweno_solve_2d(u, d, d, 0.25, 0.1, npw.NPW_FLUX_ADVECTION, npw.NPW_BC_PERIODIC, p)
    torch.cuda.synchronize()
    assert st["status"] == 0
    got = u.cpu().numpy().astype(np.float64)
    assert _close(got, ref)
    tol = 4 * 2.0 ** -24
    assert got.max() <= 1.0 + tol and got.min() >= -1.0 - tol
    assert np.abs(np.diff(got, axis=0)).sum(axis=0).max() <= 2.0 + 100 * tol


def test_bc_y_rejects_bad_values(npw):
    u = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        npw.npweno_solve_2d(u, 0.1, 0.1, 0.1, 0.1, npw.NPW_FLUX_ADVECTION, npw.NPW_BC_PERIODIC, npw.Params(bc_y=7))
