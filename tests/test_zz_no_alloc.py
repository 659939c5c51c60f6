"""npweno_rk3_step_noalloc, the entry point for callers that cannot allocate device memory.

It must give the same results as npweno_rk3_step with a caller workspace, call after call
(the fixed scratch array keeps the previous call's contents, so a second call checks that
nothing stale is read).  Collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # the bar of the FP64 parity tests
FP32_TOL = 2e-6    # the single-step bar of the mixed-precision tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_00182_gb300 import build as b
    b.build()
    import paper_1602_00182_gb300.npweno as npw
    L = npw.load()
    return npw, L


def _data(n, seed):
    g = np.random.default_rng(seed)
    x = np.linspace(0, 1, n, endpoint=False)
    u = 1.0 + 0.4 * np.sin(2 * np.pi * 2 * x + g.uniform(0, 6))
    u[x > 0.5] -= 0.3
    return u


@pytest.mark.parametrize("precision,dtype,tol", [(0, torch.float64, FP64_TOL), (1, torch.float32, FP32_TOL)])
@pytest.mark.parametrize("n", [6, 1000, 3001])
def test_noalloc_matches_workspace_entry_point(lib, precision, dtype, tol, n):
    npw, L = lib
    params = npw.Params(rbf=npw.NPW_RBF_GA, precision=precision).c()
    u0 = _data(n, n)
    ua = torch.tensor(u0, dtype=dtype, device="cuda")
    ub = ua.clone()
    ws = torch.empty(L.npw_workspace_size(n, 1, ctypes.byref(params)), dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dx, dt = 1.0 / n, 0.3 / n
    for call in range(2):  # two calls in a row through the C ABI
        st = L.npweno_rk3_step_noalloc(ctypes.c_void_p(ua.data_ptr()), n, 1, dx, dt, npw.NPW_FLUX_BURGERS,
                                       npw.NPW_BC_PERIODIC, ctypes.byref(params), stream)
        assert st == npw.NPW_OK, L.npw_last_error()
        st = L.npweno_rk3_step(ctypes.c_void_p(ub.data_ptr()), n, 1, dx, dt, npw.NPW_FLUX_BURGERS,
                               npw.NPW_BC_PERIODIC, ctypes.byref(params), ctypes.c_void_p(ws.data_ptr()),
                               ws.numel(), None, stream)
        assert st == npw.NPW_OK, L.npw_last_error()
        torch.cuda.synchronize()
        a = ua.cpu().numpy().astype(np.float64)
        b = ub.cpu().numpy().astype(np.float64)
        assert np.abs(a - b).max() <= tol * np.abs(b).max(), call


@pytest.mark.parametrize("precision,dtype,tol", [(0, torch.float64, FP64_TOL), (1, torch.float32, FP32_TOL)])
@pytest.mark.parametrize("char", [0, 1])
def test_noalloc_matches_workspace_entry_point_euler(lib, precision, dtype, tol, char):
    """1D Euler (m = 3), component- and characteristic-wise: a Sod-type state with a smooth
    density wave, two calls in a row."""
    npw, L = lib
    params = npw.Params(precision=precision, characteristic=char).c()
    n = 2500
    x = (np.arange(n) + 0.5) / n
    rho = np.where(x < 0.5, 1.0, 0.125) + 0.05 * np.sin(8 * np.pi * x)
    p = np.where(x < 0.5, 1.0, 0.1)
    U = np.stack([rho, rho * 0.1, p / 0.4 + 0.5 * rho * 0.01])
    ua = torch.tensor(U, dtype=dtype, device="cuda")
    ub = ua.clone()
    ws = torch.empty(L.npw_workspace_size(n, 3, ctypes.byref(params)), dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dx, dt = 1.0 / n, 0.2 / n
    for call in range(2):
        st = L.npweno_rk3_step_noalloc(ctypes.c_void_p(ua.data_ptr()), n, 3, dx, dt, npw.NPW_FLUX_EULER1D,
                                       npw.NPW_BC_TRANSMISSIVE, ctypes.byref(params), stream)
        assert st == npw.NPW_OK, L.npw_last_error()
        st = L.npweno_rk3_step(ctypes.c_void_p(ub.data_ptr()), n, 3, dx, dt, npw.NPW_FLUX_EULER1D,
                               npw.NPW_BC_TRANSMISSIVE, ctypes.byref(params), ctypes.c_void_p(ws.data_ptr()),
                               ws.numel(), None, stream)
        assert st == npw.NPW_OK, L.npw_last_error()
        torch.cuda.synchronize()
        a = ua.cpu().numpy().astype(np.float64)
        b = ub.cpu().numpy().astype(np.float64)
        for k in range(3):
            assert np.abs(a[k] - b[k]).max() <= tol * np.abs(b[k]).max(), (call, k)


@pytest.mark.parametrize("precision,m", [(0, 1), (1, 1), (1, 3)])
def test_noalloc_limit_is_the_workspace_size(lib, precision, m):
    """The largest accepted size is the one whose workspace fits the scratch (about 5.2e5 cells
    times fields in either precision); one more cell is rejected before anything runs."""
    npw, L = lib
    params = npw.Params(precision=precision).c()
    cap = L.npw_noalloc_scratch_bytes()
    lo, hi = 6, 1 << 22
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if L.npw_workspace_size(mid, m, ctypes.byref(params)) <= cap:
            lo = mid
        else:
            hi = mid
    assert 5.0e5 <= lo * m <= 5.3e5, lo * m
    dtype = torch.float64 if precision == 0 else torch.float32
    kind = npw.NPW_FLUX_BURGERS if m == 1 else npw.NPW_FLUX_EULER1D
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    u = torch.ones((m, lo), dtype=dtype, device="cuda")
    u[1:] = 0.0
    if m == 3:
        u[2] = 2.5
    st = L.npweno_rk3_step_noalloc(ctypes.c_void_p(u.data_ptr()), lo, m, 1.0 / lo, 0.1 / lo, kind,
                                   npw.NPW_BC_PERIODIC, ctypes.byref(params), stream)
    assert st == npw.NPW_OK, L.npw_last_error()
    torch.cuda.synchronize()
    v = torch.ones((m, hi), dtype=dtype, device="cuda")
    st = L.npweno_rk3_step_noalloc(ctypes.c_void_p(v.data_ptr()), hi, m, 1.0 / hi, 0.1 / hi, kind,
                                   npw.NPW_BC_PERIODIC, ctypes.byref(params), stream)
    assert st == npw.NPW_EINVAL


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    npw, L = lib
    params = npw.Params().c()
    cap = L.npw_noalloc_scratch_bytes()
    n = cap // 16 + 4096  # two FP64 stage buffers no longer fit
    assert L.npw_workspace_size(n, 1, ctypes.byref(params)) > cap
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = L.npweno_rk3_step_noalloc(ctypes.c_void_p(u.data_ptr()), n, 1, 1.0 / n, 0.1 / n, npw.NPW_FLUX_BURGERS,
                                   npw.NPW_BC_PERIODIC, ctypes.byref(params),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == npw.NPW_EINVAL
    assert b"8 MiB" in L.npw_last_error()
    assert torch.count_nonzero(u).item() == 0  # nothing ran
