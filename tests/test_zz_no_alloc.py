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
