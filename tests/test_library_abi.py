"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every function
include/npweno.h declares (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "npweno.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(npw[e]?\w*)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("npw_status") and n not in ("npw_params",)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("npweno_reconstruct", "npweno_flux", "npweno_rk3_step", "npweno_solve",
                     "npw_workspace_size", "npweno_batch_solve", "npweno_solve_2d", "npw_last_error"):
        assert required in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_1602_00182_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in npweno.h but not exported"


def test_default_params_and_errors_without_gpu():
    from paper_1602_00182_gb300 import build as b
    from paper_1602_00182_gb300 import npweno as npw
    b.build()
    lib = npw.load()
    p = npw.npw_params()
    lib.npw_default_params(ctypes.byref(p))
    assert (p.k, p.scheme, p.rbf, p.monotone_switch, p.precision) == (3, npw.NPW_RBF_WENO, npw.NPW_RBF_MQ, 1, npw.NPW_FP64)
    assert p.eps_weno == 1e-6 and p.gamma == 1.4 and p.eps_M == 1e-12
    # the shape parameter as printed: no bound, no step limit, the default tie margin
    assert p.eta_max == 0.0 and p.max_steps == 0 and p.tie_tol == 0.0
    # one quadrature point per face (the paper's runs) unless the Gauss rule is asked for
    assert p.gauss_2d == 0
    for kw, msg in ((dict(gauss_2d=1), b"k = 2"), (dict(gauss_2d=1, k=2, scheme=npw.NPW_RBF_ENO), b"cross_2d"),
                    (dict(gauss_2d=2), b"gauss_2d")):
        g = npw.Params(**kw).c()
        st = lib.npweno_solve_2d(ctypes.c_void_p(16), 32, 32, 1, 0.1, 0.1, 0.1, 0.5, npw.NPW_FLUX_ADVECTION, 0,
                                 ctypes.byref(g), ctypes.c_void_p(16), 1 << 30, None, None)
        assert st == npw.NPW_EINVAL and msg in lib.npw_last_error(), (kw, lib.npw_last_error())
    # the work queue takes the Gauss rule in FP64 only (the 2D entry points in both precisions)
    table, _, _ = npw.make_queue_instances([dict(kind=npw.NPW_FLUX_ADVECTION, nx=32, ny=32, dx=0.1, dy=0.1,
                                                 t_end=0.5, cfl=0.4)])
    g = npw.Params(gauss_2d=1, k=2, scheme=npw.NPW_ENO, precision=1).c()
    st = lib.npweno_queue_solve(ctypes.c_void_p(16), table, 1, ctypes.byref(g), ctypes.c_void_p(16), 1 << 30, None,
                                None)
    assert st == npw.NPW_EINVAL and b"NPW_FP64" in lib.npw_last_error(), lib.npw_last_error()
    # argument validation happens before any CUDA call
    bad = npw.Params(k=4).c()
    st = lib.npweno_reconstruct(ctypes.c_void_p(16), 100, 1, 0, ctypes.byref(bad), ctypes.c_void_p(16),
                                ctypes.c_void_p(16), None, None, None)
    assert st == npw.NPW_EINVAL and b"k must be 2" in lib.npw_last_error()
    badtile = npw.Params(tile_1d=300).c()
    st = lib.npweno_reconstruct(ctypes.c_void_p(16), 100, 1, 0, ctypes.byref(badtile), ctypes.c_void_p(16),
                                ctypes.c_void_p(16), None, None, None)
    assert st == npw.NPW_EINVAL and b"tile_1d" in lib.npw_last_error()
    assert lib.npw_autotune_scratch_bytes(1, ctypes.byref(npw.Params(precision=1).c())) > (1 << 21) * 4
    good = npw.Params().c()
    st = lib.npweno_reconstruct(ctypes.c_void_p(16), 5, 1, 0, ctypes.byref(good), ctypes.c_void_p(16),
                                ctypes.c_void_p(16), None, None, None)
    assert st == npw.NPW_EINVAL
    assert lib.npw_workspace_size(1000, 1, ctypes.byref(good)) > 2 * 1000 * 8
    assert lib.npw_version() >= 10000


def test_no_cpu_fallback_in_product_path():
    """The binding refuses to run without a GPU rather than computing on the CPU, and the
    package never imports the oracle."""
    import torch
    from paper_1602_00182_gb300 import npweno as npw
    pkg = os.path.join(ROOT, "paper_1602_00182_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            assert "import oracle" not in open(os.path.join(pkg, f)).read()
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError):
            npw.npweno_reconstruct(torch.zeros(10, dtype=torch.float64), 0, npw.Params())


def test_server_arguments_without_gpu():
    """The request server's sizing and argument checks run on the host before any CUDA call: the
    arena grows with the heap and the slot count; a null arena, characteristic or Gauss-rule
    parameters, an arena too small for its slots, and null handles are refused with NPW_EINVAL."""
    from paper_1602_00182_gb300 import build as b
    from paper_1602_00182_gb300 import npweno as npw
    b.build()
    lib = npw.load()
    p = npw.Params(precision=1).c()
    a1 = lib.npw_server_arena_bytes(1 << 20, 64, ctypes.byref(p))
    assert a1 > (1 << 20) * (3 * 4 + 2 * 4 + 3 * 8)  # both lanes' three state buffers, the float carries
    assert lib.npw_server_arena_bytes(1 << 21, 64, ctypes.byref(p)) > a1
    assert lib.npw_server_arena_bytes(1 << 20, 128, ctypes.byref(p)) > a1
    assert lib.npw_server_arena_bytes(0, 64, ctypes.byref(p)) == 0
    assert lib.npw_server_arena_bytes(1 << 20, 0, ctypes.byref(p)) == 0
    h = ctypes.c_void_p()
    cases = ((None, a1, p, b"bad server arguments"),
             (ctypes.c_void_p(256), a1, npw.Params(precision=1, characteristic=1).c(), b"component-wise"),
             (ctypes.c_void_p(256), a1, npw.Params(precision=1, k=2, cross_2d=1, gauss_2d=1).c(), b"gauss_2d"),
             (ctypes.c_void_p(256), 4096, p, b"arena too small"))
    for arena, size, pp, msg in cases:
        st = lib.npw_server_create(arena, size, 64, ctypes.byref(pp), None, ctypes.byref(h))
        assert st == npw.NPW_EINVAL and msg in lib.npw_last_error(), (msg, lib.npw_last_error())
    n = ctypes.c_int32()
    assert lib.npw_server_step(None, 8, None, None) == npw.NPW_EINVAL
    assert lib.npw_server_submit(None, None, None) == npw.NPW_EINVAL
    assert lib.npw_server_poll(None, None, 0, ctypes.byref(n)) == npw.NPW_EINVAL
