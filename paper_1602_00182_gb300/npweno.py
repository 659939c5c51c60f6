"""Thin Python binding of libnpweno (include/npweno.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module passes device pointers of
torch tensors, sizes, the parameter struct and the current CUDA stream.  There is no CPU
fallback: if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnpweno.so")

# enums of npweno.h
NPW_OK, NPW_EINVAL, NPW_ENOMEM, NPW_ECUDA, NPW_ETIMEOUT, NPW_ENONFINITE, NPW_EBUSY = 0, -1, -2, -3, -4, -5, -6
NPW_FLUX_ADVECTION, NPW_FLUX_BURGERS, NPW_FLUX_EULER1D, NPW_FLUX_EULER2D = 0, 1, 2, 3
NPW_BC_PERIODIC, NPW_BC_TRANSMISSIVE, NPW_BC_INFLOW = 0, 1, 2
NPW_ENO, NPW_WENO_JS, NPW_RBF_ENO, NPW_RBF_WENO = 0, 1, 2, 3
NPW_RBF_MQ, NPW_RBF_GA = 0, 1
NPW_FP64, NPW_FP32_MIXED = 0, 1


class npw_params(C.Structure):
    _fields_ = [("k", C.c_int32), ("scheme", C.c_int32), ("rbf", C.c_int32), ("monotone_switch", C.c_int32),
                ("switch_variant", C.c_int32), ("characteristic", C.c_int32), ("precision", C.c_int32),
                ("eta_eval", C.c_int32), ("eps_M", C.c_double), ("eps_weno", C.c_double), ("gamma", C.c_double),
                ("adv_speed", C.c_double), ("adv_speed_y", C.c_double), ("inflow", C.c_double * 4),
                ("eta_guard", C.c_double), ("batch_mode", C.c_int32), ("tile_1d", C.c_int32),
                ("eta_max", C.c_double), ("cross_2d", C.c_int32), ("bc_y", C.c_int32), ("tie_tol", C.c_double),
                ("max_steps", C.c_int64), ("gauss_2d", C.c_int32), ("reserved_", C.c_int32)]


class npw_solve_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("t", C.c_double), ("alpha_max", C.c_double), ("status", C.c_int32),
                ("pad_", C.c_int32), ("eta_switch", C.c_int64), ("eta_eval", C.c_int64), ("eta_guard", C.c_int64),
                ("eta_bound", C.c_int64)]


class npw_instance(C.Structure):
    _fields_ = [("offset", C.c_int64), ("n", C.c_int64), ("dx", C.c_double), ("t_end", C.c_double),
                ("cfl", C.c_double), ("bc", C.c_int32), ("pad_", C.c_int32)]


class NpwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"npweno status {status}: {msg}")
        self.status = status


@dataclass
class Params:
    """Python mirror of npw_params (defaults = npw_default_params)."""
    scheme: int = NPW_RBF_WENO
    rbf: int = NPW_RBF_MQ
    monotone_switch: int = 1
    switch_variant: int = 0
    characteristic: int = 0
    precision: int = NPW_FP64
    eta_eval: int = 0
    eps_M: float = 1e-12
    eps_weno: float = 1e-6
    gamma: float = 1.4
    adv_speed: float = 1.0
    adv_speed_y: float = 1.0
    inflow: Sequence[float] = (0.0, 0.0, 0.0, 0.0)
    eta_guard: float = 0.0
    batch_mode: int = 0
    eta_max: float = 0.0
    k: int = 3
    tile_1d: int = 0
    cross_2d: int = 0
    bc_y: int = -1  # 2D: boundary of the y direction (-1: the bc argument)
    tie_tol: float = 0.0  # near-tie margin of npweno_reconstruct's flags (0: 1e-10)
    max_steps: int = 0  # step limit of a solve (0: automatic); NPW_ETIMEOUT when reached
    gauss_2d: int = 0  # 2D, k = 2: two Gauss points per face (0: the midpoint)

    def c(self) -> npw_params:
        p = npw_params()
        for f in ("k", "scheme", "rbf", "monotone_switch", "switch_variant", "characteristic", "precision",
                  "eta_eval", "batch_mode", "tile_1d", "cross_2d", "bc_y", "max_steps",
                  "gauss_2d"):
            setattr(p, f, int(getattr(self, f)))
        for f in ("eps_M", "eps_weno", "gamma", "adv_speed", "adv_speed_y", "eta_guard", "eta_max", "tie_tol"):
            setattr(p, f, float(getattr(self, f)))
        for i in range(4):
            p.inflow[i] = float(self.inflow[i]) if i < len(self.inflow) else 0.0
        return p


_lib = None


def load():
    """Load libnpweno.so (built by paper_1602_00182_gb300.build).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1602_00182_gb300.build` "
                           "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, d, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    P = C.POINTER
    lib.npw_default_params.argtypes = [P(npw_params)]
    lib.npw_default_params.restype = None
    lib.npw_last_error.restype = C.c_char_p
    lib.npw_version.restype = i32
    lib.npweno_reconstruct.argtypes = [vp, i64, i32, i32, P(npw_params), vp, vp, vp, vp, vp]
    lib.npweno_flux.argtypes = [vp, vp, i64, i32, i32, d, P(npw_params), vp, vp]
    lib.npw_workspace_size.argtypes = [i64, i32, P(npw_params)]
    lib.npw_workspace_size.restype = sz
    lib.npweno_rk3_step.argtypes = [vp, i64, i32, d, d, i32, i32, P(npw_params), vp, sz, P(d), vp]
    lib.npweno_solve.argtypes = [vp, i64, i32, d, d, d, i32, i32, P(npw_params), vp, sz, P(npw_solve_stats), vp]
    lib.npw_batch_workspace_size.argtypes = [P(npw_instance), i32, i32, P(npw_params)]
    lib.npw_batch_workspace_size.restype = sz
    lib.npweno_batch_solve.argtypes = [vp, P(npw_instance), i32, i32, i32, P(npw_params), vp, sz,
                                       P(npw_solve_stats), vp]
    lib.npw_workspace_size_2d.argtypes = [i64, i64, i32, P(npw_params)]
    lib.npw_workspace_size_2d.restype = sz
    lib.npweno_rk3_step_2d.argtypes = [vp, i64, i64, i32, d, d, d, i32, i32, P(npw_params), vp, sz, vp]
    lib.npweno_solve_2d.argtypes = [vp, i64, i64, i32, d, d, d, d, i32, i32, P(npw_params), vp, sz,
                                    P(npw_solve_stats), vp]
    lib.npweno_rk3_step_noalloc.argtypes = [vp, i64, i32, d, d, i32, i32, P(npw_params), vp]
    lib.npw_noalloc_scratch_bytes.restype = sz
    lib.npw_autotune_scratch_bytes.argtypes = [i32, P(npw_params)]
    lib.npw_autotune_scratch_bytes.restype = sz
    lib.npw_autotune_1d.argtypes = [i32, i32, P(npw_params), vp, sz, vp, P(i32)]
    lib.npw_format_check.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.npw_queue_workspace_size.argtypes = [P(npw_queue_instance), i32, P(npw_params)]
    lib.npw_queue_workspace_size.restype = sz
    lib.npweno_queue_solve.argtypes = [vp, P(npw_queue_instance), i32, P(npw_params), vp, sz, P(npw_solve_stats), vp]
    for f in ("npweno_reconstruct", "npweno_flux", "npweno_rk3_step", "npweno_solve", "npweno_batch_solve",
              "npweno_rk3_step_2d", "npweno_solve_2d", "npweno_rk3_step_noalloc", "npw_autotune_1d",
              "npw_format_check", "npweno_queue_solve"):
        getattr(lib, f).restype = i32
    _lib = lib
    return lib


def _check(st: int):
    if st != NPW_OK:
        raise NpwError(st, load().npw_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libnpweno needs a CUDA GPU (there is no CPU fallback)")
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dtype(params: Params):
    torch = _torch()
    return torch.float32 if params.precision == NPW_FP32_MIXED else torch.float64


def _dev(t, params: Params, name: str):
    torch = _torch()
    if not (t.is_cuda and t.is_contiguous() and t.dtype == _dtype(params)):
        raise ValueError(f"{name} must be a contiguous CUDA tensor of dtype {_dtype(params)}")
    return C.c_void_p(t.data_ptr())


def npw_default_params() -> Params:
    return Params()


def npw_version() -> int:
    return load().npw_version()


def npweno_reconstruct(vbar, bc: int, params: Params, with_flags: bool = True, with_eta: bool = False):
    """Face values of vbar [m][n] (or [n]) -> (v_minus, v_plus, flags[, eta]), each [m][n+1]."""
    torch = _torch()
    squeeze = vbar.dim() == 1
    v = vbar[None] if squeeze else vbar
    m, n = v.shape
    vm = torch.empty((m, n + 1), dtype=v.dtype, device=v.device)
    vp = torch.empty_like(vm)
    fl = torch.empty((m, n + 1), dtype=torch.uint8, device=v.device) if with_flags else None
    eta = torch.empty_like(vm) if with_eta else None
    p = params.c()
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    _check(load().npweno_reconstruct(_dev(v, params, "vbar"), n, m, bc, C.byref(p), ptr(vm), ptr(vp), ptr(fl),
                                     ptr(eta), _stream()))
    out = (vm, vp, fl) + ((eta,) if with_eta else ())
    if squeeze:
        return tuple(x[0] if x is not None else None for x in out)
    return out


def npweno_flux(v_minus, v_plus, flux_kind: int, alpha: float, params: Params):
    torch = _torch()
    squeeze = v_minus.dim() == 1
    a = v_minus[None] if squeeze else v_minus
    b = v_plus[None] if squeeze else v_plus
    m, nf = a.shape
    h = torch.empty_like(a)
    p = params.c()
    _check(load().npweno_flux(_dev(a, params, "v_minus"), _dev(b, params, "v_plus"), nf, m, flux_kind, float(alpha),
                              C.byref(p), C.c_void_p(h.data_ptr()), _stream()))
    return h[0] if squeeze else h


def npw_workspace_size(n: int, m: int, params: Params) -> int:
    p = params.c()
    return int(load().npw_workspace_size(n, m, C.byref(p)))


def _workspace(nbytes: int, device, given=None):
    torch = _torch()
    if given is not None:
        if given.numel() * given.element_size() < nbytes:
            raise ValueError("workspace too small")
        return given
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)


def npweno_rk3_step(u, dx: float, dt: float, flux_kind: int, bc: int, params: Params, workspace=None,
                    want_alpha: bool = False) -> Optional[float]:
    """One TVD-RK3 step of u [m][n] (or [n]) in place; returns alpha if want_alpha."""
    uu = u[None] if u.dim() == 1 else u
    m, n = uu.shape
    nbytes = npw_workspace_size(n, m, params)
    ws = _workspace(nbytes, u.device, workspace)
    p = params.c()
    a = C.c_double(0.0)
    _check(load().npweno_rk3_step(_dev(uu, params, "u"), n, m, float(dx), float(dt), flux_kind, bc, C.byref(p),
                                  C.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size(),
                                  C.byref(a) if want_alpha else None, _stream()))
    return a.value if want_alpha else None


def npweno_rk3_step_noalloc(u, dx: float, dt: float, flux_kind: int, bc: int, params: Params):
    """npweno_rk3_step without a workspace: the library's fixed scratch array is used (for
    callers that cannot allocate device memory; see include/npweno.h for the size limit and
    the rule that calls must not overlap on the GPU)."""
    uu = u[None] if u.dim() == 1 else u
    m, n = uu.shape
    p = params.c()
    _check(load().npweno_rk3_step_noalloc(_dev(uu, params, "u"), n, m, float(dx), float(dt), flux_kind, bc,
                                          C.byref(p), _stream()))


def npw_format_check(f_in, d_in):
    """Run the library's integer float<->double format changes on the device tensors f_in
    (float32) and d_in (float64, same length) next to the hardware conversions; returns a dict
    of device tensors (see include/npweno.h)."""
    import torch
    if f_in.dtype != torch.float32 or d_in.dtype != torch.float64 or f_in.numel() != d_in.numel():
        raise ValueError("f_in must be float32 and d_in float64 of the same length")
    if not (f_in.is_cuda and d_in.is_cuda and f_in.is_contiguous() and d_in.is_contiguous()):
        raise ValueError("f_in and d_in must be contiguous CUDA tensors")
    cnt = f_in.numel()
    out = dict(widen=torch.empty(cnt, dtype=torch.float64, device=f_in.device),
               widen_nz=torch.empty(cnt, dtype=torch.float64, device=f_in.device),
               narrow=torch.empty(cnt, dtype=torch.float32, device=f_in.device),
               seed=torch.empty(cnt, dtype=torch.float32, device=f_in.device),
               flags=torch.empty(cnt, dtype=torch.int32, device=f_in.device),
               hw_widen=torch.empty(cnt, dtype=torch.float64, device=f_in.device),
               hw_narrow=torch.empty(cnt, dtype=torch.float32, device=f_in.device))
    ptr = lambda t: C.c_void_p(t.data_ptr())
    _check(load().npw_format_check(ptr(f_in), ptr(d_in), cnt, ptr(out["widen"]), ptr(out["widen_nz"]),
                                   ptr(out["narrow"]), ptr(out["seed"]), ptr(out["flags"]), ptr(out["hw_widen"]),
                                   ptr(out["hw_narrow"]), _stream()))
    return out


def _stats(s: npw_solve_stats) -> dict:
    return dict(steps=int(s.steps), t=float(s.t), alpha_max=float(s.alpha_max), status=int(s.status),
                eta=dict(switch=int(s.eta_switch), eval=int(s.eta_eval), guard=int(s.eta_guard),
                         bound=int(s.eta_bound)))


def npweno_solve(u, dx: float, t_end: float, cfl: float, flux_kind: int, bc: int, params: Params, workspace=None):
    """Advance u [m][n] (or [n]) in place to t_end; returns the statistics dict."""
    uu = u[None] if u.dim() == 1 else u
    m, n = uu.shape
    nbytes = npw_workspace_size(n, m, params)
    ws = _workspace(nbytes, u.device, workspace)
    p = params.c()
    st = npw_solve_stats()
    _check(load().npweno_solve(_dev(uu, params, "u"), n, m, float(dx), float(t_end), float(cfl), flux_kind, bc,
                               C.byref(p), C.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size(), C.byref(st),
                               _stream()))
    return _stats(st)


def make_instances(ns: Sequence[int], dxs: Sequence[float], t_ends: Sequence[float], cfls: Sequence[float],
                   bcs: Sequence[int], m: int = 1):
    """Instance table for a packed arena: instance i occupies [off_i, off_i + m*n_i)."""
    arr = (npw_instance * len(ns))()
    off = 0
    for i, n in enumerate(ns):
        arr[i].offset = off
        arr[i].n = int(n)
        arr[i].dx = float(dxs[i])
        arr[i].t_end = float(t_ends[i])
        arr[i].cfl = float(cfls[i])
        arr[i].bc = int(bcs[i])
        off += m * int(n)
    return arr, off


def npw_batch_workspace_size(instances, m: int, params: Params) -> int:
    p = params.c()
    return int(load().npw_batch_workspace_size(instances, len(instances), m, C.byref(p)))


def npw_autotune_1d(flux_kind: int, m: int, params: Params, device=None) -> int:
    """Time the 1D per-stage kernels with each tile size on a synthetic 2^21-cell instance
    (scratch allocated here) and return the fastest; later runs with tile_1d = 0 use it."""
    import torch
    p = params.c()
    lib = load()
    nbytes = lib.npw_autotune_scratch_bytes(m, C.byref(p))
    if nbytes == 0:
        raise NpwError(NPW_EINVAL, "npw_autotune_scratch_bytes: bad arguments")
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    best = C.c_int32(0)
    _check(lib.npw_autotune_1d(flux_kind, m, C.byref(p), C.c_void_p(scratch.data_ptr()), nbytes, _stream(),
                               C.byref(best)))
    return best.value


def npweno_batch_solve(arena, instances, m: int, flux_kind: int, params: Params, workspace=None,
                       raise_on_error: bool = True):
    """Advance every instance of the packed arena (device) to its t_end; returns (status,
    list of per-instance stats)."""
    count = len(instances)
    nbytes = npw_batch_workspace_size(instances, m, params)
    ws = _workspace(nbytes, arena.device, workspace)
    p = params.c()
    out = (npw_solve_stats * count)()
    st = load().npweno_batch_solve(_dev(arena, params, "arena"), instances, count, m, flux_kind, C.byref(p),
                                   C.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size(), out, _stream())
    if raise_on_error and st not in (NPW_OK, NPW_ENONFINITE):
        _check(st)
    return st, [_stats(out[i]) for i in range(count)]


class npw_queue_instance(C.Structure):
    _fields_ = [("offset", C.c_int64), ("nx", C.c_int64), ("ny", C.c_int64), ("dx", C.c_double), ("dy", C.c_double),
                ("t_end", C.c_double), ("cfl", C.c_double), ("flux_kind", C.c_int32), ("bc", C.c_int32),
                ("bc_y", C.c_int32), ("pad_", C.c_int32)]


_KIND_M = {NPW_FLUX_ADVECTION: 1, NPW_FLUX_BURGERS: 1, NPW_FLUX_EULER1D: 3, NPW_FLUX_EULER2D: 4}


def make_queue_instances(specs):
    """Descriptor table of a work-queue batch packed into one arena.  specs: dicts with keys
    kind, nx, (ny, dy for 2D), dx, t_end, cfl, bc, (bc_y); instance i occupies
    [off_i, off_i + m * nx * max(ny, 1)).  Returns (table, total elements, offsets)."""
    arr = (npw_queue_instance * len(specs))()
    off, offs = 0, []
    for i, sp in enumerate(specs):
        ny = int(sp.get("ny", 0))
        arr[i].offset = off
        arr[i].nx = int(sp["nx"])
        arr[i].ny = ny
        arr[i].dx = float(sp["dx"])
        arr[i].dy = float(sp.get("dy", 0.0))
        arr[i].t_end = float(sp["t_end"])
        arr[i].cfl = float(sp["cfl"])
        arr[i].flux_kind = int(sp["kind"])
        arr[i].bc = int(sp.get("bc", NPW_BC_PERIODIC))
        arr[i].bc_y = int(sp.get("bc_y", -1))
        offs.append(off)
        off += _KIND_M[int(sp["kind"])] * int(sp["nx"]) * max(ny, 1)
    return arr, off, offs


def npw_queue_workspace_size(instances, params: Params) -> int:
    p = params.c()
    return int(load().npw_queue_workspace_size(instances, len(instances), C.byref(p)))


def npweno_queue_solve(arena, instances, params: Params, workspace=None, raise_on_error: bool = True):
    """Advance every instance (1D and 2D) of the packed arena through the work-queue kernel;
    returns (status, list of per-instance stats)."""
    count = len(instances)
    nbytes = npw_queue_workspace_size(instances, params)
    if nbytes == 0:
        raise NpwError(NPW_EINVAL, "npw_queue_workspace_size: bad instances or params")
    ws = _workspace(nbytes, arena.device, workspace)
    p = params.c()
    out = (npw_solve_stats * count)()
    st = load().npweno_queue_solve(_dev(arena, params, "arena"), instances, count, C.byref(p),
                                   C.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size(), out, _stream())
    if raise_on_error and st not in (NPW_OK, NPW_ENONFINITE, NPW_ETIMEOUT):
        _check(st)
    return st, [_stats(out[i]) for i in range(count)]


def npw_workspace_size_2d(nx: int, ny: int, m: int, params: Params) -> int:
    p = params.c()
    return int(load().npw_workspace_size_2d(nx, ny, m, C.byref(p)))


def npweno_rk3_step_2d(u, dx: float, dy: float, dt: float, flux_kind: int, bc: int, params: Params,
                       workspace=None):
    uu = u[None] if u.dim() == 2 else u
    m, ny, nx = uu.shape
    ws = _workspace(npw_workspace_size_2d(nx, ny, m, params), u.device, workspace)
    p = params.c()
    _check(load().npweno_rk3_step_2d(_dev(uu, params, "u"), nx, ny, m, float(dx), float(dy), float(dt), flux_kind,
                                     bc, C.byref(p), C.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size(),
                                     _stream()))


def npweno_solve_2d(u, dx: float, dy: float, t_end: float, cfl: float, flux_kind: int, bc: int, params: Params,
                    workspace=None):
    uu = u[None] if u.dim() == 2 else u
    m, ny, nx = uu.shape
    ws = _workspace(npw_workspace_size_2d(nx, ny, m, params), u.device, workspace)
    p = params.c()
    st = npw_solve_stats()
    _check(load().npweno_solve_2d(_dev(uu, params, "u"), nx, ny, m, float(dx), float(dy), float(t_end), float(cfl),
                                  flux_kind, bc, C.byref(p), C.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size(),
                                  C.byref(st), _stream()))
    return _stats(st)


# ---------------------------------------------------------------------------------------
# request server
# ---------------------------------------------------------------------------------------
class npw_request(C.Structure):
    _fields_ = [("flux_kind", C.c_int32), ("bc", C.c_int32), ("n", C.c_int64), ("dx", C.c_double),
                ("t_end", C.c_double), ("cfl", C.c_double), ("u0_host", C.c_void_p), ("out_host", C.c_void_p),
                ("tag", C.c_uint64), ("ny", C.c_int64), ("dy", C.c_double), ("bc_y", C.c_int32),
                ("reserved_", C.c_int32), ("tolerance", C.c_double)]


class npw_result(C.Structure):
    _fields_ = [("id", C.c_uint64), ("tag", C.c_uint64), ("status", C.c_int32), ("precision", C.c_int32),
                ("steps", C.c_int64), ("t", C.c_double), ("submit_s", C.c_double), ("admit_s", C.c_double),
                ("done_s", C.c_double)]


MIXED_TOLERANCE = 1e-4  # requests with a tolerance at least this large take the mixed-precision lane


def _server_protos(lib):
    if getattr(lib, "_server_protos", False):
        return
    P, vp, i32, i64, sz = C.POINTER, C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
    lib.npw_server_arena_bytes.argtypes = [i64, i32, P(npw_params)]
    lib.npw_server_arena_bytes.restype = sz
    lib.npw_server_create.argtypes = [vp, sz, i32, P(npw_params), vp, P(vp)]
    lib.npw_server_create.restype = i32
    lib.npw_server_submit.argtypes = [vp, P(npw_request), P(C.c_uint64)]
    lib.npw_server_submit.restype = i32
    lib.npw_server_step.argtypes = [vp, i32, P(i32), P(i32)]
    lib.npw_server_step.restype = i32
    lib.npw_server_poll.argtypes = [vp, P(npw_result), i32, P(i32)]
    lib.npw_server_poll.restype = i32
    lib.npw_server_destroy.argtypes = [vp]
    lib.npw_server_destroy.restype = None
    lib._server_protos = True


class Server:
    """npw_server_*: continuous batching of 1D and 2D solves on one device arena (allocated here
    with torch, owned by this object), one lane per precision: a request's tolerance picks its
    lane (>= MIXED_TOLERANCE: NPW_FP32_MIXED, below: NPW_FP64, 0: params.precision).  Host
    arrays of each request are kept alive until polled."""

    def __init__(self, heap_cells: int, max_slots: int, params: Params, device=None):
        torch = _torch()
        lib = load()
        _server_protos(lib)
        self.params = params
        self._p = params.c()
        nbytes = int(lib.npw_server_arena_bytes(heap_cells, max_slots, C.byref(self._p)))
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")
        self.stream = torch.cuda.current_stream(self.arena.device)
        h = C.c_void_p()
        _check(lib.npw_server_create(C.c_void_p(self.arena.data_ptr()), nbytes, max_slots, C.byref(self._p),
                                     C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h
        self._keep = {}

    def lane_precision(self, tolerance: float) -> int:
        if tolerance > 0.0:
            return NPW_FP32_MIXED if tolerance >= MIXED_TOLERANCE else NPW_FP64
        return self.params.precision

    def submit(self, u0, flux_kind: int, bc: int, dx: float, t_end: float, cfl: float, tag: int = 0,
               dy: float = 0.0, bc_y: int = -1, tolerance: float = 0.0) -> int:
        """1D: u0 is [m][n] (or [n]); 2D (dy > 0): u0 is [m][ny][nx] (or [ny][nx]).  tolerance
        picks the precision lane (0: the server's precision)."""
        import numpy as np
        dtype = "float32" if self.lane_precision(tolerance) == NPW_FP32_MIXED else "float64"
        a = np.ascontiguousarray(np.asarray(u0, dtype=dtype))
        m = {NPW_FLUX_EULER1D: 3, NPW_FLUX_EULER2D: 4}.get(flux_kind, 1)
        if dy > 0.0:
            ny, n = a.shape[-2], a.shape[-1]
        else:
            ny, n = 0, a.size // m
        out = np.empty_like(a)
        r = npw_request(flux_kind, bc, n, dx, t_end, cfl, a.ctypes.data, out.ctypes.data, tag, ny, dy, bc_y, 0,
                        float(tolerance))
        rid = C.c_uint64(0)
        _check(load().npw_server_submit(self._h, C.byref(r), C.byref(rid)))
        self._keep[rid.value] = (a, out)
        return rid.value

    def step(self, max_steps: int = 32):
        act, q = C.c_int32(0), C.c_int32(0)
        _check(load().npw_server_step(self._h, max_steps, C.byref(act), C.byref(q)))
        return act.value, q.value

    def poll(self, max_results: int = 1024):
        buf = (npw_result * max_results)()
        nout = C.c_int32(0)
        _check(load().npw_server_poll(self._h, buf, max_results, C.byref(nout)))
        out = []
        for k in range(nout.value):
            r = buf[k]
            a, res = self._keep.pop(r.id)
            out.append(dict(id=r.id, tag=r.tag, status=r.status, precision=r.precision, steps=r.steps, t=r.t,
                            submit_s=r.submit_s, admit_s=r.admit_s, done_s=r.done_s, u=res))
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().npw_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
