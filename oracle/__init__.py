"""FP64 CPU oracle for the non-polynomial ENO/WENO finite-volume method (arXiv 1602.00182).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA library:
the arithmetic lives in ``npw_oracle.c`` (plain loops, double precision, compiled with
``-ffp-contract=off``); this module only builds it and marshals numpy arrays through ctypes.

Paper passages followed (see npw_oracle.c for the per-routine citations):
Sec. 2 (cell averages, stencils, WENO combination eq. weno_re), Sec. 3.5 Table k3
(coefficients and eta; the printed 6/11 is read as 11/6), Sec. 3.3 (Gaussian recipe, k=3
rows derived), Sec. 4 (monotone switch eq. root_value / eq. adaptation), Sec. 5.1 (eq. PDE1,
Lax-Friedrichs flux, TVD-RK3), Sec. 5.2 Example 4 (Euler), Sec. 6 (the 5-cell cross, at the
midpoint or any point of a face), Sec. 7 (eq. 2DIntegral, midpoint or two-point Gauss quadrature).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "npw_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libnpw_oracle.so")

# enumerations of npw_oracle.h
ENO, WENO_JS, RBF_ENO, RBF_WENO = 0, 1, 2, 3
MQ, GA = 0, 1
PERIODIC, TRANSMISSIVE, INFLOW = 0, 1, 2
ADVECTION, BURGERS, EULER1D, EULER2D = 0, 1, 2, 3
FLAG_SWITCH, FLAG_SWITCH_TIE, FLAG_ENO_TIE_L, FLAG_ENO_TIE_R = 0x01, 0x02, 0x40, 0x80
FLAG_SWITCH_R_K2 = 0x08  # k = 2: switch of the right cell of the face (bit 0: left cell)
# zero-reason byte of reconstruct(with_reason=True): the guard or the bound (neither is in the
# paper) set an evaluated shape parameter to 0; _L: eta of v^- (k = 3: the face's eta), _R: of
# v^+ (k = 2)
ZERO_GUARD_L, ZERO_BOUND_L, ZERO_GUARD_R, ZERO_BOUND_R = 0x01, 0x02, 0x04, 0x08
COUNTERS = ("switch", "eval", "guard", "bound")  # order of the counters of npw_oracle.h

SCHEMES = {"eno": ENO, "weno_js": WENO_JS, "rbf_eno": RBF_ENO, "rbf_weno": RBF_WENO}


class _Params(C.Structure):
    _fields_ = [
        ("scheme", C.c_int), ("rbf", C.c_int), ("monotone_switch", C.c_int), ("switch_variant", C.c_int),
        ("characteristic", C.c_int), ("k", C.c_int), ("cross_2d", C.c_int), ("bc_y", C.c_int),
        ("gauss_2d", C.c_int), ("eps_M", C.c_double), ("eps_weno", C.c_double), ("gamma", C.c_double),
        ("adv_speed", C.c_double), ("adv_speed_y", C.c_double), ("inflow", C.c_double * 4),
        ("tie_tol", C.c_double), ("eta_guard", C.c_double), ("eta_max", C.c_double),
        ("counters", C.POINTER(C.c_long)),
    ]


class _Stats(C.Structure):
    _fields_ = [("steps", C.c_long), ("t", C.c_double), ("alpha_max", C.c_double),
                ("status", C.c_int), ("pad_", C.c_int)]


@dataclass
class Params:
    """Method parameters (defaults: RBF-WENO5, multiquadric, switch on)."""
    scheme: int = RBF_WENO
    rbf: int = MQ
    monotone_switch: int = 1
    switch_variant: int = 0
    characteristic: int = 0
    k: int = 3
    cross_2d: int = 0
    bc_y: int = -1  # 2D: boundary of the y direction (-1: the same as the bc argument)
    gauss_2d: int = 0  # 2D, k = 2: two Gauss points per face in eq. 2DIntegral (0: the midpoint)
    eps_M: float = 1e-12
    eps_weno: float = 1e-6
    gamma: float = 1.4
    adv_speed: float = 1.0
    adv_speed_y: float = 1.0
    inflow: tuple = (0.0, 0.0, 0.0, 0.0)
    tie_tol: float = 1e-10
    eta_guard: float = 0.0
    eta_max: float = 0.0  # 0: off, the paper's eta (Table k3); > 0: optional bound |eta| <= eta_max

    def _c(self) -> _Params:
        p = _Params()
        for f in ("scheme", "rbf", "monotone_switch", "switch_variant", "characteristic", "k", "cross_2d", "bc_y", "gauss_2d"):
            setattr(p, f, int(getattr(self, f)))
        for f in ("eps_M", "eps_weno", "gamma", "adv_speed", "adv_speed_y", "tie_tol", "eta_guard", "eta_max"):
            setattr(p, f, float(getattr(self, f)))
        for k in range(4):
            p.inflow[k] = float(self.inflow[k]) if k < len(self.inflow) else 0.0
        p.counters = None
        return p


def _with_counters(p: _Params):
    """Attach a fresh counter array (shape-parameter decisions) to the C params."""
    cnt = (C.c_long * len(COUNTERS))()
    p.counters = C.cast(cnt, C.POINTER(C.c_long))
    return cnt


def _counts(cnt) -> dict:
    return {name: int(cnt[k]) for k, name in enumerate(COUNTERS)}


def build(force: bool = False) -> str:
    """Compile npw_oracle.c into a shared object next to it (gcc, FP64, no contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "npw_oracle.h"))):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, l = C.c_double, C.c_int, C.c_long
        P = C.POINTER
        _lib.orc_table_coef.restype = d
        _lib.orc_table_coef.argtypes = [i, i, i, d]
        _lib.orc_switch_k3.argtypes = [P(d), i, d, P(i)]
        _lib.orc_table_coef_k2.restype = d
        _lib.orc_table_coef_k2.argtypes = [i, i, i, d]
        _lib.orc_switch_k2.argtypes = [P(d), d, P(i)]
        _lib.orc_eta_k2.restype = d
        _lib.orc_eta_k2.argtypes = [P(d), i, P(_Params)]
        _lib.orc_eta_k2_cross.restype = d
        _lib.orc_eta_k2_cross.argtypes = [P(d), i, i, d, P(_Params)]
        _lib.orc_reconstruct_2d.argtypes = [P(d), l, l, i, i, P(_Params), P(d), P(d), P(d), P(d)]
        _lib.orc_reconstruct_2d_at.argtypes = [P(d), l, l, i, i, P(_Params), d, P(d), P(d), P(d), P(d)]
        _lib.orc_eta_k2_point.restype = d
        _lib.orc_eta_k2_point.argtypes = [P(d), i, i, d, d, d, d, P(_Params)]
        _lib.orc_eno_choice.argtypes = [P(d), d, P(i)]
        _lib.orc_beta_k3.argtypes = [P(d), P(d)]
        _lib.orc_euler_eigvec.argtypes = [P(d), P(d), d, P(d), P(d)]
        _lib.orc_reconstruct.argtypes = [P(d), l, i, i, P(_Params), P(d), P(d), P(C.c_uint8), P(d), P(C.c_uint8),
                                         P(C.c_uint8)]
        _lib.orc_flux.argtypes = [P(d), P(d), l, i, i, i, d, P(_Params), P(d)]
        _lib.orc_max_speed.restype = d
        _lib.orc_max_speed.argtypes = [P(d), l, i, i, i, P(_Params)]
        _lib.orc_rk3_step.argtypes = [P(d), l, i, d, d, i, i, P(_Params), P(d)]
        _lib.orc_rk3_step_2d.argtypes = [P(d), l, l, i, d, d, d, i, i, P(_Params)]
        _lib.orc_solve.argtypes = [P(d), l, i, d, d, d, i, i, P(_Params), l, P(_Stats)]
        _lib.orc_solve_2d.argtypes = [P(d), l, l, i, d, d, d, d, i, i, P(_Params), l, P(_Stats)]
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u8p(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_uint8))


def _f64(u) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(u, dtype=np.float64))


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(f"{what}: oracle status {st}")


# ---------------------------------------------------------------------------------------
# pieces, exposed for the pins
# ---------------------------------------------------------------------------------------
def table_coef(rbf: int, r: int, j: int, eta: float) -> float:
    """c_rj(eta) of Table k3 (poly row + eta * perturbation row)."""
    return lib().orc_table_coef(rbf, r, j, eta)


def table_coef_k2(rbf: int, r: int, j: int, eta: float) -> float:
    """c_rj(eta) of Table k2 (poly row + eta * perturbation row), r = -1, 0, 1; j = 0, 1."""
    return lib().orc_table_coef_k2(rbf, r, j, eta)


def switch_k2(c3, tol: float = 0.0):
    """k = 2 switch of a cell from its stencil (cells i-1, i, i+1): (fires, near tie)."""
    c = _f64(c3)
    near = C.c_int(0)
    fires = lib().orc_switch_k2(_dp(c), tol, C.byref(near))
    return bool(fires), bool(near.value)


def eta_k2(c3, side: int, params: "Params") -> float:
    """k = 2 shape parameter of a cell (cells i-1, i, i+1): side 0 for v^-_{i+1/2}, 1 for
    v^+_{i-1/2}."""
    c = _f64(c3)
    p = params._c()
    return lib().orc_eta_k2(_dp(c), side, C.byref(p))


def eta_k2_cross(c3, side: int, central: bool, trans: float, params: "Params") -> float:
    """k = 2 shape parameter on the 5-cell cross (Sec. 6): c3 = cells along the face normal,
    trans = transverse second difference of the cell, central: the stencil of the two cells at
    the face."""
    c = _f64(c3)
    p = params._c()
    return lib().orc_eta_k2_cross(_dp(c), side, int(central), float(trans), C.byref(p))


def eta_k2_point(c3, side: int, central: bool, trans: float, sg: float, xy: float, sigma: float,
                 params: "Params") -> float:
    """k = 2 shape parameter on the 5-cell cross (Sec. 6) at the point sigma (cell widths from
    the face midpoint) of the face: sg = ENO side (+1 / -1) of the transverse neighbour, xy =
    mixed difference with the cell across the face."""
    c = _f64(c3)
    p = params._c()
    return lib().orc_eta_k2_point(_dp(c), side, int(central), float(trans), float(sg), float(xy), float(sigma),
                                  C.byref(p))


GAUSS2 = 0.28867513459481288225  # the two Gauss points of a face: +-1/(2 sqrt 3) cell widths


def reconstruct_2d(u, bc: int, params: "Params", sigma: float = 0.0):
    """Face values of u [m][ny][nx] (or [ny][nx]) at the point sigma of every face (cell widths
    from the midpoint along the face, |sigma| <= 1/2; sigma != 0 needs k = 2): (vmx, vpx)
    [m][ny][nx+1] at the x faces (points at y_j + sigma dy) and (vmy, vpy) [m][ny+1][nx] at the
    y faces (x_i + sigma dx)."""
    u = _f64(u)
    squeeze = u.ndim == 2
    if squeeze:
        u = u[None]
    m, ny, nx = u.shape
    vmx, vpx = np.zeros((m, ny, nx + 1)), np.zeros((m, ny, nx + 1))
    vmy, vpy = np.zeros((m, ny + 1, nx)), np.zeros((m, ny + 1, nx))
    p = params._c()
    _check(lib().orc_reconstruct_2d_at(_dp(u), nx, ny, m, bc, C.byref(p), float(sigma), _dp(vmx), _dp(vpx),
                                       _dp(vmy), _dp(vpy)), "reconstruct_2d")
    if squeeze:
        return vmx[0], vpx[0], vmy[0], vpy[0]
    return vmx, vpx, vmy, vpy


def switch_k3(w4, variant: int = 0, tol: float = 0.0):
    w = _f64(w4)
    near = C.c_int(0)
    fires = lib().orc_switch_k3(_dp(w), variant, tol, C.byref(near))
    return bool(fires), bool(near.value)


def eno_choice(c5, tol: float = 0.0):
    c = _f64(c5)
    near = C.c_int(0)
    r = lib().orc_eno_choice(_dp(c), tol, C.byref(near))
    return r, bool(near.value)


def beta_k3(c5) -> np.ndarray:
    c = _f64(c5)
    out = np.zeros(3)
    lib().orc_beta_k3(_dp(c), _dp(out))
    return out


def euler_eigvec(UL, UR, gamma: float = 1.4):
    """Roe-averaged right eigenvectors R (columns) and L = R^-1 of the 1D Euler Jacobian."""
    a, b = _f64(UL), _f64(UR)
    R = np.zeros((3, 3))
    L = np.zeros((3, 3))
    _check(lib().orc_euler_eigvec(_dp(a), _dp(b), gamma, _dp(R), _dp(L)), "euler_eigvec")
    return R, L


# ---------------------------------------------------------------------------------------
# the method
# ---------------------------------------------------------------------------------------
def reconstruct(u, bc: int, params: Params, replay=None, with_reason: bool = False):
    """Face values of a 1D field set u[m][n] (or u[n]).  Returns (vm, vp, flags, eta),
    each [m][n+1]; face f lies between cell f-1 and cell f.  replay: a flag array of the same
    shape whose switch and ENO decisions are taken instead of the oracle's own.  with_reason:
    also return the zero-reason bytes (ZERO_*) and the decision counts (a dict)."""
    u = _f64(u)
    squeeze = u.ndim == 1
    if squeeze:
        u = u[None, :]
    m, n = u.shape
    vm = np.zeros((m, n + 1))
    vp = np.zeros((m, n + 1))
    flags = np.zeros((m, n + 1), dtype=np.uint8)
    eta = np.zeros((m, n + 1))
    reason = np.zeros((m, n + 1), dtype=np.uint8)
    rp = None if replay is None else np.ascontiguousarray(np.asarray(replay, dtype=np.uint8).reshape(m, n + 1))
    p = params._c()
    cnt = _with_counters(p)
    _check(lib().orc_reconstruct(_dp(u), n, m, bc, C.byref(p), _dp(vm), _dp(vp), _u8p(flags), _dp(eta), _u8p(rp),
                                 _u8p(reason)), "reconstruct")
    out = (vm, vp, flags, eta, reason) if not squeeze else (vm[0], vp[0], flags[0], eta[0], reason[0])
    if with_reason:
        return out + (_counts(cnt),)
    return out[:4]


def flux(vm, vp, kind: int, alpha: float, params: Params, direction: int = 0):
    vm = _f64(vm)
    vp = _f64(vp)
    squeeze = vm.ndim == 1
    if squeeze:
        vm, vp = vm[None, :], vp[None, :]
    m, nf = vm.shape
    h = np.zeros((m, nf))
    p = params._c()
    _check(lib().orc_flux(_dp(vm), _dp(vp), nf, m, kind, direction, alpha, C.byref(p), _dp(h)), "flux")
    return h[0] if squeeze else h


def max_speed(u, kind: int, params: Params, direction: int = 0) -> float:
    u = _f64(u)
    m = 1 if u.ndim == 1 else u.shape[0]
    ncell = u.size // m
    p = params._c()
    return lib().orc_max_speed(_dp(u), ncell, m, kind, direction, C.byref(p))


def rk3_step(u, dx: float, dt: float, kind: int, bc: int, params: Params):
    """One TVD-RK3 step of u[m][n] with alpha from u^n.  Returns (u_new, alpha)."""
    u = _f64(u).copy()
    squeeze = u.ndim == 1
    uu = u[None, :] if squeeze else u
    m, n = uu.shape
    a = C.c_double(0.0)
    p = params._c()
    _check(lib().orc_rk3_step(_dp(uu), n, m, dx, dt, kind, bc, C.byref(p), C.byref(a)), "rk3_step")
    return (uu[0] if squeeze else uu), a.value


def rk3_step_2d(u, dx: float, dy: float, dt: float, kind: int, bc: int, params: Params):
    u = _f64(u).copy()
    squeeze = u.ndim == 2
    uu = u[None] if squeeze else u
    m, ny, nx = uu.shape
    p = params._c()
    _check(lib().orc_rk3_step_2d(_dp(uu), nx, ny, m, dx, dy, dt, kind, bc, C.byref(p)), "rk3_step_2d")
    return uu[0] if squeeze else uu


def solve(u, dx: float, t_end: float, cfl: float, kind: int, bc: int, params: Params, max_steps: int = -1):
    """Advance u[m][n] to t_end.  Returns (u, {'steps','t','alpha_max','status'})."""
    u = _f64(u).copy()
    squeeze = u.ndim == 1
    uu = u[None, :] if squeeze else u
    m, n = uu.shape
    st = _Stats()
    p = params._c()
    cnt = _with_counters(p)
    _check(lib().orc_solve(_dp(uu), n, m, dx, t_end, cfl, kind, bc, C.byref(p), max_steps, C.byref(st)), "solve")
    return (uu[0] if squeeze else uu), dict(steps=st.steps, t=st.t, alpha_max=st.alpha_max, status=st.status,
                                            eta=_counts(cnt))


def solve_2d(u, dx: float, dy: float, t_end: float, cfl: float, kind: int, bc: int, params: Params,
             max_steps: int = -1):
    u = _f64(u).copy()
    squeeze = u.ndim == 2
    uu = u[None] if squeeze else u
    m, ny, nx = uu.shape
    st = _Stats()
    p = params._c()
    cnt = _with_counters(p)
    _check(lib().orc_solve_2d(_dp(uu), nx, ny, m, dx, dy, t_end, cfl, kind, bc, C.byref(p), max_steps,
                              C.byref(st)), "solve_2d")
    return (uu[0] if squeeze else uu), dict(steps=st.steps, t=st.t, alpha_max=st.alpha_max, status=st.status,
                                            eta=_counts(cnt))
