"""Seeded synthetic workloads shaped like the paper's test problems.

This module only builds initial cell averages and instance descriptions: it holds none
of the method's arithmetic.  Both the CUDA path (tests, bench) and the CPU oracle read
their inputs from here.  All averages are exact (closed-form antiderivatives, exact
overlap fractions for jumps), since point sampling would cap the convergence order at 2.

Workloads:
  * advection_sin       -- u_t + u_x = 0 on [-1, 1], periodic, sin(pi x)  (Sec. 5.2, Ex. 1)
  * burgers_batch       -- many periodic Burgers instances on [0, 2 pi], N log-uniform,
                           four Fourier modes + offset 1 + up to two jumps  (Sec. 5.2, Ex. 3
                           family, batched)
  * euler_batch         -- 1D Euler instances, transmissive: Riemann data on [0, 1] and
                           Shu-Osher-type shock/entropy-wave data on [-5, 5]  (Sec. 5.2, Ex. 4
                           family)
  * euler2d_*           -- 2D Euler on periodic squares: isentropic vortex, four-quadrant
                           Riemann data  (Sec. 7 family, dimension by dimension)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 1602_00182
GAMMA = 1.4


def rng(config_index: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_index + 7919 * salt))


# ---------------------------------------------------------------------------------------
# 1D scalar
# ---------------------------------------------------------------------------------------


def advection_sin(n: int, shift: float = 0.0):
    """Exact cell averages of sin(pi (x - shift)) on n uniform cells of [-1, 1]; returns (u, dx)."""
    edges = np.linspace(-1.0, 1.0, n + 1)
    a, b = edges[:-1] - shift, edges[1:] - shift
    u = (np.cos(np.pi * a) - np.cos(np.pi * b)) / (np.pi * (b - a))
    return u, 2.0 / n


@dataclass
class Instance:
    n: int
    dx: float
    t_end: float
    u0: np.ndarray  # [m][n] float64 cell averages
    kind: str = ""


def _fourier_jumps_avg(edges, offset, amps, phases, jumps):
    a, b = edges[:-1], edges[1:]
    w = b - a
    u = np.full(a.shape, offset, dtype=np.float64)
    for mode, (A, ph) in enumerate(zip(amps, phases), start=1):
        u += A * (np.cos(mode * a + ph) - np.cos(mode * b + ph)) / (mode * w)
    for (xj, hj) in jumps:
        u += hj * np.clip((b - xj) / w, 0.0, 1.0)
    return u


def burgers_batch(count: int = 4096, nmin: int = 64, nmax: int = 8192, t_end: float = 1.5, seed_index: int = 1):
    """Periodic Burgers instances on [0, 2 pi].

    N = round(exp(U(ln nmin, ln nmax))); u0 = 1 + sum_{m=1..4} A_m sin(m x + phi_m) with
    A_m ~ U(0, 0.5), phi_m ~ U(0, 2 pi), plus J ~ U{0,1,2} jumps h_j 1[x >= x_j],
    x_j ~ U(0, 2 pi), h_j ~ U(-0.5, 0.5) (the periodic wrap closes each jump at x = 0).
    """
    g = rng(seed_index)
    out = []
    L = 2.0 * np.pi
    for _ in range(count):
        n = int(np.round(np.exp(g.uniform(np.log(nmin), np.log(nmax)))))
        amps = g.uniform(0.0, 0.5, size=4)
        phases = g.uniform(0.0, 2.0 * np.pi, size=4)
        nj = int(g.integers(0, 3))
        jumps = [(g.uniform(0.0, L), g.uniform(-0.5, 0.5)) for _ in range(nj)]
        edges = np.linspace(0.0, L, n + 1)
        u = _fourier_jumps_avg(edges, 1.0, amps, phases, jumps)
        out.append(Instance(n=n, dx=L / n, t_end=t_end, u0=u[None, :], kind="burgers"))
    return out


# ---------------------------------------------------------------------------------------
# 1D Euler
# ---------------------------------------------------------------------------------------


def prim_to_cons(rho, u, p, gamma: float = GAMMA):
    rho, u, p = (np.asarray(v, dtype=np.float64) for v in (rho, u, p))
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def _riemann_instance(g, n):
    rL, rR = g.uniform(0.1, 1.0, size=2)
    uL, uR = g.uniform(-1.0, 1.0, size=2)
    pL, pR = g.uniform(0.1, 1.0, size=2)
    x0 = g.uniform(0.3, 0.7)
    edges = np.linspace(0.0, 1.0, n + 1)
    a, b = edges[:-1], edges[1:]
    fl = np.clip((x0 - a) / (b - a), 0.0, 1.0)  # exact fraction of each cell left of x0
    UL, UR = prim_to_cons(rL, uL, pL), prim_to_cons(rR, uR, pR)
    U = UL[:, None] * fl[None, :] + UR[:, None] * (1.0 - fl[None, :])
    cL, cR = np.sqrt(GAMMA * pL / rL), np.sqrt(GAMMA * pR / rR)
    s_est = max(abs(uL) + cL, abs(uR) + cR) + abs(uL - uR) + abs(cL - cR)
    t_end = float(min(0.25, 0.9 * min(x0, 1.0 - x0) / s_est))
    return Instance(n=n, dx=1.0 / n, t_end=t_end, u0=U, kind="riemann")


def _shu_osher_instance(g, n):
    k = int(g.integers(2, 9))
    gm = GAMMA
    M = 3.0
    # post-shock state of a Mach-M shock running right into (rho=1, u=0, p=1), from the
    # Rankine-Hugoniot conditions
    p2 = 1.0 + 2.0 * gm / (gm + 1.0) * (M * M - 1.0)
    r2 = (gm + 1.0) * M * M / ((gm - 1.0) * M * M + 2.0)
    S = M * np.sqrt(gm)
    u2 = S * (1.0 - 1.0 / r2)
    x0 = -4.0
    edges = np.linspace(-5.0, 5.0, n + 1)
    a, b = edges[:-1], edges[1:]
    w = b - a
    fl = np.clip((x0 - a) / w, 0.0, 1.0)
    # right state: rho = 1 + 0.2 sin(k x), u = 0, p = 1 (exact averages over the part right of x0)
    ar = np.maximum(a, x0)
    rho_r_int = np.where(b > x0, (b - ar) + 0.2 * (np.cos(k * ar) - np.cos(k * b)) / k, 0.0)
    UL = prim_to_cons(r2, u2, p2)
    rho = UL[0] * fl + rho_r_int / w
    mom = UL[1] * fl
    E = UL[2] * fl + (1.0 / (gm - 1.0)) * (1.0 - fl)
    t_end = float(min(1.8, (4.5 - x0 - 0.0) / (1.1 * (S + 1.0))))
    return Instance(n=n, dx=10.0 / n, t_end=t_end, u0=np.stack([rho, mom, E]), kind="shu_osher")


def euler_batch(count: int = 512, nmin: int = 256, nmax: int = 65536, seed_index: int = 2):
    """1D Euler instances (m = 3, gamma = 1.4, transmissive): half Riemann data on [0, 1]
    (rho, p ~ U(0.1, 1), u ~ U(-1, 1) per side, one jump at x0 ~ U(0.3, 0.7)), half
    Shu-Osher-type data on [-5, 5] (Mach-3 shock at x = -4 into rho = 1 + 0.2 sin(k x),
    k ~ U{2..8})."""
    g = rng(seed_index)
    out = []
    for i in range(count):
        n = int(np.round(np.exp(g.uniform(np.log(nmin), np.log(nmax)))))
        out.append(_riemann_instance(g, n) if i % 2 == 0 else _shu_osher_instance(g, n))
    return out


def sod(n: int):
    """Sod shock tube on [-0.5, 0.5] (Sec. 5.2, Ex. 4): (1, 0, 1) | (0.125, 0, 0.1), T = 0.2."""
    edges = np.linspace(-0.5, 0.5, n + 1)
    a, b = edges[:-1], edges[1:]
    fl = np.clip((0.0 - a) / (b - a), 0.0, 1.0)
    UL, UR = prim_to_cons(1.0, 0.0, 1.0), prim_to_cons(0.125, 0.0, 0.1)
    return UL[:, None] * fl[None, :] + UR[:, None] * (1.0 - fl[None, :]), 1.0 / n


# ---------------------------------------------------------------------------------------
# 2D Euler (periodic squares, dimension by dimension)
# ---------------------------------------------------------------------------------------


def _gauss_2d_avg(n, L, fn, npts=4):
    xg, wg = np.polynomial.legendre.leggauss(npts)
    h = L / n
    centres = (np.arange(n) + 0.5) * h
    acc = None
    for a, wa in zip(xg, wg):
        for b, wb in zip(xg, wg):
            X = centres[None, :] + 0.5 * h * a
            Y = centres[:, None] + 0.5 * h * b
            v = fn(np.broadcast_to(X, (n, n)), np.broadcast_to(Y, (n, n))) * (0.25 * wa * wb)
            acc = v if acc is None else acc + v
    return acc


def isentropic_vortex(n: int, strength: float, xc: float, yc: float, L: float = 10.0, gamma: float = GAMMA,
                      npts: int = 4):
    """Isentropic vortex on the periodic square [0, L]^2 over a (1, 1, 1, 1) background;
    returns U[4][n][n] (rho, rho u, rho v, E) cell averages by Gauss quadrature."""
    def prim(X, Y):
        dxp = (X - xc + L / 2) % L - L / 2
        dyp = (Y - yc + L / 2) % L - L / 2
        r2 = dxp * dxp + dyp * dyp
        e = np.exp(0.5 * (1.0 - r2))
        du = -strength / (2 * np.pi) * e * dyp
        dv = strength / (2 * np.pi) * e * dxp
        T = 1.0 - (gamma - 1.0) * strength ** 2 / (8 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
        rho = T ** (1.0 / (gamma - 1.0))
        return rho, 1.0 + du, 1.0 + dv, rho * T

    comps = []
    for k in range(4):
        def fk(X, Y, k=k):
            rho, u, v, p = prim(X, Y)
            return [rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)][k]
        comps.append(_gauss_2d_avg(n, L, fk, npts))
    return np.stack(comps), L / n


def four_quadrant(n: int, g: np.random.Generator, L: float = 1.0, gamma: float = GAMMA):
    """Piecewise-constant four-quadrant data split at the centre: rho, p ~ U(0.1, 1),
    u, v ~ U(-1, 1) per quadrant.  Returns U[4][n][n] and the cell size."""
    U = np.zeros((4, n, n))
    half = n // 2
    for qy in range(2):
        for qx in range(2):
            rho, p = g.uniform(0.1, 1.0, size=2)
            u, v = g.uniform(-1.0, 1.0, size=2)
            sl = (slice(qy * half, n if qy else half), slice(qx * half, n if qx else half))
            U[0][sl] = rho
            U[1][sl] = rho * u
            U[2][sl] = rho * v
            U[3][sl] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return U, L / n


def euler2d_batch(n: int, count: int, seed_index: int = 3):
    """count periodic squares of n x n cells, half isentropic vortices (strength U(3, 5),
    random centre, domain [0, 10]^2) and half four-quadrant data on [0, 1]^2."""
    g = rng(seed_index, salt=n)
    out = []
    for i in range(count):
        if i % 2 == 0:
            U, d = isentropic_vortex(n, g.uniform(3.0, 5.0), g.uniform(0.0, 10.0), g.uniform(0.0, 10.0), npts=2)
        else:
            U, d = four_quadrant(n, g)
        out.append((U, d))
    return out
