"""Exact solutions used to pin the oracle (test infrastructure only).

* linear advection: translation of the initial profile (Sec. 5.2, Example 1);
* Burgers: the smooth solution before the shock by characteristics, u = u0(x - u t)
  (Sec. 5.2, Example 3), and the Riemann solution (shock with the Rankine-Hugoniot speed
  (uL + uR)/2 or a rarefaction fan u = x/t);
* Euler: the exact Riemann solution of the ideal-gas Euler equations (Sec. 5.2, Example 4,
  "the exact solution is also provided"), written from the standard two-wave pressure
  function: a shock branch from the Rankine-Hugoniot conditions and a rarefaction branch
  from the isentropic Riemann invariants, solved by Newton's method for the star pressure.

Cell averages of smooth solutions use Gauss-Legendre quadrature per cell; discontinuous
Riemann solutions are averaged by dense midpoint sampling.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------------------
# linear advection / smooth Burgers
# ---------------------------------------------------------------------------------------


def sin_pi_avg(edges: np.ndarray, shift: float = 0.0) -> np.ndarray:
    """Exact cell averages of sin(pi (x - shift)) over the cells [edges[i], edges[i+1]]."""
    a, b = edges[:-1] - shift, edges[1:] - shift
    return (np.cos(np.pi * a) - np.cos(np.pi * b)) / (np.pi * (b - a))


def gauss_avg(edges: np.ndarray, fn, npts: int = 8) -> np.ndarray:
    """Cell averages of a smooth point function fn(x) by npts-point Gauss-Legendre."""
    xg, wg = np.polynomial.legendre.leggauss(npts)
    a, b = edges[:-1], edges[1:]
    mid, half = 0.5 * (a + b), 0.5 * (b - a)
    x = mid[:, None] + half[:, None] * xg[None, :]
    return (fn(x) * wg[None, :]).sum(axis=1) * 0.5


def burgers_smooth(x: np.ndarray, t: float, u0, du0, iters: int = 60) -> np.ndarray:
    """u(x,t) of u_t + (u^2/2)_x = 0 before shock formation: solve u = u0(x - u t) by Newton."""
    u = u0(x)
    for _ in range(iters):
        g = u - u0(x - u * t)
        dg = 1.0 + t * du0(x - u * t)
        du = g / dg
        u = u - du
        if np.max(np.abs(du)) < 1e-15:
            break
    return u


def burgers_riemann(x: np.ndarray, t: float, x0: float, uL: float, uR: float) -> np.ndarray:
    """Entropy solution of the Burgers Riemann problem centred at x0."""
    xi = (x - x0) / t
    if uL > uR:
        s = 0.5 * (uL + uR)  # Rankine-Hugoniot
        return np.where(xi < s, uL, uR)
    return np.where(xi <= uL, uL, np.where(xi >= uR, uR, xi))


# ---------------------------------------------------------------------------------------
# Euler exact Riemann solver
# ---------------------------------------------------------------------------------------


def _fK(p, rho, pK, cK, g):
    if p > pK:  # shock branch
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        f = (p - pK) * np.sqrt(A / (p + B))
        df = np.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pK) / (B + p))
    else:  # rarefaction branch
        f = 2.0 * cK / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * cK) * (p / pK) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def riemann_star(left, right, gamma: float = 1.4):
    """Star-region pressure and velocity for primitive states (rho, u, p)."""
    rL, uL, pL = left
    rR, uR, pR = right
    g = gamma
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    if 2.0 * (cL + cR) / (g - 1.0) <= uR - uL:
        raise ValueError("vacuum is generated")
    p = max(1e-10, 0.5 * (pL + pR))
    for _ in range(200):
        fL, dL = _fK(p, rL, pL, cL, g)
        fR, dR = _fK(p, rR, pR, cR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        pn = max(1e-12, p - dp)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fK(p, rL, pL, cL, g)
    fR, _ = _fK(p, rR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def riemann_sample(xi: np.ndarray, left, right, gamma: float = 1.4):
    """Primitive (rho, u, p) of the exact solution at similarity coordinates xi = x/t."""
    rL, uL, pL = left
    rR, uR, pR = right
    g = gamma
    ps, us = riemann_star(left, right, g)
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for idx, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pL:  # left shock
                SL = uL - cL * np.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
                if s <= SL:
                    r, v, q = rL, uL, pL
                else:
                    r, v, q = rL * (ps / pL + gm) / (gm * ps / pL + 1.0), us, ps
            else:  # left rarefaction
                csL = cL * (ps / pL) ** ((g - 1.0) / (2.0 * g))
                if s <= uL - cL:
                    r, v, q = rL, uL, pL
                elif s >= us - csL:
                    r, v, q = rL * (ps / pL) ** (1.0 / g), us, ps
                else:
                    v = 2.0 / (g + 1.0) * (cL + (g - 1.0) / 2.0 * uL + s)
                    c = 2.0 / (g + 1.0) * (cL + (g - 1.0) / 2.0 * (uL - s))
                    r = rL * (c / cL) ** (2.0 / (g - 1.0))
                    q = pL * (c / cL) ** (2.0 * g / (g - 1.0))
        else:  # right of the contact
            if ps > pR:  # right shock
                SR = uR + cR * np.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
                if s >= SR:
                    r, v, q = rR, uR, pR
                else:
                    r, v, q = rR * (ps / pR + gm) / (gm * ps / pR + 1.0), us, ps
            else:  # right rarefaction
                csR = cR * (ps / pR) ** ((g - 1.0) / (2.0 * g))
                if s >= uR + cR:
                    r, v, q = rR, uR, pR
                elif s <= us + csR:
                    r, v, q = rR * (ps / pR) ** (1.0 / g), us, ps
                else:
                    v = 2.0 / (g + 1.0) * (-cR + (g - 1.0) / 2.0 * uR + s)
                    c = 2.0 / (g + 1.0) * (cR - (g - 1.0) / 2.0 * (uR - s))
                    r = rR * (c / cR) ** (2.0 / (g - 1.0))
                    q = pR * (c / cR) ** (2.0 * g / (g - 1.0))
        rho[idx], u[idx], p[idx] = r, v, q
    return rho, u, p


def riemann_max_speed(left, right, gamma: float = 1.4) -> float:
    """Fastest wave speed |S| of the exact Riemann solution (shock or rarefaction head)."""
    rL, uL, pL = left
    rR, uR, pR = right
    g = gamma
    ps, us = riemann_star(left, right, g)
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    if ps > pL:
        sl = uL - cL * np.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
    else:
        sl = uL - cL
    if ps > pR:
        sr = uR + cR * np.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
    else:
        sr = uR + cR
    return float(max(abs(sl), abs(sr)))


def euler_riemann_avg(edges: np.ndarray, x0: float, t: float, left, right, gamma: float = 1.4, sub: int = 64):
    """Cell averages of the conserved variables (rho, rho u, E) of the exact solution."""
    a, b = edges[:-1], edges[1:]
    frac = (np.arange(sub) + 0.5) / sub
    x = a[:, None] + (b - a)[:, None] * frac[None, :]
    rho, u, p = riemann_sample((x - x0) / t, left, right, gamma)
    E = p / (gamma - 1.0) + 0.5 * rho * u * u
    return np.stack([rho.mean(axis=1), (rho * u).mean(axis=1), E.mean(axis=1)])


def prim_to_cons(rho, u, p, gamma: float = 1.4):
    rho, u, p = (np.asarray(v, dtype=np.float64) for v in (rho, u, p))
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])
