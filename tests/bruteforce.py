"""Exact-arithmetic (fractions) restatement of the reconstruction from its definitions,
for tiny grids.  Used only to pin the oracle.

Every quantity is built from the definitions of Sec. 2 of the paper rather than from the
printed tables:
  * polynomial candidates: derivative at the face of the polynomial interpolant of the
    primitive V(x) (Lagrange form, exact rationals);
  * linear WENO weights d_r: the unique combination of the three 3-cell candidates equal
    to the 5-cell candidate;
  * smoothness indicators: beta_r = sum_l dx^(2l-1) int_cell (d^l p_r/dx^l)^2 dx evaluated
    by exact polynomial integration;
  * ENO choice: Newton divided differences of V (the smaller in magnitude wins; a tie
    goes right);
  * monotone switch: roots of p' located exactly (high-precision square root);
  * perturbation rows q_rj: derived from the flat limit of the pure RBF interpolant of the
    primitive (multiquadric / Gaussian) with mpmath, then rationalised.
Cells are unit intervals: cell j = [j, j+1], so the face between cell j-1 and j is x = j.
"""
from __future__ import annotations

from fractions import Fraction as F

# ---------------------------------------------------------------------------------------
# polynomials as coefficient lists (lowest degree first), exact rationals
# ---------------------------------------------------------------------------------------


def pmul(a, b):
    out = [F(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def pscale(a, s):
    return [x * s for x in a]


def pder(a):
    return [a[i] * i for i in range(1, len(a))] or [F(0)]


def pint(a, lo, hi):
    s = F(0)
    for i, x in enumerate(a):
        s += x * (F(hi) ** (i + 1) - F(lo) ** (i + 1)) / (i + 1)
    return s


def peval(a, x):
    s = F(0)
    for c in reversed(a):
        s = s * x + c
    return s


def interp(xs, ys):
    """Lagrange interpolating polynomial through (xs, ys), as coefficients."""
    out = [F(0)]
    for k, (xk, yk) in enumerate(zip(xs, ys)):
        basis = [F(1)]
        den = F(1)
        for j, xj in enumerate(xs):
            if j != k:
                basis = pmul(basis, [F(-xj), F(1)])
                den *= (xk - xj)
        out = padd(out, pscale(basis, F(yk) / den))
    return out


def cell_poly(v, first, ncell):
    """p = V' for the polynomial interpolant of the primitive through the interfaces of
    cells first..first+ncell-1 (v indexed by absolute cell number)."""
    xs = [F(first + k) for k in range(ncell + 1)]
    ys = [F(0)]
    for k in range(ncell):
        ys.append(ys[-1] + F(v[first + k]))
    return pder(interp(xs, ys))


# ---------------------------------------------------------------------------------------
# derived tables
# ---------------------------------------------------------------------------------------


def poly_row(r, side):
    """Coefficients of the 3-cell candidate of cell 0 with r cells to its left, at its
    right face (side 0, x = 1) or left face (side 1, x = 0)."""
    out = []
    for j in range(3):
        v = {c: F(0) for c in range(-r, -r + 3)}
        v[-r + j] = F(1)
        p = cell_poly(v, -r, 3)
        out.append(peval(p, F(1) if side == 0 else F(0)))
    return out


def linear_weights(side):
    """d_r with sum_r d_r * candidate_r == 5-cell candidate for all data."""
    rows = [poly_row(r, side) for r in range(3)]
    five = []
    for j in range(5):
        v = {c: F(0) for c in range(-2, 3)}
        v[-2 + j] = F(1)
        five.append(peval(cell_poly(v, -2, 5), F(1) if side == 0 else F(0)))
    # coefficient of cell c (c = -2..2) in candidate r is rows[r][c + r] when 0 <= c+r < 3
    # cell -2 appears only in r = 2, cell 2 only in r = 0: solve directly, verify the rest
    d2 = five[0] / rows[2][0]
    d0 = five[4] / rows[0][2]
    # cell -1: r = 2 (j=1) and r = 1 (j=0)
    d1 = (five[1] - d2 * rows[2][1]) / rows[1][0]
    d = [d0, d1, d2]
    for c in range(-2, 3):
        s = sum(d[r] * rows[r][c + r] for r in range(3) if 0 <= c + r < 3)
        assert s == five[c + 2]
    return d


def beta(v, i, r):
    """Jiang-Shu indicator from its definition for cell i, stencil i-r..i-r+2 (dx = 1)."""
    p = cell_poly(v, i - r, 3)
    d1 = pder(p)
    d2 = pder(d1)
    return pint(pmul(d1, d1), i, i + 1) + pint(pmul(d2, d2), i, i + 1)


_Q_CACHE = {}


def rbf_rows(kind):
    """Perturbation rows q[r] (r = -1..2) from the flat limit of the pure RBF
    interpolant of the primitive anchored at the face (V(face) = 0)."""
    if kind in _Q_CACHE:
        return _Q_CACHE[kind]
    import mpmath as mp
    mp.mp.dps = 260

    def coeffs(r, eta):
        xs = [mp.mpf(-r - 1 + j) for j in range(4)]  # interfaces of cells -r..-r+2 (face at 0)

        def phi(dd):
            return mp.sqrt(1 + eta * dd * dd) if kind == "mq" else mp.exp(-eta * dd * dd)

        def dphi(dd):
            return eta * dd / mp.sqrt(1 + eta * dd * dd) if kind == "mq" else -2 * eta * dd * mp.exp(-eta * dd * dd)

        out = []
        for c in range(3):
            def V(x):
                s = mp.mpf(0)
                a, b = -r - 1 + c, -r + c
                lo, hi = (0, x) if x >= 0 else (x, 0)
                ov = max(0, min(b, hi) - max(a, lo))
                return ov * (1 if x >= 0 else -1)
            A = mp.matrix(4, 4)
            for a in range(4):
                for b in range(4):
                    A[a, b] = phi(xs[a] - xs[b])
            lam = mp.lu_solve(A, mp.matrix([V(x) for x in xs]))
            out.append(sum(lam[j] * dphi(0 - xs[j]) for j in range(4)))
        return out

    h = mp.mpf("1e-40")
    rows = {}
    for r in (-1, 0, 1, 2):
        c1, c2 = coeffs(r, h), coeffs(r, 2 * h)
        rows[r] = [F(str(mp.nstr((b - a) / h, 30))).limit_denominator(1000) for a, b in zip(c1, c2)]
    _Q_CACHE[kind] = rows
    return rows


# ---------------------------------------------------------------------------------------
# decisions
# ---------------------------------------------------------------------------------------


def divided_difference(xs, ys):
    if len(xs) == 1:
        return ys[0]
    return (divided_difference(xs[1:], ys[1:]) - divided_difference(xs[:-1], ys[:-1])) / (xs[-1] - xs[0])


def eno_r(v, i):
    """Newton divided-difference stencil choice for cell i (3 cells)."""
    def V(x):  # primitive anchored at x = i - 2
        return sum((F(v[c]) for c in range(i - 2, x)), F(0))
    lo, hi = i, i + 1  # interfaces of cell i
    for _ in range(2):
        left = [lo - 1] + list(range(lo, hi + 1))
        right = list(range(lo, hi + 1)) + [hi + 1]
        dl = abs(divided_difference([F(x) for x in left], [V(x) for x in left]))
        dr = abs(divided_difference([F(x) for x in right], [V(x) for x in right]))
        if dl < dr:
            lo -= 1
        else:
            hi += 1
    return i - lo


def switch_fires(w4):
    """True when the cubic with averages w4 over cells [-2,-1],[-1,0],[0,1],[1,2] is
    non-monotone on (-2, 2): p' has a root strictly inside (roots located exactly)."""
    import mpmath as mp
    v = {c: F(w4[c + 2]) for c in range(-2, 2)}
    p = cell_poly(v, -2, 4)
    dp = pder(p) + [F(0)] * 3
    c, b, a = dp[0], dp[1], dp[2]
    if a == 0:
        if b == 0:
            return False
        root = -c / b
        return -2 < root < 2
    disc = b * b - 4 * a * c
    if disc <= 0:
        return False
    mp.mp.dps = 80
    sq = mp.sqrt(mp.mpf(disc.numerator) / disc.denominator)
    for sgn in (-1, 1):
        root = (mp.mpf(-b.numerator) / b.denominator + sgn * sq) / (2 * mp.mpf(a.numerator) / a.denominator)
        if -2 < root < 2:
            return True
    return False


# ---------------------------------------------------------------------------------------
# the reconstruction on a periodic grid
# ---------------------------------------------------------------------------------------


def reconstruct_periodic(vals, scheme, rbf="mq", monotone_switch=False, eps_M=F(1, 10 ** 12),
                         eps_weno=F(1, 10 ** 6)):
    """(vm, vp) at faces f = 0..n (face f between cell f-1 and f) for scheme in
    'eno', 'weno_js', 'rbf_eno', 'rbf_weno'."""
    n = len(vals)
    v = {c: F(vals[c % n]) for c in range(-6, n + 6)}
    q = rbf_rows(rbf) if scheme.startswith("rbf") else None
    dm, dp_ = linear_weights(0), linear_weights(1)

    def face_eta(f):  # face f: cells f-2, f-1, f, f+1
        if q is None:
            return F(0)
        w = [v[f - 2], v[f - 1], v[f], v[f + 1]]
        if monotone_switch and switch_fires(w):
            return F(0)
        num = w[0] - 3 * w[1] + 3 * w[2] - w[3]
        den = w[0] - 15 * w[1] + 15 * w[2] - w[3] + eps_M
        return num / den

    def cand(i, r, side, eta):
        row = poly_row(r, side)
        s = F(0)
        for j in range(3):
            coef = row[j]
            if q is not None:
                coef += q[r - side][j] * eta
            s += coef * v[i - r + j]
        return s

    def value(i, side, eta):
        if scheme in ("eno", "rbf_eno"):
            return cand(i, eno_r(v, i), side, eta)
        d = dm if side == 0 else dp_
        al = [d[r] / (eps_weno + beta(v, i, r)) ** 2 for r in range(3)]
        tot = sum(al)
        return sum(al[r] / tot * cand(i, r, side, eta) for r in range(3))

    vm, vp = [], []
    for f in range(n + 1):
        eta = face_eta(f)
        vm.append(value(f - 1, 0, eta))
        vp.append(value(f, 1, eta))
    return vm, vp


# ---------------------------------------------------------------------------------------
# k = 2 (two-cell stencils), from the same definitions
# ---------------------------------------------------------------------------------------


def poly_row_k2(r, side):
    """Coefficients of the 2-cell candidate of cell 0 with r cells to its left (r = 0, 1), at
    its right face (side 0, x = 1) or left face (side 1, x = 0)."""
    out = []
    for j in range(2):
        v = {c: F(0) for c in range(-r, -r + 2)}
        v[-r + j] = F(1)
        out.append(peval(cell_poly(v, -r, 2), F(1) if side == 0 else F(0)))
    return out


def linear_weights_k2(side):
    """d_r (r = 0, 1) with d_0 * candidate_0 + d_1 * candidate_1 == 3-cell candidate."""
    rows = [poly_row_k2(r, side) for r in range(2)]
    three = []
    for j in range(3):
        v = {c: F(0) for c in range(-1, 2)}
        v[-1 + j] = F(1)
        three.append(peval(cell_poly(v, -1, 3), F(1) if side == 0 else F(0)))
    # cell 1 appears only in r = 0 (its j = 1), cell -1 only in r = 1 (its j = 0)
    d0 = three[2] / rows[0][1]
    d1 = three[0] / rows[1][0]
    assert d0 * rows[0][0] + d1 * rows[1][1] == three[1]
    return [d0, d1]


def beta_k2(v, i, r):
    """Indicator of the linear p on cells i-r, i-r+1 over cell i (dx = 1): int (p')^2."""
    d1 = pder(cell_poly(v, i - r, 2))
    return pint(pmul(d1, d1), i, i + 1)


def eno_r_k2(v, i):
    """One Newton divided-difference step from the interfaces of cell i."""
    def V(x):
        return sum((F(v[c]) for c in range(i - 2, x)), F(0))
    left = [i - 1, i, i + 1]
    right = [i, i + 1, i + 2]
    dl = abs(divided_difference([F(x) for x in left], [V(x) for x in left]))
    dr = abs(divided_difference([F(x) for x in right], [V(x) for x in right]))
    return 1 if dl < dr else 0


def switch_fires_k2(c3):
    """p = V' of the cubic primitive interpolant on cells [0,1], [1,2], [2,3] (averages c3):
    True when the vertex of the quadratic p lies strictly inside (0, 3)."""
    v = {c: F(c3[c]) for c in range(3)}
    p = cell_poly(v, 0, 3) + [F(0)] * 3
    b, a = p[1], p[2]
    if a == 0:
        return False
    xp = -b / (2 * a)
    return 0 < xp < 3


def eta_k2_from_derivation(c3, side, kind):
    """eps^2 dx^2 that cancels the dx^2 error term (Sec. 3.2 / 3.3): with v and v'' at the face
    taken from the cubic interpolant of the primitive through the four interfaces of cells
    i-1, i, i+1, the MQ condition is eta/2 v + v''/6 = 0 and the Gaussian one eta v + v''/6 = 0.
    side 0: face x_{i+1/2}; side 1: x_{i-1/2}.  Cells at [0,1], [1,2], [2,3]."""
    v = {c: F(c3[c]) for c in range(3)}
    p = cell_poly(v, 0, 3)
    x = F(2) if side == 0 else F(1)
    val = peval(p, x)
    dd = peval(pder(pder(p)), x)
    return -dd / (3 * val) if kind == "mq" else -dd / (6 * val)


_Q2_CACHE = {}


def rbf_rows_k2(kind):
    """k = 2 perturbation rows q[r] (r = -1, 0, 1) from the flat limit of the pure RBF
    interpolant of the primitive through the 3 interfaces of the 2-cell stencil."""
    if kind in _Q2_CACHE:
        return _Q2_CACHE[kind]
    import mpmath as mp
    mp.mp.dps = 260

    def coeffs(r, eta):
        xs = [mp.mpf(-r - 1 + j) for j in range(3)]

        def phi(dd):
            return mp.sqrt(1 + eta * dd * dd) if kind == "mq" else mp.exp(-eta * dd * dd)

        def dphi(dd):
            return eta * dd / mp.sqrt(1 + eta * dd * dd) if kind == "mq" else -2 * eta * dd * mp.exp(-eta * dd * dd)

        out = []
        for c in range(2):
            def V(x):
                a, b = -r - 1 + c, -r + c
                lo, hi = (0, x) if x >= 0 else (x, 0)
                ov = max(0, min(b, hi) - max(a, lo))
                return ov * (1 if x >= 0 else -1)
            A = mp.matrix(3, 3)
            for a in range(3):
                for b in range(3):
                    A[a, b] = phi(xs[a] - xs[b])
            lam = mp.lu_solve(A, mp.matrix([V(x) for x in xs]))
            out.append(sum(lam[j] * dphi(0 - xs[j]) for j in range(3)))
        return out

    h = mp.mpf("1e-40")
    rows = {}
    for r in (-1, 0, 1):
        c1, c2 = coeffs(r, h), coeffs(r, 2 * h)
        rows[r] = [F(str(mp.nstr((b - a) / h, 30))).limit_denominator(1000) for a, b in zip(c1, c2)]
    _Q2_CACHE[kind] = rows
    return rows


def reconstruct_periodic_k2(vals, scheme, rbf="mq", monotone_switch=False, eps_weno=F(1, 10 ** 6)):
    """(vm, vp) at faces f = 0..n for the k = 2 schemes.  The shape parameter of a cell comes
    from the derivation above (no eps_M), zero where the switch fires."""
    n = len(vals)
    v = {c: F(vals[c % n]) for c in range(-6, n + 6)}
    q = rbf_rows_k2(rbf) if scheme.startswith("rbf") else None
    dm, dp_ = linear_weights_k2(0), linear_weights_k2(1)

    def cell_eta(i, side):
        if q is None:
            return F(0)
        c3 = [v[i - 1], v[i], v[i + 1]]
        if monotone_switch and switch_fires_k2(c3):
            return F(0)
        return eta_k2_from_derivation(c3, side, rbf)

    def cand(i, r, side, eta):
        row = poly_row_k2(r, side)
        s = F(0)
        for j in range(2):
            coef = row[j]
            if q is not None:
                coef += q[r - side][j] * eta
            s += coef * v[i - r + j]
        return s

    def value(i, side):
        eta = cell_eta(i, side)
        if scheme in ("eno", "rbf_eno"):
            return cand(i, eno_r_k2(v, i), side, eta)
        d = dm if side == 0 else dp_
        al = [d[r] / (eps_weno + beta_k2(v, i, r)) ** 2 for r in range(2)]
        tot = sum(al)
        return sum(al[r] / tot * cand(i, r, side, eta) for r in range(2))

    vm = [value(f - 1, 0) for f in range(n + 1)]
    vp = [value(f, 1) for f in range(n + 1)]
    return vm, vp
