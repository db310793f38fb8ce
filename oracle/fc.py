"""Fourier continuation (FC) tables and extension (Sec. 4).

Every FC variant here is one linear map per line.  With the n_match values
nearest each wall collected as

    b = [f_{N-n_match}, ..., f_{N-1},  f_0, ..., f_{n_match-1}]

(right wall block first, then the left wall block), the n_cont continuation
values appended after f_{N-1} are  E @ b,  E of shape (n_cont, 2*n_match).
The extended line F = [f_0..f_{N-1}, E@b] is periodic with period
(N + n_cont) * dy: the node after the last continuation node is f_0 again.

Two constructions of E:

``paper_table``  -- the paper's own FC (Sec. 4.1-4.4): least-squares fit of a
    degree-p polynomial to the n_match points nearest each wall in wall-local
    coordinates (Eqs. 14-20), extrapolation of the right fit forward and the
    left fit backward into the gap (Eqs. 21-23), quintic blending (Eqs. 24-26),
    and for Neumann data one extra least-squares row forcing the linear
    coefficient to zero (Eqs. 27-29).  Coordinates are in units of dy, which
    leaves the fitted values unchanged and keeps the Vandermonde well scaled.

``gram_table``   -- FC(Gram), which Sec. 4.5 names (Albin & Bruno) without
    giving a construction.  Built here from its mathematical definition: the
    right-wall data are represented by their degree-(n_match-1) polynomial
    (the projection onto the Gram basis of the n_match matching nodes, which
    with n_match basis functions is the interpolant), and each such polynomial
    is continued by a "blend-to-zero" trigonometric polynomial fitted in the
    least-squares sense to (i) the polynomial on the matching interval and
    (ii) zero on the interval where the left-wall data sit in the periodic
    extension.  The left wall is the mirror image.  The trig fit is
    ill-conditioned, so it is solved in 80-digit arithmetic (mpmath) and
    rounded to FP64 once.

    Parameters (unit = dy; matching nodes u = 0..d-1 with the wall at u = d-1,
    continuation nodes u = d..d+C-1, left-wall block u = d+C..2d+C-1):
        period T = 2 (2d + C - 2), K = floor(T/4) cosine+sine modes,
        20 fit points per unit interval on both fit intervals.
"""
import numpy as np

DIRICHLET = 0
NEUMANN = 1

GRAM_OVERSAMPLE = 20


def blend_sigma(t):
    """Quintic blending function of Eq. 25: sigma(t) = 10t^3 - 15t^4 + 6t^5."""
    return 10.0 * t ** 3 - 15.0 * t ** 4 + 6.0 * t ** 5


def _vandermonde(xi, p):
    """Eq. 19: rows [xi^p, xi^(p-1), ..., xi, 1]."""
    return np.stack([xi ** (p - m) for m in range(p + 1)], axis=1)


def _ls_operator(xi, p, bc):
    """Linear map from the n_match wall values to the polynomial coefficients.

    Least squares via QR (Eq. 20).  For Neumann data the row [0 .. 0 1 0]
    with right-hand side 0 is appended (Eq. 28), which pins the coefficient of
    xi^1 (the wall derivative, Eq. 27) towards zero."""
    V = _vandermonde(xi, p)
    n = len(xi)
    if bc == NEUMANN:
        row = np.zeros((1, p + 1))
        row[0, p - 1] = 1.0
        V = np.vstack([V, row])
    Q, R = np.linalg.qr(V)
    # c = R^{-1} Q^T [f; 0]  ->  only the first n columns of Q^T act on f
    return np.linalg.solve(R, Q.T[:, :n])


def paper_table(n_match, n_cont, p, bc=DIRICHLET):
    """E for the paper's polynomial FC (Sec. 4.1-4.4, Eqs. 14-29).

    Continuation node j = 1..n_cont lies j*dy past the last wall node.  The
    right fit is evaluated at xi = j (Eq. 22); the left fit at
    xi = -(n_cont + 1 - j) (Eq. 23 with n_cont + 1 distinct gap intervals,
    so the node after the gap is f_0 itself); t_j = (j-1)/(n_cont-1) (Eq. 24).
    """
    if not (n_match > p):
        raise ValueError("need n_match > p")
    if n_cont < 2:
        raise ValueError("need n_cont >= 2")
    xi_r = np.arange(-(n_match - 1), 1, dtype=np.float64)   # right wall at xi = 0 (Eq. 14)
    xi_l = np.arange(0, n_match, dtype=np.float64)          # left wall at xi = 0
    Cr = _ls_operator(xi_r, p, bc)
    Cl = _ls_operator(xi_l, p, bc)
    j = np.arange(1, n_cont + 1, dtype=np.float64)
    t = (j - 1.0) / (n_cont - 1.0)
    s = blend_sigma(t)
    Vr = _vandermonde(j, p)                         # p_r(j dy), Eq. 22
    Vl = _vandermonde(-(n_cont + 1.0 - j), p)       # p_l(-(n_cont+1-j) dy), Eq. 23
    Er = (1.0 - s)[:, None] * (Vr @ Cr)
    El = s[:, None] * (Vl @ Cl)
    return np.hstack([Er, El])


def gram_params(n_match, n_cont):
    T = 2 * (2 * n_match + n_cont - 2)
    K = T // 4
    return T, K


def gram_table(n_match, n_cont, bc=DIRICHLET, dps=80, modes=None, ridge=0.0):
    """E for FC(Gram) (Sec. 4.5), construction in the module docstring.

    bc is accepted for interface symmetry; the Gram continuation treats
    Dirichlet and Neumann data alike (the Neumann condition is carried by the
    data themselves).

    modes, ridge: alternatives kept only to measure the conditioning/accuracy
    trade-off of the construction (the tables in use take the defaults):
    `modes` trig modes instead of floor(T/4), and a ridge (Tikhonov) term
    ridge^2 * max_i (A^T A)_ii * I added to the normal equations."""
    import mpmath as mp

    d, C = n_match, n_cont
    T, K = gram_params(d, C)
    if modes is not None:
        K = modes
    with mp.workdps(dps):
        ovs = GRAM_OVERSAMPLE
        u_match = [mp.mpf(i) / ovs for i in range((d - 1) * ovs + 1)]
        u_zero = [mp.mpf(d + C) + mp.mpf(i) / ovs for i in range((d - 1) * ovs + 1)]

        def trig_row(u):
            row = [mp.mpf(1)]
            for k in range(1, K + 1):
                a = 2 * mp.pi * k * u / T
                row.append(mp.cos(a))
                row.append(mp.sin(a))
            return row

        A = mp.matrix([trig_row(u) for u in u_match] + [trig_row(u) for u in u_zero])
        # Target: the degree-(d-1) polynomial through the d matching values,
        # as a linear map of those values (Lagrange basis), zero on u_zero.
        nrow = len(u_match) + len(u_zero)
        rhs = mp.matrix(nrow, d)
        for i, u in enumerate(u_match):
            for a in range(d):
                v = mp.mpf(1)
                for b in range(d):
                    if a != b:
                        v *= (u - b) / mp.mpf(a - b)
                rhs[i, a] = v
        # Least squares by the normal equations, exact enough at this precision.
        AtA = A.T * A
        Atb = A.T * rhs
        if ridge:
            scale = max(AtA[i, i] for i in range(AtA.rows))
            AtA = AtA + (mp.mpf(ridge) ** 2 * scale) * mp.eye(AtA.rows)
        B = mp.matrix([trig_row(mp.mpf(u)) for u in range(d, d + C)])
        Er = np.zeros((C, d))
        for a in range(d):
            coef = mp.lu_solve(AtA, Atb.column(a))
            vals = B * coef
            for c in range(C):
                Er[c, a] = float(vals[c])
    El = Er[::-1, ::-1]
    return np.hstack([Er, El]).copy()


def fc_table(variant, n_match, n_cont, bc=DIRICHLET, p=None):
    if variant == "gram":
        return gram_table(n_match, n_cont, bc)
    if variant == "paper":
        if p is None:
            p = min(5, n_match - 2)
        return paper_table(n_match, n_cont, p, bc)
    raise ValueError(variant)


def extend_last_axis(f, E):
    """Append the FC continuation E @ b along the last axis (Eq. 30).

    The table entries reach ~1e4 while E @ b is O(|b|), so the products are
    accumulated in extended precision (np.longdouble) and rounded once."""
    n_cont, two_m = E.shape
    m = two_m // 2
    b = np.concatenate([f[..., -m:], f[..., :m]], axis=-1)
    cont = (b.astype(np.longdouble) @ E.T.astype(np.longdouble)).astype(np.float64)
    return np.concatenate([f, cont], axis=-1)


def extend2d(f, E_y, E_x=None):
    """FC-extend a 2D field f[x, y]: y (walls) first, then x if it has walls.

    Sec. 4.6 extends y only (x periodic).  With walls on x as well the paper
    gives no construction; the tensor product is used (y then x), which
    commutes with the x-then-y order in exact arithmetic."""
    F = extend_last_axis(f, E_y) if E_y is not None else f
    if E_x is not None:
        F = extend_last_axis(F.T, E_x).T
    return F
