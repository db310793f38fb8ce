"""High-order Gaussian SPH kernels (Sec. 3.3 and Appendix A).

A kernel of order 2n is  W_2n(q) = alpha * sum_{m<n} A_m q^(2m) exp(-q^2),
q = r/h, with the A_m fixed by removing the even moments (Appendix A):
    sum_m A_m I_{m+j} = delta_{j0},  j = 0..n-1,
where I_k is the k-th moment of the base Gaussian.  In 2D, I_k = k! and
alpha = 1/(pi h^2) (Appendix A).  In 3D, I_k = Gamma(k+3/2)/Gamma(3/2) and
alpha = 1/(pi^(3/2) h^3) (same recipe, 3D moments).

Only derivatives of the radial form are needed: with s = q^2 = |x|^2/h^2 and
P(s) = sum_m A_m s^m,
    W        = alpha P(s) e^{-s}
    dW/dx_a  = alpha (P'(s) - P(s)) e^{-s} * 2 x_a / h^2
    lap W    = alpha e^{-s} (4/h^2) [ s (P'' - 2P' + P) + (dim/2) (P' - P) ]
"""
import math
from fractions import Fraction

import numpy as np

FAMILIES = {"G2": 1, "G4": 2, "G6": 3, "G8": 4, "G10": 5}


def moments(k, dim=2):
    """k-th moment I_k of alpha*exp(-q^2): int q^(2k) alpha e^{-q^2} dV (Appendix A).

    2D: k!;  3D: Gamma(k+3/2)/Gamma(3/2) = (3/2)(5/2)...((2k+1)/2).  Exact rationals."""
    if dim == 2:
        return Fraction(math.factorial(k))
    if dim == 3:
        r = Fraction(1)
        for i in range(1, k + 1):
            r *= Fraction(2 * i + 1, 2)
        return r
    raise ValueError(dim)


def coefficients(family, dim=2):
    """A_0..A_{n-1} from the moment system of Appendix A, solved exactly
    (Gauss-Jordan elimination in rationals), then rounded to FP64."""
    n = FAMILIES[family]
    M = [[moments(m + j, dim) for m in range(n)] + [Fraction(1 if j == 0 else 0)] for j in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        M[c] = [x / M[c][c] for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return np.array([float(M[j][n]) for j in range(n)])


def alpha(h, dim=2):
    """Normalisation constant of the base Gaussian (Appendix A: 1/(pi h^2) in 2D)."""
    if dim == 2:
        return 1.0 / (math.pi * h * h)
    return 1.0 / (math.pi ** 1.5 * h ** 3)


def _poly(A, s):
    P = np.zeros_like(s)
    dP = np.zeros_like(s)
    d2P = np.zeros_like(s)
    for m, a in enumerate(A):
        P += a * s ** m
        if m >= 1:
            dP += a * m * s ** (m - 1)
        if m >= 2:
            d2P += a * m * (m - 1) * s ** (m - 2)
    return P, dP, d2P


def W(family, h, x, y):
    """Kernel value at offset (x, y) (2D)."""
    A = coefficients(family, 2)
    s = (x * x + y * y) / (h * h)
    P, _, _ = _poly(A, s)
    return alpha(h, 2) * P * np.exp(-s)


def dW(family, h, x, y, axis):
    """Partial derivative of W with respect to x (axis=0) or y (axis=1)."""
    A = coefficients(family, 2)
    s = (x * x + y * y) / (h * h)
    P, dP, _ = _poly(A, s)
    xa = x if axis == 0 else y
    return alpha(h, 2) * (dP - P) * np.exp(-s) * 2.0 * xa / (h * h)


def lapW(family, h, x, y):
    """Laplacian of W (2D)."""
    A = coefficients(family, 2)
    s = (x * x + y * y) / (h * h)
    P, dP, d2P = _poly(A, s)
    return alpha(h, 2) * np.exp(-s) * (4.0 / (h * h)) * (s * (d2P - 2 * dP + P) + (dP - P))
