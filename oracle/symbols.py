"""Fourier symbols of the SPH kernel derivatives on the extended grid (Eq. 13, Fig. 1).

The circular convolution of Eq. 13 evaluates the kernel at the minimum-image
separation and weights each particle by its volume dx*dy.  On an extended
grid of m0 x m1 nodes with spacings (dx, dy), the kernel array is sampled at
the signed offsets a*dx, b*dy with a in (-m0/2, m0/2], wrapped to the corners
(Fig. 1b).  Its 2D DFT times dx*dy is the operator's symbol:

    (f (*) w)_i = IDFT( DFT(f) . dx dy DFT(w) )_i.

At exactly half a period (even m) the two images +L/2 and -L/2 are equally
near; the sample there is the average of both, so odd derivatives vanish and
even ones keep their value.
"""
import numpy as np

from . import kernels
from .dft import dft2

OPS = ("W", "DX", "DY", "LAP")


def _offsets(m):
    """Signed offsets of an m-point periodic axis: (plus-image, minus-image).

    They differ only at the half-period index a = m/2 (even m), where the
    first gives +m/2 and the second -m/2."""
    a = np.arange(m)
    plus = np.where(2 * a <= m, a, a - m)
    minus = np.where(2 * a < m, a, a - m)
    return plus.astype(np.float64), minus.astype(np.float64)


def _eval(op, family, h, x, y):
    if op == "W":
        return kernels.W(family, h, x, y)
    if op == "DX":
        return kernels.dW(family, h, x, y, 0)
    if op == "DY":
        return kernels.dW(family, h, x, y, 1)
    if op == "LAP":
        return kernels.lapW(family, h, x, y)
    raise ValueError(op)


def sampled_kernel(op, family, h, m0, m1, dx, dy):
    """w[a, b] = op(W) at the minimum-image offset (a dx, b dy), Eq. 13.

    Averaged pairwise over the images so that every sample which has a single
    nearest image keeps its value exactly ((v + v) / 2 == v)."""
    xp, xm = _offsets(m0)
    yp, ym = _offsets(m1)
    X1, Y1 = np.meshgrid(xp * dx, yp * dy, indexing="ij")
    X2, Y2 = np.meshgrid(xm * dx, ym * dy, indexing="ij")
    a = (_eval(op, family, h, X1, Y1) + _eval(op, family, h, X2, Y1)) * 0.5
    b = (_eval(op, family, h, X1, Y2) + _eval(op, family, h, X2, Y2)) * 0.5
    return (a + b) * 0.5


def symbol(op, family, h, m0, m1, dx, dy):
    """dx*dy*DFT2 of the sampled kernel derivative (complex m0 x m1 array)."""
    return dx * dy * dft2(sampled_kernel(op, family, h, m0, m1, dx, dy))


def kernel_transform(family, s):
    """Continuous 2D Fourier transform of the Gaussian kernel family at s = |k|^2 h^2 / 4.

    For W_2n = alpha sum_{m<n} A_m q^(2m) e^{-q^2} with the Appendix A moment
    conditions, the transform is e^{-s} sum_{m<n} s^m / m! (the first n terms
    of the Taylor series of e^{s}, times e^{-s})."""
    n = kernels.FAMILIES[family]
    acc = np.zeros_like(s)
    term = np.ones_like(s)
    for m in range(n):
        if m > 0:
            term = term * s / m
        acc = acc + term
    return np.exp(-s) * acc


def wavenumbers(m, d):
    """Angular wavenumbers 2 pi kappa / (m d) of an m-point periodic axis (signed kappa)."""
    a = np.arange(m)
    kappa = np.where(2 * a <= m, a, a - m)
    return 2.0 * np.pi * kappa / (m * d)


def symbol_closed(op, family, h, m0, m1, dx, dy):
    """Eq. 16 form of the symbols on an m0 x m1 extended grid:
    W -> W_hat(k), DX -> i kx W_hat, DY -> i ky W_hat, LAP -> -|k|^2 W_hat.

    The first-derivative symbol is zero on the Nyquist line of its own axis
    (even m), where i k has no real-valued counterpart."""
    kx = wavenumbers(m0, dx)
    ky = wavenumbers(m1, dy)
    KX, KY = np.meshgrid(kx, ky, indexing="ij")
    Wh = kernel_transform(family, (KX * KX + KY * KY) * (h * h) / 4.0)
    if op == "W":
        return Wh.astype(np.complex128)
    if op == "DX":
        kxo = kx.copy()
        if m0 % 2 == 0:
            kxo[m0 // 2] = 0.0
        return 1j * kxo[:, None] * Wh
    if op == "DY":
        kyo = ky.copy()
        if m1 % 2 == 0:
            kyo[m1 // 2] = 0.0
        return 1j * kyo[None, :] * Wh
    if op == "LAP":
        return (-(KX * KX + KY * KY) * Wh).astype(np.complex128)
    raise ValueError(op)
