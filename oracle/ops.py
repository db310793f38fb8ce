"""Spectral SPH operators on the FC-extended grid (Eqs. 11, 13, 30).

    F = FC-extend(f)                       (Eq. 30; tensor product if x has walls)
    out = IDFT2( DFT2(F) . S )[:nx, :ny]   (Eqs. 11/13; S from symbols.py)

The physical nodes are the first nx x ny of the extended grid.
"""
import numpy as np

from .dft import dft2, idft2
from .fc import extend2d


def apply_symbols(f, symbols, E_y, E_x=None):
    """One forward transform of the extended field, one inverse per symbol."""
    nx, ny = f.shape
    F = extend2d(np.asarray(f, dtype=np.float64), E_y, E_x)
    Fh = dft2(F)
    outs = []
    for S in symbols:
        g = idft2(Fh * S)
        outs.append(np.real(g[:nx, :ny]).copy())
    return outs


def divergence(fx, fy, Sx, Sy, E_y, E_x=None):
    """div = IDFT(Sx DFT(Fx) + Sy DFT(Fy)) on the physical nodes."""
    nx, ny = fx.shape
    Fx = dft2(extend2d(np.asarray(fx, dtype=np.float64), E_y, E_x))
    Fy = dft2(extend2d(np.asarray(fy, dtype=np.float64), E_y, E_x))
    return np.real(idft2(Sx * Fx + Sy * Fy)[:nx, :ny]).copy()


def circular_sum(f, w_sampled, dx, dy, E_y, E_x=None):
    """Eq. 13 written out as the direct circular sum (brute force, tiny grids).

    out_i = sum_j F_j w((i - j) mod m) dx dy, restricted to physical i."""
    nx, ny = f.shape
    F = extend2d(np.asarray(f, dtype=np.float64), E_y, E_x)
    m0, m1 = F.shape
    out = np.zeros((nx, ny))
    for i0 in range(nx):
        for i1 in range(ny):
            acc = 0.0
            for j0 in range(m0):
                for j1 in range(m1):
                    acc += F[j0, j1] * w_sampled[(i0 - j0) % m0, (i1 - j1) % m1]
            out[i0, i1] = acc * dx * dy
    return out
