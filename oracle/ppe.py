"""Spectral pressure Poisson solve on the physical nodes (Sec. 5.1, Eqs. 31-33).

x periodic (channel): DFT in x times DCT-I in y (Eq. 32).
walls on x too (cavity): DCT-I in both directions (Eq. 31).

The transforms diagonalise the Laplacian; with its eigenvalues
-(lam_k^2 + lam_l^2) the solve is the division of Eq. 33,

    phi_hat[k, l] = -b_hat[k, l] / (lam_k^2 + lam_l^2),   phi_hat[0, 0] = 0,

lam_k = 2 pi k / Lx for the DFT (signed k, Nyquist kept positive),
lam_k = pi k / Lx for DCT-I on a wall-to-wall length Lx = (nx-1) dx,
lam_l = pi l / Ly with Ly = (ny-1) dy.  The sign makes phi solve
lap(phi) = b.  The (0,0) mode is set to zero (Neumann solvability).
"""
import numpy as np

from .dft import dft_matrix, idft_matrix, dct1_matrix, idct1_matrix, signed_wavenumbers


def eigenvalues(nx, ny, Lx, Ly, x_walls):
    if x_walls:
        lam_k = np.pi * np.arange(nx) / Lx
    else:
        lam_k = 2.0 * np.pi * signed_wavenumbers(nx) / Lx
    lam_l = np.pi * np.arange(ny) / Ly
    return lam_k, lam_l


def ppe_solve(b, Lx, Ly, x_walls):
    """phi with lap(phi) = b under the spectral diagonalisation of Eqs. 31-33."""
    nx, ny = b.shape
    Ty = dct1_matrix(ny)
    Tyi = idct1_matrix(ny)
    if x_walls:
        Tx = dct1_matrix(nx)
        Txi = idct1_matrix(nx)
    else:
        Tx = dft_matrix(nx)
        Txi = idft_matrix(nx)
    bh = Tx @ np.asarray(b, dtype=np.float64) @ Ty.T
    lam_k, lam_l = eigenvalues(nx, ny, Lx, Ly, x_walls)
    den = lam_k[:, None] ** 2 + lam_l[None, :] ** 2
    den[0, 0] = 1.0
    ph = -bh / den
    ph[0, 0] = 0.0
    phi = Txi @ ph @ Tyi.T
    return np.real(phi).copy()


def laplacian(phi, Lx, Ly, x_walls):
    """The operator that ppe_solve inverts: transform, times -(lam^2), inverse."""
    nx, ny = phi.shape
    Ty = dct1_matrix(ny)
    Tyi = idct1_matrix(ny)
    if x_walls:
        Tx, Txi = dct1_matrix(nx), idct1_matrix(nx)
    else:
        Tx, Txi = dft_matrix(nx), idft_matrix(nx)
    lam_k, lam_l = eigenvalues(nx, ny, Lx, Ly, x_walls)
    ph = Tx @ np.asarray(phi, dtype=np.float64) @ Ty.T
    return np.real(Txi @ (-(lam_k[:, None] ** 2 + lam_l[None, :] ** 2) * ph) @ Tyi.T).copy()
