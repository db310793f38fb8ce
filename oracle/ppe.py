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

from .dft import dct1_matrix, dft2, dft_matrix, idct1_matrix, idft2, idft_matrix, signed_wavenumbers
from .fc import extend2d


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


def extended_projection(us, vs, Sx, Sy, E_y, E_x=None, return_extended=False):
    """The projection on the FC-extended periodic grid (the alternative to the
    physical-domain solve that Sec. 5.2 names and leaves for future work).

    With the gradient symbols G = (Sx, Sy) of the operators (Eq. 13/16; they
    are i k W_hat with the odd symbols zero on their Nyquist lines), the
    pressure is the Fourier multiplier solve of div(grad phi) = div(u*) on the
    extended grid, and the corrected spectrum is

        phi_hat = (Sx U + Sy V) / (Sx^2 + Sy^2),   (U, V) <- (U, V) - (Sx, Sy) phi_hat

    (modes where Sx^2 + Sy^2 = 0 are left as they are; their divergence is
    zero).  The extended divergence Sx U + Sy V of the result is zero at every
    mode.  Returns the corrected fields on the physical nodes (and the
    corrected extended fields when return_extended)."""
    nx, ny = us.shape
    U = dft2(extend2d(np.asarray(us, dtype=np.float64), E_y, E_x))
    V = dft2(extend2d(np.asarray(vs, dtype=np.float64), E_y, E_x))
    GG = Sx * Sx + Sy * Sy
    nz = np.abs(GG) > 0
    phi = np.zeros_like(U)
    phi[nz] = (Sx[nz] * U[nz] + Sy[nz] * V[nz]) / GG[nz]
    Un = U - Sx * phi
    Vn = V - Sy * phi
    ue, ve = np.real(idft2(Un)), np.real(idft2(Vn))
    out = (ue[:nx, :ny].copy(), ve[:nx, :ny].copy())
    if return_extended:
        return out + (ue, ve)
    return out
