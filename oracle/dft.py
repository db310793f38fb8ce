"""Naive O(N^2) transforms written as their defining sums (Eqs. 11, 31, 32).

No FFT: each transform is the explicit matrix of its definition, applied with
a plain matrix product.
"""
import numpy as np


def dft_matrix(n):
    """F[k, m] = exp(-2 pi i k m / n): forward DFT, X = F @ x (Eq. 11 kernel)."""
    k = np.arange(n)
    # (k*m) mod n keeps the phase argument exact before scaling
    return np.exp(-2j * np.pi * ((np.outer(k, k) % n) / n))


def idft_matrix(n):
    """Inverse DFT with the 1/n factor of Eq. 11: x = G @ X."""
    k = np.arange(n)
    return np.exp(2j * np.pi * ((np.outer(k, k) % n) / n)) / n


def dct1_matrix(n):
    """DCT-I of Eq. 31 in 1D: X_k = x_0 + (-1)^k x_{n-1} + 2 sum_{j=1}^{n-2} x_j cos(pi j k/(n-1))."""
    k = np.arange(n)
    C = np.cos(np.pi * ((np.outer(k, k) % (2 * (n - 1))) / (n - 1)))
    w = np.full(n, 2.0)
    w[0] = 1.0
    w[-1] = 1.0
    return C * w[None, :]


def idct1_matrix(n):
    """Inverse of the DCT-I above: the same matrix divided by 2(n-1)."""
    return dct1_matrix(n) / (2.0 * (n - 1))


def dft2(F):
    """2D DFT of an (n0, n1) array."""
    return dft_matrix(F.shape[0]) @ F @ dft_matrix(F.shape[1]).T


def idft2(G):
    """Inverse 2D DFT (with 1/(n0 n1))."""
    return idft_matrix(G.shape[0]) @ G @ idft_matrix(G.shape[1]).T


def signed_wavenumbers(n):
    """Integer wavenumbers k for DFT index 0..n-1 (k for k <= n/2, k-n above).

    For even n the Nyquist index n/2 is kept positive."""
    k = np.arange(n)
    return np.where(k <= n // 2, k, k - n)
