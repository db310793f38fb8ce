"""Pins for oracle.dft: the naive transform matrices against library routines."""
import numpy as np
import pytest
from scipy import fft as sfft

from oracle import dft


@pytest.mark.parametrize("n", [1, 2, 7, 16, 89, 153])
def test_dft_matrix_is_numpy_fft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    np.testing.assert_allclose(dft.dft_matrix(n) @ x, np.fft.fft(x), rtol=0, atol=1e-12 * max(1, n))
    np.testing.assert_allclose(dft.idft_matrix(n) @ np.fft.fft(x), x, rtol=0, atol=1e-13 * max(1, n))


@pytest.mark.parametrize("n", [2, 3, 9, 64, 65])
def test_dct1_matrix_is_scipy_dct1(n):
    # Eq. 31 in 1D is the unnormalised DCT-I.
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    np.testing.assert_allclose(dft.dct1_matrix(n) @ x, sfft.dct(x, type=1), rtol=0, atol=1e-12 * n)
    np.testing.assert_allclose(dft.idct1_matrix(n) @ (dft.dct1_matrix(n) @ x), x, rtol=0, atol=1e-13 * n)


def test_signed_wavenumbers():
    assert list(dft.signed_wavenumbers(6)) == [0, 1, 2, 3, -2, -1]
    assert list(dft.signed_wavenumbers(5)) == [0, 1, 2, -2, -1]
