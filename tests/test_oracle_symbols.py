"""Pins for oracle.symbols: the closed-form symbols (Eq. 16 reading) against
the sampled-kernel DFT of Eq. 13 built from oracle.kernels, and the FFT path
against the direct circular sum of Eq. 13."""
import numpy as np
import pytest

from oracle import fc, ops, symbols
from tables import gram_golden


@pytest.mark.parametrize("family", ["G2", "G4", "G6", "G8", "G10"])
@pytest.mark.parametrize("op", ["W", "DX", "DY", "LAP"])
def test_closed_form_equals_sampled_kernel_dft(family, op):
    # With h = 5 dx on a 96 x 80 periodic grid, the Nyquist image (s = 25 pi^2/4)
    # and the minimum-image truncation (half period = 8 h, e^{-64}) are below
    # rounding even for G10, so Eq. 13 and the continuous transform must agree.
    m0, m1 = 96, 80
    dx, dy = 1.0 / 96, 1.0 / 96
    h = 5.0 * dx
    S13 = symbols.symbol(op, family, h, m0, m1, dx, dy)
    S16 = symbols.symbol_closed(op, family, h, m0, m1, dx, dy)
    scale = np.abs(S16).max()
    assert np.abs(S13 - S16).max() < 1e-11 * scale


def test_brute_force_circular_sum_equals_fft_path():
    # Eq. 13 written out as a direct sum over the FC-extended grid.
    rng = np.random.default_rng(5)
    nx, ny = 6, 7
    dx, dy = 1.0 / 6, 1.0 / 6
    f = rng.standard_normal((nx, ny))
    E = gram_golden(5, 25)
    m0, m1 = nx, ny + 25
    h = 1.3 * dx
    for op in ("DX", "DY", "LAP"):
        w = symbols.sampled_kernel(op, "G4", h, m0, m1, dx, dy)
        S = symbols.symbol(op, "G4", h, m0, m1, dx, dy)
        fast = ops.apply_symbols(f, [S], E)[0]
        slow = ops.circular_sum(f, w, dx, dy, E)
        assert np.abs(fast - slow).max() < 1e-12 * np.abs(slow).max()


def test_half_period_sample_is_average_of_images():
    m = 8
    d = 0.1
    h = 0.2
    w = symbols.sampled_kernel("DX", "G4", h, m, 5, d, d)
    assert np.all(w[m // 2, :] == 0.0)
    wW = symbols.sampled_kernel("W", "G4", h, m, 5, d, d)
    from oracle import kernels
    assert abs(wW[m // 2, 0] - kernels.W("G4", h, np.float64(m // 2 * d), np.float64(0.0))) < 1e-15


def test_kernel_transform_g4_closed_form():
    # For G4 = (2 - q^2) e^{-q^2}/(pi h^2) the transform is (1 + s) e^{-s}, s = |k|^2 h^2/4.
    s = np.linspace(0, 10, 11)
    np.testing.assert_allclose(symbols.kernel_transform("G4", s), (1 + s) * np.exp(-s), rtol=1e-15, atol=0)
