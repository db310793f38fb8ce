"""Pins for oracle.kernels (Sec. 3.3, Appendix A): printed coefficients,
moments by independent quadrature, derivatives by finite differences."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kernels
from tables import paper_constants


def test_g8_coefficients_are_the_printed_ones():
    # Appendix A prints A_0..A_3 = 4, -6, 2, -1/6 for G8.
    printed = paper_constants()["G8_coefficients"]
    np.testing.assert_array_equal(kernels.coefficients("G8"), printed)


def _moment_2d(A, j):
    # int_0^inf q^{2j} P(q^2) e^{-q^2} 2 pi q dq / pi   (h = 1, alpha = 1/pi)
    f = lambda q: q ** (2 * j) * sum(a * q ** (2 * m) for m, a in enumerate(A)) * math.exp(-q * q) * 2.0 * q
    return integrate.quad(f, 0, 40, limit=400, epsabs=1e-14, epsrel=1e-13)[0]


@pytest.mark.parametrize("family", ["G2", "G4", "G6", "G8", "G10"])
def test_even_moments_vanish_by_quadrature(family):
    # Appendix A: the kernel integrates to one and its even moments q^2..q^{2(n-1)} vanish.
    A = kernels.coefficients(family)
    n = kernels.FAMILIES[family]
    assert abs(_moment_2d(A, 0) - 1.0) < 1e-11
    for j in range(1, n):
        assert abs(_moment_2d(A, j)) < 1e-9 * math.factorial(2 * j)


def test_printed_g10_is_not_normalised():
    # Sec. 3.3 prints G10 = 5 - 10q^2 + 4q^4 - 2q^6/6 + q^8/24; its integral is 2, not 1,
    # so the oracle uses the moment recipe's G10 instead (5, -10, 5, -5/6, 1/24).
    printed = paper_constants()["G10_printed_coefficients"]
    assert abs(_moment_2d(printed, 0) - 2.0) < 1e-10
    np.testing.assert_allclose(kernels.coefficients("G10"), [5, -10, 5, -5 / 6, 1 / 24], atol=1e-12)


def test_alpha_2d():
    h = 0.37
    assert abs(kernels.alpha(h) * math.pi * h * h - paper_constants()["G8_alpha_2d_times_pi_h2"][0]) < 1e-15


@pytest.mark.parametrize("family", ["G4", "G8"])
def test_derivatives_match_finite_differences(family):
    h = 0.3
    rng = np.random.default_rng(0)
    pts = rng.uniform(-0.6, 0.6, (20, 2))
    e = 1e-5
    for x, y in pts:
        W = lambda a, b: kernels.W(family, h, np.float64(a), np.float64(b))
        dx = (W(x + e, y) - W(x - e, y)) / (2 * e)
        dy = (W(x, y + e) - W(x, y - e)) / (2 * e)
        lap = (W(x + e, y) + W(x - e, y) + W(x, y + e) + W(x, y - e) - 4 * W(x, y)) / (e * e)
        scale = kernels.alpha(h) / h
        assert abs(kernels.dW(family, h, x, y, 0) - dx) < 1e-6 * scale
        assert abs(kernels.dW(family, h, x, y, 1) - dy) < 1e-6 * scale
        assert abs(kernels.lapW(family, h, x, y) - lap) < 1e-3 * scale / h
