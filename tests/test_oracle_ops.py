"""Pins for oracle.ops (Eqs. 11, 13, 16, 30)."""
import numpy as np
import pytest

from oracle import ops, symbols, norms
from tables import gram_golden


def test_delta_kernel_gives_exact_fourier_derivative():
    # h = 0: W_hat = 1, the operator is textbook Fourier differentiation; exact on
    # band-limited periodic fields (no FC in either direction).
    m0, m1 = 16, 12
    dx, dy = 1.0 / m0, 1.0 / m1
    x = np.arange(m0) * dx
    y = np.arange(m1) * dy
    X, Y = np.meshgrid(x, y, indexing="ij")
    f = np.sin(2 * np.pi * 3 * X + 0.3) * np.cos(2 * np.pi * 2 * Y) + np.cos(2 * np.pi * 5 * Y - 1.0)
    fx = 2 * np.pi * 3 * np.cos(2 * np.pi * 3 * X + 0.3) * np.cos(2 * np.pi * 2 * Y)
    fy = -2 * np.pi * 2 * np.sin(2 * np.pi * 3 * X + 0.3) * np.sin(2 * np.pi * 2 * Y) - 2 * np.pi * 5 * np.sin(2 * np.pi * 5 * Y - 1.0)
    lap = -(2 * np.pi) ** 2 * ((9 + 4) * np.sin(2 * np.pi * 3 * X + 0.3) * np.cos(2 * np.pi * 2 * Y) + 25 * np.cos(2 * np.pi * 5 * Y - 1.0))
    S = [symbols.symbol_closed(op, "G4", 0.0, m0, m1, dx, dy) for op in ("DX", "DY", "LAP")]
    ox, oy, ol = ops.apply_symbols(f, S, None, None)
    assert np.abs(ox - fx).max() < 1e-11
    assert np.abs(oy - fy).max() < 1e-11
    assert np.abs(ol - lap).max() < 1e-9


def test_single_mode_is_multiplied_by_its_symbol():
    m0, m1 = 12, 10
    dx = dy = 0.1
    h = 0.13
    kx = 2 * np.pi * 2 / (m0 * dx)
    ky = 2 * np.pi * 3 / (m1 * dy)
    X, Y = np.meshgrid(np.arange(m0) * dx, np.arange(m1) * dy, indexing="ij")
    f = np.cos(kx * X + ky * Y)
    s = (kx * kx + ky * ky) * h * h / 4
    Wh = symbols.kernel_transform("G8", np.array(s))
    S = symbols.symbol_closed("DX", "G8", h, m0, m1, dx, dy)
    out = ops.apply_symbols(f, [S], None, None)[0]
    np.testing.assert_allclose(out, -kx * Wh * np.sin(kx * X + ky * Y), atol=1e-12)


def _paper_test_function(N):
    dx = 1.0 / N
    dy = 1.0 / (N - 1)
    X, Y = np.meshgrid(np.arange(N) * dx, np.arange(N) * dy, indexing="ij")
    g1 = Y * (1 - Y)
    g2 = g1 ** 2
    f = np.sin(2 * np.pi * X) * g1 + 0.5 * np.cos(4 * np.pi * X) * g2
    fx = 2 * np.pi * np.cos(2 * np.pi * X) * g1 - 2 * np.pi * np.sin(4 * np.pi * X) * g2
    g2pp = 2 - 12 * Y + 12 * Y ** 2
    lap = np.sin(2 * np.pi * X) * (-4 * np.pi ** 2 * g1 - 2) + 0.5 * np.cos(4 * np.pi * X) * (-16 * np.pi ** 2 * g2 + g2pp)
    return f, fx, lap, dx, dy


def test_operator_convergence_on_paper_test_function():
    # Sec. 6.1, Eq. 35: gradient and Laplacian converge at better than 4th order in
    # the paper; here FC(Gram) d=5, C=25 with G4, h = 1.3 dy gives slope ~4.
    E = gram_golden(5, 25)
    eg, el = [], []
    for N in (32, 64, 128):
        f, fx, lap, dx, dy = _paper_test_function(N)
        h = 1.3 * dy
        S = [symbols.symbol_closed(op, "G4", h, N, N + 25, dx, dy) for op in ("DX", "LAP")]
        ox, ol = ops.apply_symbols(f, S, E)
        eg.append(norms.l2_abs(ox, fx))
        el.append(norms.l2_abs(ol, lap))
    rg = np.log2(np.array(eg[:-1]) / np.array(eg[1:]))
    rl = np.log2(np.array(el[:-1]) / np.array(el[1:]))
    assert np.all(rg > 3.7) and np.all(rl > 3.7), (eg, el)
    assert eg[1] < 1e-4 and el[1] < 1e-3
