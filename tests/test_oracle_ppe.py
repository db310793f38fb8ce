"""Pins for oracle.ppe (Eqs. 31-33): manufactured eigenfunctions are recovered
to round-off, and the solve inverts the transform-space Laplacian."""
import numpy as np
import pytest

from oracle import ppe


@pytest.mark.parametrize("nx,ny", [(12, 9), (16, 16), (7, 20)])
def test_channel_eigenfunctions(nx, ny):
    Lx, Ly = 1.3, 1.0
    x = np.arange(nx) * Lx / nx
    y = np.arange(ny) * Ly / (ny - 1)
    X, Y = np.meshgrid(x, y, indexing="ij")
    for k, l in [(1, 0), (0, 3), (2, 1), (nx // 2, ny - 1)]:
        phi = np.cos(2 * np.pi * k * X / Lx + 0.4 * (k > 0)) * np.cos(np.pi * l * Y / Ly)
        b = -((2 * np.pi * k / Lx) ** 2 + (np.pi * l / Ly) ** 2) * phi
        got = ppe.ppe_solve(b, Lx, Ly, x_walls=False)
        if k == nx // 2 and nx % 2 == 0:
            continue  # the Nyquist mode of the sine part is not representable
        np.testing.assert_allclose(got, phi, atol=1e-11)


@pytest.mark.parametrize("nx,ny", [(9, 9), (13, 8)])
def test_cavity_eigenfunctions(nx, ny):
    Lx, Ly = 1.0, 0.8
    X, Y = np.meshgrid(np.linspace(0, Lx, nx), np.linspace(0, Ly, ny), indexing="ij")
    for k, l in [(1, 0), (0, 2), (3, 4), (nx - 1, ny - 1)]:
        phi = np.cos(np.pi * k * X / Lx) * np.cos(np.pi * l * Y / Ly)
        b = -((np.pi * k / Lx) ** 2 + (np.pi * l / Ly) ** 2) * phi
        np.testing.assert_allclose(ppe.ppe_solve(b, Lx, Ly, x_walls=True), phi, atol=1e-11)


def test_solve_inverts_laplacian_up_to_the_mean_mode():
    rng = np.random.default_rng(1)
    for xw in (False, True):
        b = rng.standard_normal((10, 11))
        phi = ppe.ppe_solve(b, 1.0, 1.0, xw)
        r = ppe.laplacian(phi, 1.0, 1.0, xw) - b
        # the residual is the (0,0) transform mode of b alone: a constant field
        assert np.abs(r - r.mean()).max() < 1e-12 * np.abs(b).max()

