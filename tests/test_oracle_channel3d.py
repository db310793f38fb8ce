"""Pins for oracle.channel3d: the 3D transforms against numpy's FFT, the 3D
operators against the 2D oracle on fields that do not depend on z (or on x),
the 3D PPE on manufactured eigenfunctions, and the 3D channel start-up against
the analytic series (Sec. 6.3)."""
import numpy as np
import pytest

from oracle import channel3d as c3
from oracle import norms, ops
from oracle.symbols import symbol_closed
from paper_2606_06247_gb300 import inputs
from tables import gram_golden

E = gram_golden(5, 25)


def test_dft3_is_numpy_fftn():
    rng = np.random.default_rng(1)
    F = rng.standard_normal((5, 6, 7)) + 1j * rng.standard_normal((5, 6, 7))
    np.testing.assert_allclose(c3.dft3(F), np.fft.fftn(F), rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(c3.idft3(c3.dft3(F)), F, rtol=1e-12, atol=1e-12)


def _grid(nx, nz, ny):
    dy = 1.0 / (ny - 1)
    return nx * dy, nz * dy, 1.0  # isotropic lattice: dx = dz = dy


@pytest.mark.parametrize("op", ["W", "DX", "DY", "LAP"])
def test_z_invariant_field_gives_the_2d_operators(op):
    nx, nz, ny = 8, 5, 14
    Lx, Lz, Ly = _grid(nx, nz, ny)
    f2 = inputs.smooth_field(nx, ny, seed=3)
    f3 = np.repeat(f2[:, None, :], nz, axis=1)
    dx, dz, dy = Lx / nx, Lz / nz, Ly / (ny - 1)
    h = 1.3 * dx
    my = ny + 25
    S3 = c3.symbol3(op, "G4", h, nx, nz, my, dx, dz, dy)
    out3 = c3.apply_symbols3(f3, [S3], E)[0]
    S2 = symbol_closed(op, "G4", h, nx, my, dx, dy)
    out2 = ops.apply_symbols(f2, [S2], E)[0]
    for k in range(nz):
        np.testing.assert_allclose(out3[:, k, :], out2, rtol=0, atol=1e-12 * max(1.0, np.abs(out2).max()))
    if op == "W":
        return
    # d/dz of a z-invariant field is zero
    Sz = c3.symbol3("DZ", "G4", h, nx, nz, my, dx, dz, dy)
    assert np.abs(c3.apply_symbols3(f3, [Sz], E)[0]).max() < 1e-12 * np.abs(f3).max()


def test_x_invariant_field_gives_dz_as_the_2d_dx():
    nx, nz, ny = 4, 8, 14
    Lx, Lz, Ly = _grid(nx, nz, ny)
    g2 = inputs.smooth_field(nz, ny, seed=4)          # g(z, y)
    f3 = np.repeat(g2[None, :, :], nx, axis=0)
    dx, dz, dy = Lx / nx, Lz / nz, Ly / (ny - 1)
    h = 1.3 * dx
    my = ny + 25
    Sz = c3.symbol3("DZ", "G4", h, nx, nz, my, dx, dz, dy)
    out3 = c3.apply_symbols3(f3, [Sz], E)[0]
    S2 = symbol_closed("DX", "G4", h, nz, my, dz, dy)  # the z axis in the role of x
    out2 = ops.apply_symbols(g2, [S2], E)[0]
    for i in range(nx):
        np.testing.assert_allclose(out3[i], out2, rtol=0, atol=1e-12 * np.abs(out2).max())


def test_ppe3_recovers_manufactured_eigenfunctions():
    nx, nz, ny = 6, 8, 9
    Lx, Lz, Ly = 1.3, 0.7, 1.0
    x = np.arange(nx) * Lx / nx
    z = np.arange(nz) * Lz / nz
    y = np.linspace(0, Ly, ny)
    X, Z, Y = np.meshgrid(x, z, y, indexing="ij")
    for a, c, l in [(1, 2, 3), (2, 0, 1), (0, 3, 4), (3, 4, 8)]:
        phi = np.cos(2 * np.pi * a * X / Lx) * np.cos(2 * np.pi * c * Z / Lz) * np.cos(np.pi * l * Y / Ly)
        lam = (2 * np.pi * a / Lx) ** 2 + (2 * np.pi * c / Lz) ** 2 + (np.pi * l / Ly) ** 2
        got = c3.ppe_solve3(-lam * phi, Lx, Lz, Ly)
        np.testing.assert_allclose(got, phi, rtol=0, atol=1e-12)
    rng = np.random.default_rng(2)
    b = rng.standard_normal((nx, nz, ny))
    r = c3.laplacian3(c3.ppe_solve3(b, Lx, Lz, Ly), Lx, Lz, Ly) - b
    assert np.abs(r - r.mean()).max() < 1e-12 * np.abs(b).max()


def _series(y, t, F, nu, nterms=199):
    u = F / (2 * nu) * y * (1 - y)
    for n in range(1, nterms, 2):
        u = u - 4 * F / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * y) * np.exp(-nu * n * n * np.pi ** 2 * t)
    return u


def test_channel3d_startup_matches_analytic_series():
    nx, nz, ny = 6, 4, 24
    Lx, Lz, Ly = _grid(nx, nz, ny)
    p = c3.Problem3(nx=nx, nz=nz, ny=ny, Lx=Lx, Lz=Lz, Ly=Ly, family="G4", h_over_dx=1.3, E_dir=E, E_neu=E,
                    nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0, 0.0), scheme="rk3").build_symbols()
    z = np.zeros((nx, nz, ny))
    u, v, w, phi = c3.isph_steps3(p, z, z, z, 40)
    ua = np.broadcast_to(_series(np.linspace(0, 1, ny), 0.04, 0.8, 0.1), u.shape)
    assert norms.l2_rel(u, ua) < 1e-3
    assert np.abs(v).max() < 1e-12 and np.abs(w).max() < 1e-12
