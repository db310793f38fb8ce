"""The projection on the FC-extended periodic grid (the alternative Sec. 5.2
names and leaves for future work): oracle.ppe.extended_projection.

Pins: the corrected extended field has zero discrete divergence (the same
gradient symbols' divergence) at round-off; the projection is idempotent; it
removes gradient fields and keeps divergence-free (stream-function) fields.
Finding, recorded as a test: used inside the time step (truncate to the
physical nodes, reset the walls, FC-extend again at the next substep) it is
unstable with either FC variant, while the physical-domain DCT solve of the
method is stable on the same grid."""
import numpy as np
import pytest

from oracle import fc, ppe, step, symbols
from oracle.dft import dft2, idft2
from tables import gram_golden


def _walled_case(nx=14, ny=12, x_walls=True, seed=0):
    E = gram_golden(5, 25)
    dy = 1.0 / (ny - 1)
    dx = dy
    mx = nx + 25 if x_walls else nx
    h = 1.3 * dy
    Sx = symbols.symbol_closed("DX", "G4", h, mx, ny + 25, dx, dy)
    Sy = symbols.symbol_closed("DY", "G4", h, mx, ny + 25, dx, dy)
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nx, ny)), rng.standard_normal((nx, ny)), Sx, Sy, E, (E if x_walls else None)


def _ext_div(ue, ve, Sx, Sy):
    return np.real(idft2(Sx * dft2(ue) + Sy * dft2(ve)))


@pytest.mark.parametrize("x_walls", [False, True])
def test_extended_divergence_vanishes_at_round_off(x_walls):
    us, vs, Sx, Sy, Ey, Ex = _walled_case(x_walls=x_walls)
    u, v, ue, ve = ppe.extended_projection(us, vs, Sx, Sy, Ey, Ex, return_extended=True)
    Ue = fc.extend2d(us, Ey, Ex)
    Ve = fc.extend2d(vs, Ey, Ex)
    before = np.abs(_ext_div(Ue, Ve, Sx, Sy)).max()
    after = np.abs(_ext_div(ue, ve, Sx, Sy)).max()
    scale = max(np.abs(Ue).max(), np.abs(Ve).max()) * max(np.abs(Sx).max(), np.abs(Sy).max())
    assert before > 1.0 and after < 1e-13 * scale, (before, after, scale)
    np.testing.assert_array_equal(u, ue[:us.shape[0], :us.shape[1]])


def _periodic(m0=16, m1=18):
    dx, dy = 1.0 / m0, 1.0 / m1
    h = 1.3 * dx
    Sx = symbols.symbol_closed("DX", "G4", h, m0, m1, dx, dy)
    Sy = symbols.symbol_closed("DY", "G4", h, m0, m1, dx, dy)
    X, Y = np.meshgrid(np.arange(m0) * dx, np.arange(m1) * dy, indexing="ij")
    return Sx, Sy, X, Y


def test_projection_is_idempotent():
    Sx, Sy, X, Y = _periodic()
    rng = np.random.default_rng(2)
    u, v = rng.standard_normal(X.shape), rng.standard_normal(X.shape)
    u1, v1 = ppe.extended_projection(u, v, Sx, Sy, None, None)
    u2, v2 = ppe.extended_projection(u1, v1, Sx, Sy, None, None)
    assert np.abs(u2 - u1).max() < 1e-13 and np.abs(v2 - v1).max() < 1e-13
    assert np.abs(u1 - u).max() > 0.1


def test_gradients_are_removed_and_solenoidal_fields_kept():
    Sx, Sy, X, Y = _periodic()
    tp = 2 * np.pi
    psi = np.sin(tp * (2 * X + 3 * Y) + 0.4) + np.cos(tp * (X - 5 * Y))
    P = dft2(psi)
    gx, gy = np.real(idft2(Sx * P)), np.real(idft2(Sy * P))       # discrete gradient of psi
    u, v = ppe.extended_projection(gx, gy, Sx, Sy, None, None)
    assert np.abs(u).max() < 1e-12 * np.abs(gx).max() and np.abs(v).max() < 1e-12 * np.abs(gy).max()
    su, sv = np.real(idft2(Sy * P)), -np.real(idft2(Sx * P))       # discrete curl of psi: divergence-free
    u, v = ppe.extended_projection(su, sv, Sx, Sy, None, None)
    assert np.abs(u - su).max() < 1e-12 * np.abs(su).max() and np.abs(v - sv).max() < 1e-12 * np.abs(sv).max()


def _substep_radius(proj, variant, N=32, iters=60):
    if variant == "gram":
        E = En = gram_golden(5, 25)
    else:
        E, En = fc.paper_table(10, N // 4, 5, fc.DIRICHLET), fc.paper_table(10, N // 4, 5, fc.NEUMANN)
    dy = 1.0 / (N - 1)
    p = step.Problem(nx=N, ny=N, Lx=N * dy, Ly=1.0, x_walls=False, family="G4", h_over_dx=1.3, E_dir=E, E_neu=En,
                     nu=0.1, rho=1.0, dt=1e-3, scheme="fop", proj=proj).build_symbols()
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal((N, N)), rng.standard_normal((N, N))
    z = np.zeros((N, N))
    eps = 1e-8
    lam = 0.0
    for _ in range(iters):
        n0 = np.sqrt((u * u).sum() + (v * v).sum())
        u, v = u / n0, v / n0
        un, vn, _, _, _ = step.substep(p, eps * u, eps * v, z, z, 1.0, 1.0, 0.0)
        u, v = un / eps, vn / eps
        lam = np.sqrt((u * u).sum() + (v * v).sum())
    return lam


@pytest.mark.parametrize("variant,at_least", [("gram", 100.0), ("paper", 5.0)])
def test_extended_projection_in_the_step_is_unstable(variant, at_least):
    # channel 32^2, nu = 0.1, dt = 1e-3, h = 1.3 dx: the DCT solve contracts
    # (0.987), the extended projection amplifies (195 with FC(Gram), 7 with the
    # paper's FC): the continuation of each re-extension (||E|| ~ 1e4 for
    # FC(Gram)) feeds the extended solve's correction back into the fluid.
    assert _substep_radius("dct", variant) < 1.0
    assert _substep_radius("extended", variant) > at_least
