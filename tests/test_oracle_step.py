"""Pins for oracle.step (Sec. 2.2, Eqs. 5-9, Sec. 6.3)."""
import numpy as np
import pytest

from oracle import step, norms
from paper_2606_06247_gb300 import inputs
from tables import gram_golden, paper_constants


def test_rk3_coefficients_are_the_printed_ones():
    c = paper_constants()
    np.testing.assert_allclose(step.RK3_A, c["RK3_a"], rtol=1e-15)
    np.testing.assert_allclose(step.RK3_G, c["RK3_g"], rtol=1e-15)
    np.testing.assert_allclose(step.RK3_Z, c["RK3_z"], rtol=1e-15)


def _ode_error(scheme, dt, lam=-1.3, T=1.0):
    A, G, Z = step.scheme_coefficients(scheme)
    u = np.array([1.0])
    Fp = np.zeros(1)
    for _ in range(int(round(T / dt))):
        for k in range(len(A)):
            F = -lam * u           # du/dt = -F
            u = step.momentum_update(u, F, Fp, 0.0, dt, A[k], G[k], Z[k])
            Fp = F
    return abs(u[0] - np.exp(lam * T))


def test_rk3_is_third_order_and_fop_first_order():
    e = [_ode_error("rk3", dt) for dt in (0.1, 0.05, 0.025)]
    r = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(np.abs(r - 3) < 0.2), r
    e = [_ode_error("fop", dt) for dt in (0.01, 0.005)]
    assert abs(np.log2(e[0] / e[1]) - 1) < 0.1


def _startup_series(y, t, F, nu, nterms=4001):
    u = F / (2 * nu) * y * (1 - y)
    for n in range(1, nterms, 2):
        u -= 4 * F / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * y) * np.exp(-nu * n * n * np.pi ** 2 * t)
    return u


def test_channel_startup_matches_analytic_series():
    # Sec. 6.3 channel from rest: u(y,t) = F/(2nu) y(1-y) - sum_{n odd} 4F/(nu pi^3 n^3) sin(n pi y) e^{-nu n^2 pi^2 t}.
    N = 32
    E = gram_golden(5, 25)
    p = step.Problem(nx=N, ny=N, Lx=N / (N - 1), Ly=1.0, x_walls=False, family="G4", h_over_dx=1.3,
                     E_dir=E, E_neu=E, nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0), scheme="rk3").build_symbols()
    u, v = inputs.channel_initial(N, N, seed=1)
    u, v, phi = step.isph_steps(p, u, v, 40)
    y = np.linspace(0, 1, N)
    ua = np.tile(_startup_series(y, 0.04, 0.8, 0.1), (N, 1))
    assert norms.l2_rel(u, ua) < 1e-3
    assert np.abs(v).max() < 1e-5 and np.abs(phi).max() < 1e-4
    assert np.all(u[:, 0] == 0) and np.all(u[:, -1] == 0) and np.all(v[:, [0, -1]] == 0)


def test_cavity_walls_and_lid_are_imposed():
    N = 16
    E = gram_golden(5, 25)
    p = step.Problem(nx=N, ny=N, Lx=1.0, Ly=1.0, x_walls=True, family="G8", h_over_dx=1.3,
                     E_dir=E, E_neu=E, nu=1e-3, rho=1.0, dt=1e-3, u_top=1.0, scheme="rk3").build_symbols()
    u, v = inputs.cavity_initial(N, N)
    u, v, phi = step.isph_steps(p, u, v, 3)
    assert np.all(u[1:-1, -1] == 1.0) and u[0, -1] == 0 and u[-1, -1] == 0
    assert np.all(u[0, :] == 0) and np.all(v[:, 0] == 0) and np.all(np.isfinite(u))


def _couette_series(y, t, U, nu, nterms=400):
    # Sec. 6.4: u(y,t) = U y + (2U/pi) sum_{n>=1} (-1)^n / n sin(n pi y) e^{-nu n^2 pi^2 t}
    u = U * y
    for n in range(1, nterms):
        u = u + 2 * U / np.pi * (-1) ** n / n * np.sin(n * np.pi * y) * np.exp(-nu * n * n * np.pi ** 2 * t)
    return u


def test_couette_startup_matches_analytic_series():
    # moving top wall (u = 1 at y = 1), stationary bottom wall, fluid at rest: the
    # asymmetric Dirichlet data go through the same FC extension unchanged
    N = 32
    E = gram_golden(5, 25)
    p = step.Problem(nx=N, ny=N, Lx=N / (N - 1), Ly=1.0, x_walls=False, family="G4", h_over_dx=1.3,
                     E_dir=E, E_neu=E, nu=0.1, rho=1.0, dt=1e-3, force=(0.0, 0.0), u_top=1.0,
                     scheme="rk3").build_symbols()
    z = np.zeros((N, N))
    u, v, phi = step.isph_steps(p, z, z, 100)
    y = np.linspace(0, 1, N)
    ua = np.tile(_couette_series(y, 0.1, 1.0, 0.1), (N, 1))
    assert norms.l2_rel(u, ua) < 2e-3
    assert np.abs(v).max() < 1e-12                       # the flow stays one-dimensional
    assert np.abs(u - u.mean(axis=0, keepdims=True)).max() < 1e-12
    assert np.all(u[:, 0] == 0) and np.all(u[:, -1] == 1)


def _energy(u, v, h):
    # trapezoidal rule for E = 1/2 int |u|^2 over the nodes of a walled square
    w = np.ones(u.shape[0])
    w[0] = w[-1] = 0.5
    return 0.5 * h * h * float((w[:, None] * w[None, :] * (u ** 2 + v ** 2)).sum())


def test_dipole_initial_energy_is_two():
    # Sec. 6.5: omega_e = 299.528 is chosen so that E(0) = 2 (printed to 6 digits)
    for n in (161, 401):
        u, v = inputs.dipole_initial(n)
        assert abs(_energy(u, v, 2.0 / (n - 1)) - 2.0) < 1e-5


def test_dipole_energy_decays_at_twice_nu_times_enstrophy():
    # Navier-Stokes with no-slip walls: dE/dt = -nu int |grad u|^2 = -2 nu Z,
    # Z = 1/2 int omega^2.  One RK3 step of the oracle at 161^2, Re = 100.
    n = 161
    E = gram_golden(5, 25)
    p = step.Problem(nx=n, ny=n, Lx=2.0, Ly=2.0, x_walls=True, family="G4", h_over_dx=1.3, E_dir=E, E_neu=E,
                     nu=0.01, rho=1.0, dt=1.25e-4, scheme="rk3").build_symbols()
    u0, v0 = inputs.dipole_initial(n)
    h = 2.0 / (n - 1)
    from oracle import ops
    vx, = ops.apply_symbols(v0, [p.sym["DX"]], E, E)
    uy, = ops.apply_symbols(u0, [p.sym["DY"]], E, E)
    Z0 = _energy(vx - uy, np.zeros_like(u0), h)
    u1, v1, _ = step.isph_steps(p, u0, v0, 1)
    rate = (_energy(u1, v1, h) - _energy(u0, v0, h)) / p.dt
    assert abs(rate + 2 * p.nu * Z0) < 3e-3 * 2 * p.nu * Z0
