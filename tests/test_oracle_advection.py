"""Pins for oracle.advection (Sec. 6.2): the convected Gaussian leaves the box
through the outflow edges and the error against the exact solution falls at
the fourth order the paper reports for the G4 kernel."""
import numpy as np

from oracle import advection
from oracle.symbols import symbol_closed
from tables import gram_golden


def _run(n, T=0.1, dt=5e-4):
    E = gram_golden(5, 25)
    dx = 1.0 / (n - 1)
    h = 1.3 * dx
    Sx = symbol_closed("DX", "G4", h, n + 25, n + 25, dx, dx)
    Sy = symbol_closed("DY", "G4", h, n + 25, n + 25, dx, dx)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    u = advection.advect(advection.exact(X, Y, 0.0), Sx, Sy, E, dt, int(round(T / dt)))
    return np.sqrt(np.mean((u - advection.exact(X, Y, T)) ** 2))


def test_exact_solution_moves_with_the_flow():
    x = np.linspace(0, 1, 11)
    X, Y = np.meshgrid(x, x, indexing="ij")
    assert np.isclose(advection.exact(X, Y, 0.0)[5, 5], 1.0)
    # at t = 0.2 the centre sits at (0.7, 0.6)
    assert np.isclose(advection.exact(np.array(0.7), np.array(0.6), 0.2), 1.0)


def test_gaussian_convection_converges_at_fourth_order():
    e24, e48 = _run(24), _run(48)
    order = np.log(e24 / e48) / np.log(47.0 / 23.0)
    assert e48 < 1e-3
    assert order > 3.5, (e24, e48, order)
