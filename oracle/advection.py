"""Gaussian vortex convection (Sec. 6.2): linear advection through a
non-periodic box with inflow and outflow, the spectral SPH gradient on the
FC-extended grid (both axes).

Readings of the printed equations (they are garbled): the equation is
    du/dt + Cx du/dx + Cy du/dy = 0        (the second derivative is in y),
the initial field u0 = exp(-alpha r^2), r = |x - (x0, y0)|, and the solution
    u = exp(-alpha [(x - x0 - Cx t)^2 + (y - y0 - Cy t)^2]);
alpha is not given (50 here).  Time stepping: the low-storage RK3 of the
projection step (Sec. 2.2), u <- u + dt (-g_k F_k - z_k F_{k-1}) with
F = Cx du/dx + Cy du/dy.  After every substep the inflow edges (x = 0 and
y = 0 for positive Cx, Cy) take the exact solution at the substep's time; the
outflow edges are free.  Grid: nodes on [0, 1]^2 including the edges.
"""
import numpy as np

from . import ops
from .step import scheme_coefficients


def exact(X, Y, t, alpha=50.0, x0=0.5, y0=0.5, cx=1.0, cy=0.5):
    return np.exp(-alpha * ((X - x0 - cx * t) ** 2 + (Y - y0 - cy * t) ** 2))


def advect(u, Sx, Sy, E, dt, nsteps, t0=0.0, alpha=50.0, cx=1.0, cy=0.5):
    """nsteps RK3 steps from u at time t0 (n x n nodes on [0,1]^2)."""
    n = u.shape[0]
    x = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    A, G, Z = scheme_coefficients("rk3")
    Fp = np.zeros_like(u)
    t = t0
    for _ in range(nsteps):
        tc = t
        for k in range(3):
            ux, uy = ops.apply_symbols(u, [Sx, Sy], E, E)
            F = cx * ux + cy * uy
            u = u + dt * (-G[k] * F - Z[k] * Fp)
            Fp = F
            tc += A[k] * dt
            ue = exact(X, Y, tc, alpha, cx=cx, cy=cy)
            u[0, :] = ue[0, :]
            u[:, 0] = ue[:, 0]
        t += dt
    return u
