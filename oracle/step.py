"""Projection time step of the FC-based spectral ISPH scheme (Sec. 2.2, Eqs. 5-9).

Reading of the paper's signs (its Eqs. 5-6 carry +nu lap(u) inside F and
subtract the body force): with the physical right-hand side
du/dt = -(u.grad)u + nu lap(u) - grad(P)/rho + f,

    F^k  = (u^k . grad) u^k - nu lap(u^k)                         (Eq. 6)
    u*   = u^k + dt ( -g_k F^k - z_k F^{k-1} + a_k f )             (Eq. 5, pressure-free)
    lap(phi) = rho / (a_k dt) div(u*)                              (Eq. 8)
    u^{k+1} = u* - a_k dt / rho grad(phi)                          (Eq. 9)

The PPE coefficient rho/(a_k dt) is the one for which the correction removes
the divergence (Eq. 8 as printed has a_k in the numerator; identical for the
FOP, a = 1).  Wall nodes get their prescribed velocity after u* and after the
correction (Eq. 3), and the FC reads those values.  Spatial operators are the
FC-extended spectral SPH operators (ops.py) with the Dirichlet table for
velocity and the Neumann table for phi (Sec. 4.4); the PPE is the spectral
solve on the physical nodes (ppe.py).

Schemes: FOP (a = g = 1, z = 0; one substep per step) and low-storage RK3 with
a = [8/15, 2/15, 1/3], g = [8/15, 5/12, 3/4], z = [0, -17/60, -5/12].
"""
from dataclasses import dataclass, field

import numpy as np

from . import fc as fcmod
from . import ops
from .ppe import extended_projection, ppe_solve
from .symbols import symbol_closed

RK3_A = (8.0 / 15.0, 2.0 / 15.0, 1.0 / 3.0)
RK3_G = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RK3_Z = (0.0, -17.0 / 60.0, -5.0 / 12.0)
FOP_COEF = ((1.0,), (1.0,), (0.0,))


def scheme_coefficients(scheme):
    if scheme == "fop":
        return FOP_COEF
    if scheme == "rk3":
        return (RK3_A, RK3_G, RK3_Z)
    raise ValueError(scheme)


@dataclass
class Problem:
    """A 2D wall-bounded grid: y always has walls; x periodic or walled.

    Nodes x_i = i dx (i < nx), y_j = j dy (j < ny); walls sit on nodes:
    dy = Ly/(ny-1); dx = Lx/nx for periodic x, Lx/(nx-1) with x walls."""
    nx: int
    ny: int
    Lx: float
    Ly: float
    x_walls: bool
    family: str
    h_over_dx: float
    E_dir: np.ndarray
    E_neu: np.ndarray
    nu: float = 0.1
    rho: float = 1.0
    dt: float = 1e-3
    force: tuple = (0.0, 0.0)
    u_bottom: float = 0.0
    u_top: float = 0.0
    scheme: str = "fop"
    # "dct": the physical-domain spectral PPE of Sec. 5.1 (the method);
    # "extended": the projection on the FC-extended periodic grid that Sec. 5.2
    # leaves for future work (ppe.extended_projection), kept to measure it
    proj: str = "dct"
    sym: dict = field(default_factory=dict)

    @property
    def dx(self):
        return self.Lx / (self.nx - 1) if self.x_walls else self.Lx / self.nx

    @property
    def dy(self):
        return self.Ly / (self.ny - 1)

    @property
    def h(self):
        return self.h_over_dx * self.dx

    def extended_shape(self):
        n_cont = self.E_dir.shape[0]
        mx = self.nx + n_cont if self.x_walls else self.nx
        return mx, self.ny + n_cont

    def build_symbols(self):
        mx, my = self.extended_shape()
        for op in ("DX", "DY", "LAP"):
            self.sym[op] = symbol_closed(op, self.family, self.h, mx, my, self.dx, self.dy)
        return self

    def E_x(self, bc):
        if not self.x_walls:
            return None
        return self.E_dir if bc == fcmod.DIRICHLET else self.E_neu

    def E_y(self, bc):
        return self.E_dir if bc == fcmod.DIRICHLET else self.E_neu


def wall_reset(p, u, v):
    """Prescribed wall velocity (Eq. 3).  y walls: u = u_bottom / u_top, v = 0.
    x walls (if any) get u = v = 0 and win at the corners."""
    u = u.copy()
    v = v.copy()
    u[:, 0] = p.u_bottom
    u[:, -1] = p.u_top
    v[:, 0] = 0.0
    v[:, -1] = 0.0
    if p.x_walls:
        u[0, :] = 0.0
        u[-1, :] = 0.0
        v[0, :] = 0.0
        v[-1, :] = 0.0
    return u, v


def momentum_update(u, F, F_prev, force, dt, a, g, z):
    """u* = u + dt (-g F - z F_prev + a force)  (Eq. 5 with the sign reading above)."""
    return u + dt * (-g * F - z * F_prev + a * force)


def substep(p, u, v, Fu_prev, Fv_prev, a, g, z):
    """One projection substep; returns (u, v, phi, Fu, Fv)."""
    D = fcmod.DIRICHLET
    N = fcmod.NEUMANN
    S = p.sym
    ux, uy, ul = ops.apply_symbols(u, [S["DX"], S["DY"], S["LAP"]], p.E_y(D), p.E_x(D))
    vx, vy, vl = ops.apply_symbols(v, [S["DX"], S["DY"], S["LAP"]], p.E_y(D), p.E_x(D))
    Fu = u * ux + v * uy - p.nu * ul
    Fv = u * vx + v * vy - p.nu * vl
    us = momentum_update(u, Fu, Fu_prev, p.force[0], p.dt, a, g, z)
    vs = momentum_update(v, Fv, Fv_prev, p.force[1], p.dt, a, g, z)
    us, vs = wall_reset(p, us, vs)
    if p.proj == "extended":
        un, vn = extended_projection(us, vs, S["DX"], S["DY"], p.E_y(D), p.E_x(D))
        un, vn = wall_reset(p, un, vn)
        return un, vn, np.zeros_like(u), Fu, Fv
    div = ops.divergence(us, vs, S["DX"], S["DY"], p.E_y(D), p.E_x(D))
    b = (p.rho / (a * p.dt)) * div
    phi = ppe_solve(b, p.Lx, p.Ly, p.x_walls)
    px, py = ops.apply_symbols(phi, [S["DX"], S["DY"]], p.E_y(N), p.E_x(N))
    un = us - (a * p.dt / p.rho) * px
    vn = vs - (a * p.dt / p.rho) * py
    un, vn = wall_reset(p, un, vn)
    return un, vn, phi, Fu, Fv


def isph_steps(p, u, v, nsteps):
    """Advance nsteps full steps; returns (u, v, phi)."""
    A, G, Z = scheme_coefficients(p.scheme)
    Fu_prev = np.zeros_like(u)
    Fv_prev = np.zeros_like(v)
    phi = np.zeros_like(u)
    for _ in range(nsteps):
        for k in range(len(A)):
            u, v, phi, Fu_prev, Fv_prev = substep(p, u, v, Fu_prev, Fv_prev, A[k], G[k], Z[k])
    return u, v, phi
