"""3D channel: the method of the paper in three dimensions, x and z periodic,
walls at y = 0 and y = Ly (FC in the wall-normal direction only, as for the 2D
channel of Sec. 4.6).

Arrays are f[i, k, j] = f(x_i, z_k, y_j); x_i = i dx (dx = Lx/nx), z_k = k dz
(dz = Lz/nz), y_j = j dy (dy = Ly/(ny-1), walls on nodes).

  operators (Eqs. 11/13/16 in 3D): F = FC_y(f) on the nx x nz x (ny + n_cont)
      periodic grid, out = IDFT3( DFT3(F) . S )[:, :, :ny] with S = W_hat,
      i kx W_hat, i ky W_hat, i kz W_hat or -|k|^2 W_hat, W_hat = e^{-s}
      sum_{m<n} s^m/m!, s = |k|^2 h^2 / 4 (the Gaussian family's transform has
      this form in every dimension; a first derivative is zero on the Nyquist
      plane of its own axis);
  PPE (Eqs. 31-33 in 3D): DFT in x and z, DCT-I in y, division by
      -(lam_x^2 + lam_z^2 + lam_y^2), zero (0,0,0) mode;
  step (Eqs. 5-9) for u = (u, v, w) with the same sign reading as the 2D
      step (oracle/step.py): F = (u . grad) u - nu lap u, u* = u + dt(-g F -
      z F_prev + a f), lap phi = rho/(a dt) div u*, u = u* - a dt/rho grad phi;
      y walls get u = u_bottom / u_top and v = w = 0 after u* and after the
      correction.
"""
from dataclasses import dataclass, field

import numpy as np

from .dft import dct1_matrix, dft_matrix, idct1_matrix, idft_matrix, signed_wavenumbers
from .fc import extend_last_axis
from .step import scheme_coefficients
from .symbols import kernel_transform, wavenumbers


def _along(M, F, axis):
    """Apply the matrix M along one axis of F."""
    return np.moveaxis(np.tensordot(M, F, axes=([1], [axis])), 0, axis)


def dft3(F):
    """3D DFT of an (n0, n1, n2) array (the defining sums, axis by axis)."""
    for ax in range(3):
        F = _along(dft_matrix(F.shape[ax]), F, ax)
    return F


def idft3(G):
    """Inverse 3D DFT (with 1/(n0 n1 n2))."""
    for ax in range(3):
        G = _along(idft_matrix(G.shape[ax]), G, ax)
    return G


def symbol3(op, family, h, mx, mz, my, dx, dz, dy):
    """Symbols on the extended mx x mz x my grid (axes x, z, y)."""
    kx = wavenumbers(mx, dx)
    kz = wavenumbers(mz, dz)
    ky = wavenumbers(my, dy)
    KX, KZ, KY = np.meshgrid(kx, kz, ky, indexing="ij")
    Wh = kernel_transform(family, (KX * KX + KZ * KZ + KY * KY) * (h * h) / 4.0)

    def own(k, m):
        k = k.copy()
        if m % 2 == 0:
            k[m // 2] = 0.0
        return k

    if op == "W":
        return Wh.astype(np.complex128)
    if op == "DX":
        return 1j * own(kx, mx)[:, None, None] * Wh
    if op == "DZ":
        return 1j * own(kz, mz)[None, :, None] * Wh
    if op == "DY":
        return 1j * own(ky, my)[None, None, :] * Wh
    if op == "LAP":
        return -(KX * KX + KZ * KZ + KY * KY) * Wh
    raise ValueError(op)


def apply_symbols3(f, symbols, E):
    """One forward transform of the y-extended field, one inverse per symbol."""
    nx, nz, ny = f.shape
    Fh = dft3(extend_last_axis(np.asarray(f, dtype=np.float64), E))
    return [np.real(idft3(Fh * S)[:, :, :ny]).copy() for S in symbols]


def divergence3(fx, fy, fz, Sx, Sy, Sz, E):
    nx, nz, ny = fx.shape
    G = sum(S * dft3(extend_last_axis(np.asarray(f, dtype=np.float64), E)) for f, S in ((fx, Sx), (fy, Sy), (fz, Sz)))
    return np.real(idft3(G)[:, :, :ny]).copy()


def ppe_eigenvalues3(nx, nz, ny, Lx, Lz, Ly):
    return (2.0 * np.pi * signed_wavenumbers(nx) / Lx, 2.0 * np.pi * signed_wavenumbers(nz) / Lz,
            np.pi * np.arange(ny) / Ly)


def ppe_solve3(b, Lx, Lz, Ly):
    """phi with lap(phi) = b: DFT x, DFT z, DCT-I y, division, inverse."""
    nx, nz, ny = b.shape
    bh = _along(dct1_matrix(ny), _along(dft_matrix(nz), _along(dft_matrix(nx), np.asarray(b, float), 0), 1), 2)
    lx, lz, ly = ppe_eigenvalues3(nx, nz, ny, Lx, Lz, Ly)
    den = lx[:, None, None] ** 2 + lz[None, :, None] ** 2 + ly[None, None, :] ** 2
    den[0, 0, 0] = 1.0
    ph = -bh / den
    ph[0, 0, 0] = 0.0
    phi = _along(idct1_matrix(ny), _along(idft_matrix(nz), _along(idft_matrix(nx), ph, 0), 1), 2)
    return np.real(phi).copy()


def laplacian3(phi, Lx, Lz, Ly):
    """The operator ppe_solve3 inverts."""
    nx, nz, ny = phi.shape
    ph = _along(dct1_matrix(ny), _along(dft_matrix(nz), _along(dft_matrix(nx), np.asarray(phi, float), 0), 1), 2)
    lx, lz, ly = ppe_eigenvalues3(nx, nz, ny, Lx, Lz, Ly)
    ph = -(lx[:, None, None] ** 2 + lz[None, :, None] ** 2 + ly[None, None, :] ** 2) * ph
    return np.real(_along(idct1_matrix(ny), _along(idft_matrix(nz), _along(idft_matrix(nx), ph, 0), 1), 2)).copy()


@dataclass
class Problem3:
    nx: int
    nz: int
    ny: int
    Lx: float
    Lz: float
    Ly: float
    family: str
    h_over_dx: float
    E_dir: np.ndarray
    E_neu: np.ndarray
    nu: float = 0.1
    rho: float = 1.0
    dt: float = 1e-3
    force: tuple = (0.0, 0.0, 0.0)   # (x, y, z)
    u_bottom: float = 0.0
    u_top: float = 0.0
    scheme: str = "fop"
    sym: dict = field(default_factory=dict)

    @property
    def dx(self):
        return self.Lx / self.nx

    @property
    def dz(self):
        return self.Lz / self.nz

    @property
    def dy(self):
        return self.Ly / (self.ny - 1)

    @property
    def h(self):
        return self.h_over_dx * self.dx

    def build_symbols(self):
        my = self.ny + self.E_dir.shape[0]
        for op in ("DX", "DY", "DZ", "LAP"):
            self.sym[op] = symbol3(op, self.family, self.h, self.nx, self.nz, my, self.dx, self.dz, self.dy)
        return self


def wall_reset3(p, u, v, w):
    u, v, w = u.copy(), v.copy(), w.copy()
    u[:, :, 0] = p.u_bottom
    u[:, :, -1] = p.u_top
    for a in (v, w):
        a[:, :, 0] = 0.0
        a[:, :, -1] = 0.0
    return u, v, w


def substep3(p, u, v, w, F_prev, a, g, z):
    """One projection substep; returns (u, v, w, phi, F) with F = (Fu, Fv, Fw)."""
    S = p.sym
    E, En = p.E_dir, p.E_neu
    grads = [apply_symbols3(c, [S["DX"], S["DY"], S["DZ"], S["LAP"]], E) for c in (u, v, w)]
    F = tuple(u * cx + v * cy + w * cz - p.nu * cl for cx, cy, cz, cl in grads)
    fx, fy, fz = p.force
    us = u + p.dt * (-g * F[0] - z * F_prev[0] + a * fx)
    vs = v + p.dt * (-g * F[1] - z * F_prev[1] + a * fy)
    ws = w + p.dt * (-g * F[2] - z * F_prev[2] + a * fz)
    us, vs, ws = wall_reset3(p, us, vs, ws)
    b = (p.rho / (a * p.dt)) * divergence3(us, vs, ws, S["DX"], S["DY"], S["DZ"], E)
    phi = ppe_solve3(b, p.Lx, p.Lz, p.Ly)
    px, py, pz = apply_symbols3(phi, [S["DX"], S["DY"], S["DZ"]], En)
    c = a * p.dt / p.rho
    un, vn, wn = wall_reset3(p, us - c * px, vs - c * py, ws - c * pz)
    return un, vn, wn, phi, F


def isph_steps3(p, u, v, w, nsteps):
    """Advance nsteps full steps; returns (u, v, w, phi)."""
    A, G, Z = scheme_coefficients(p.scheme)
    F = (np.zeros_like(u), np.zeros_like(v), np.zeros_like(w))
    phi = np.zeros_like(u)
    for _ in range(nsteps):
        for k in range(len(A)):
            u, v, w, phi, F = substep3(p, u, v, w, F, A[k], G[k], Z[k])
    return u, v, w, phi
