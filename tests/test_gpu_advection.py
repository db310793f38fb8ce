"""Gaussian vortex convection with inflow and outflow (Sec. 6.2) driven by the
library's FC-extended spectral gradient (spectral_op DX, DY on a grid with
walls on both axes); the low-storage RK3 combination and the inflow reset
are plain tensor arithmetic of the test.  Parity with oracle.advection and
the error against the exact solution."""
import numpy as np
import pytest

from gpu_common import binding, parity_tol, rel_l2, torch_cuda, ulp_floor
from oracle import advection
from oracle.step import scheme_coefficients
from oracle.symbols import symbol_closed
from tables import gram_golden


def _gpu_advect(b, torch, u0, dt, nsteps, prec):
    n = u0.shape[0]
    ctx = b.Context(n, n, 1.0, 1.0, x_walls=True, family="G4", h_over_dx=1.3, prec=prec)
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    A, G, Z = scheme_coefficients("rk3")
    u = torch.tensor(u0[None], dtype=torch.float64, device="cuda")
    ux, uy = torch.empty_like(u), torch.empty_like(u)
    Fp = torch.zeros_like(u)
    t = 0.0
    for _ in range(nsteps):
        tc = t
        for k in range(3):
            ctx.spectral_op(u, ["DX", "DY"], [ux, uy])
            F = ux + 0.5 * uy
            u = u + dt * (-G[k] * F - Z[k] * Fp)
            Fp = F
            tc += A[k] * dt
            ue = torch.tensor(advection.exact(X, Y, tc), device="cuda")
            u[0, 0, :] = ue[0, :]
            u[0, :, 0] = ue[:, 0]
        t += dt
    ctx.sync()
    return u[0].cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_gaussian_convection_matches_oracle(prec):
    torch = torch_cuda()
    b = binding()
    n, dt, nsteps = 48, 5e-4, 100
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    u0 = advection.exact(X, Y, 0.0)
    ug = _gpu_advect(b, torch, u0, dt, nsteps, prec)
    E = gram_golden(5, 25)
    dx = 1.0 / (n - 1)
    Sx = symbol_closed("DX", "G4", 1.3 * dx, n + 25, n + 25, dx, dx)
    Sy = symbol_closed("DY", "G4", 1.3 * dx, n + 25, n + 25, dx, dx)
    fn = lambda a: [advection.advect(a, Sx, Sy, E, dt, nsteps)]
    uo = fn(u0)[0]
    fl = ulp_floor(fn, u0)[0]
    scale = 1.0 if prec == "f64" else 32.0
    err = rel_l2(ug, uo)
    exact_err = np.sqrt(np.mean((ug - advection.exact(X, Y, dt * nsteps)) ** 2))
    print(f"gaussian convection {prec}: parity {err:.1e} (floor {fl:.1e}), rms error vs exact {exact_err:.1e}")
    assert err < parity_tol(fl, base=1e-12 * scale, factor=10.0 * scale)
    assert exact_err < 1e-3
