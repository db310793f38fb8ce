"""The lid cavity at its parity size over the configured horizon: 64 x 64
particles, walls on all four sides with FC(Gram) d = 5, C = 25 in x and y, G8
with h = 1.3 dx, Re = 1000, dt = 1e-3, 2000 low-storage RK3 steps (t = 2)
from rest, through isph_step on the GPU, against the FP64 oracle's result
after the same 2000 steps (tests/golden/cavity64_rk3_2000.npz, written by
make_cavity64.py, which calls only the oracle).

The bar is the parity rule of the other step tests: relative L2 below
max(1e-12, 10 x floor) for FP64 and 32 times that for FP32 pairs, where the
floor is the oracle's own response to a 1-ulp perturbation of the start
(stored beside the result).  FP32 transforms state their relative L2 and L-inf
against the oracle and are held to the bound measured for them."""
import os

import numpy as np
import pytest

from gpu_common import binding, parity_tol, rel_l2, torch_cuda

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cavity64_rk3_2000.npz")
N = 64


def _golden():
    g = np.load(GOLDEN)
    floors = [rel_l2(g[k + "_ulp"], g[k]) for k in ("u", "v", "phi")]
    return g, floors, int(g["nsteps"])


def _run(prec, nsteps):
    torch = torch_cuda()
    b = binding()
    ctx = b.Context(N, N, 1.0, 1.0, x_walls=True, family="G8", h_over_dx=1.3, prec=prec)
    z = torch.zeros((1, N, N), dtype=torch.float64, device="cuda")
    u, v, p, fu, fv = [z.clone() for _ in range(5)]
    ctx.isph_step(u, v, p, fu, fv, nsteps, nu=1e-3, rho=1.0, dt=1e-3, u_top=1.0, scheme="rk3", use_graph=True)
    ctx.sync()
    return [t[0].cpu().numpy() for t in (u, v, p)]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_cavity_64_rk3_2000_steps_parity(prec):
    g, floors, nsteps = _golden()
    out = _run(prec, nsteps)
    scale = 1.0 if prec == "f64" else 32.0
    errs = [rel_l2(o, g[k]) for o, k in zip(out, ("u", "v", "phi"))]
    linf = [float(np.abs(o - g[k]).max()) for o, k in zip(out, ("u", "v", "phi"))]
    print(f"cavity 64^2 RK3 x{nsteps} {prec}: rel L2 (u, v, phi) {errs}, Linf {linf}, floors {floors}")
    for e, f in zip(errs, floors):
        assert e < parity_tol(f, base=1e-12 * scale, factor=10.0 * scale)


@pytest.mark.gpu
def test_cavity_64_rk3_2000_steps_fp32_error_stated():
    g, floors, nsteps = _golden()
    out = _run("f32", nsteps)
    errs = [rel_l2(o, g[k]) for o, k in zip(out, ("u", "v"))]
    linf = [float(np.abs(o - g[k]).max()) for o, k in zip(out, ("u", "v"))]
    print(f"cavity 64^2 RK3 x{nsteps} f32: rel L2 (u, v) {errs}, Linf {linf}")
    # measured on GB300: rel L2 0.41 (u), 0.91 (v), Linf 0.29, 0.28.  FP32
    # transforms of the lid-corner continuation (~||E||^2 times the data) carry
    # absolute errors of O(1e-1) per substep; the path is not at equal L2 here.
    assert errs[0] < 0.6 and errs[1] < 1.3 and max(linf) < 0.45
