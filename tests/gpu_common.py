"""Helpers for the GPU parity tests: build + load the library, move arrays,
and build the oracle problem that matches a library context."""
import numpy as np
import pytest

from oracle import step as ostep
from tables import gram_golden


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


def binding():
    from paper_2606_06247_gb300 import build
    build.build()
    from paper_2606_06247_gb300 import binding as b
    return b


def to_dev(a, dtype="f64"):
    torch = torch_cuda()
    t = torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if dtype == "f64" else torch.float32)
    return t.cuda()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def grid_lengths(nx, ny, x_walls):
    """Isotropic lattice with walls at y = 0, 1: dy = 1/(ny-1); dx = dy."""
    dy = 1.0 / (ny - 1)
    lx = (nx - 1) * dy if x_walls else nx * dy
    return lx, 1.0


def oracle_problem(nx, ny, x_walls, family, h_over_dx, n_cont=25, **kw):
    E = gram_golden(5, n_cont)
    lx, ly = grid_lengths(nx, ny, x_walls)
    return ostep.Problem(nx=nx, ny=ny, Lx=lx, Ly=ly, x_walls=x_walls, family=family, h_over_dx=h_over_dx,
                         E_dir=E, E_neu=E, **kw).build_symbols()


def ulp_floor(fn, *inputs, seed=0, scale=None):
    """Relative change of fn's outputs when every input value is moved by one
    ulp of its magnitude (or of `scale`, the problem's value scale, when given:
    needed for inputs that are exactly zero), random sign: the FP64 rounding
    floor that any evaluation of the same problem carries.  One per output."""
    rng = np.random.default_rng(seed)
    base = fn(*inputs)
    pert = []
    for a in inputs:
        a = np.asarray(a)
        mag = np.full(a.shape, float(scale)) if scale is not None else np.abs(a)
        pert.append(a + 2.0 ** -52 * mag * rng.choice([-1.0, 1.0], size=a.shape))
    moved = fn(*pert)
    return [rel_l2(m, b) for m, b in zip(moved, base)]


def parity_tol(floor, base=1e-12, factor=10.0):
    """The FP64 parity bar: 1e-12 relative L2, unless the problem's own rounding
    floor (ulp_floor) times `factor` is larger."""
    return max(base, factor * floor)
