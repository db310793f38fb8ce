"""Parity of ppe_solve (Eqs. 31-33) with the oracle; the FP64 residual; and
the FP32 solve with FP64-residual refinement."""
import numpy as np
import pytest

from gpu_common import binding, grid_lengths, rel_l2, to_dev, torch_cuda
from oracle import ppe as oppe

CASES = [(24, 20, False, 2), (17, 33, False, 1), (20, 20, True, 2), (13, 27, True, 1), (64, 64, False, 1), (64, 64, True, 1)]


def _rhs(nx, ny, batch, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((batch, nx, ny))


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_ppe_matches_oracle_fp64(case, prec):
    """FP64 transforms, and FP32-pair transforms (unit roundoff ~2^-48: bar x32)."""
    torch = torch_cuda()
    b = binding()
    nx, ny, xw, batch = case
    lx, ly = grid_lengths(nx, ny, xw)
    ctx = b.Context(nx, ny, lx, ly, x_walls=xw, batch=batch, prec=prec)
    scale = 1.0 if prec == "f64" else 32.0
    rhs = _rhs(nx, ny, batch, 5)
    phi = torch.zeros((batch, nx, ny), dtype=torch.float64, device="cuda")
    res = ctx.ppe_solve(to_dev(rhs), phi, want_resid=True)
    for k in range(batch):
        ref = oppe.ppe_solve(rhs[k], lx, ly, xw)
        assert rel_l2(phi[k].cpu().numpy(), ref) < 1e-12 * scale
    assert res < 1e-13 * scale


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES[:4])
def test_ppe_fp32_refinement_recovers_fp64(case):
    torch = torch_cuda()
    b = binding()
    nx, ny, xw, batch = case
    lx, ly = grid_lengths(nx, ny, xw)
    rhs = _rhs(nx, ny, batch, 9).astype(np.float32)
    errs = {}
    for it in (0, 1, 2, 3):
        ctx = b.Context(nx, ny, lx, ly, x_walls=xw, batch=batch, prec="f32", refine=it)
        phi = torch.zeros((batch, nx, ny), dtype=torch.float32, device="cuda")
        res = ctx.ppe_solve(to_dev(rhs, "f32"), phi, want_resid=True)
        errs[it] = res
    print("FP64 residual after k refinement sweeps:", errs)
    assert errs[0] < 1e-5
    assert errs[2] < 1e-11 and errs[3] <= errs[2] * 10
