"""Run-to-run determinism: the kernels of the step and of the operators fix
their arithmetic order (no atomic sums, round-to-nearest intrinsics where a
compiler could contract), so the same call on the same inputs gives bitwise
the same result — for each precision, with the step graph split into instance groups,
as one persistent launch per step, with NVTX tracing on, and for the FP32
plane operator with and without its bulk-copy staging."""
import numpy as np
import pytest

from gpu_common import binding, grid_lengths, to_dev, torch_cuda
from paper_2606_06247_gb300 import inputs

CAVITY = dict(nu=1e-3, rho=1.0, dt=1e-3, u_top=1.0, scheme="rk3")


def _state(torch, nx, ny, batch, seed):
    us, vs = [], []
    for k in range(batch):
        u0, v0 = inputs.cavity_initial(nx, ny, seed=seed + k, sigma=1e-3)
        us.append(u0)
        vs.append(v0)
    u, v = to_dev(np.stack(us)), to_dev(np.stack(vs))
    return [u, v, torch.zeros_like(u), torch.zeros_like(u), torch.zeros_like(u)]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32x2", "f32"])
def test_steps_are_deterministic_in_every_launch_mode(prec):
    torch = torch_cuda()
    b = binding()
    nx, ny, batch = 48, 40, 6
    lx, ly = grid_lengths(nx, ny, True)
    modes = [dict(), dict(groups=3), dict(trace=True)]
    if prec != "f32":
        modes.append(dict(persistent=True))
    ref = None
    for mode in modes:
        for rep in range(2):
            ctx = b.Context(nx, ny, lx, ly, x_walls=True, batch=batch, family="G8", h_over_dx=1.3, prec=prec)
            if "groups" in mode:
                ctx.set_step_groups(mode["groups"])
            if mode.get("persistent"):
                ctx.set_step_persistent(True)
            if mode.get("trace"):
                ctx.set_tracing(True)
            st = _state(torch, nx, ny, batch, 41)
            ctx.isph_step(*st, 3, use_graph=True, **CAVITY)
            ctx.sync()
            out = [x.cpu().numpy() for x in st]
            if ref is None:
                ref = out
            else:
                for a, r in zip(out, ref):
                    np.testing.assert_array_equal(a, r, err_msg=f"{mode} run {rep}")


@pytest.mark.gpu
def test_plane_operator_is_deterministic():
    torch = torch_cuda()
    b = binding()
    nx, ny, batch = 64, 1024, 4
    lx, ly = grid_lengths(nx, ny, False)
    ctx = b.Context(nx, ny, lx, ly, batch=batch, n_cont=26, family="G4", h_over_dx=1.3, prec="f32")
    f = torch.tensor(np.stack([inputs.smooth_field(nx, ny, seed=k) for k in range(batch)]), dtype=torch.float32,
                     device="cuda")
    ref = None
    for tma in (True, True, False, False):
        ctx.set_tma(tma)
        outs = [torch.empty_like(f) for _ in range(3)]
        ctx.spectral_op(f, ["DX", "DY", "LAP"], outs)
        ctx.sync()
        got = [o.cpu().numpy() for o in outs]
        if ref is None:
            ref = got
        else:
            for a, r in zip(got, ref):
                np.testing.assert_array_equal(a, r)
