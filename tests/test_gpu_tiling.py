"""Launch-shape selection (fcsph_set_tiling, fcsph_autotune): the tiling only
changes which CTA carries which line, never the arithmetic of a line, so every
tiling gives bitwise the same step; the autotuner keeps a valid tiling and
leaves the caller's state alone."""
import numpy as np
import pytest

from gpu_common import binding, grid_lengths, to_dev, torch_cuda
from paper_2606_06247_gb300 import inputs

TILINGS = [(1, 1), (2, 2), (4, 1), (1, 4), (2, 1)]
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
def test_every_tiling_gives_the_same_step(prec):
    torch = torch_cuda()
    b = binding()
    nx, ny, batch = 37, 30, 3  # odd nx: a ragged last column pair; ny + 25 = 55 = 5 * 11
    lx, ly = grid_lengths(nx, ny, True)
    ctx = b.Context(nx, ny, lx, ly, x_walls=True, batch=batch, family="G8", h_over_dx=1.3, prec=prec)
    ref = None
    for t in TILINGS:
        ctx.set_tiling(*t)
        assert ctx.get_tiling() == t
        st = _state(torch, nx, ny, batch, 11)
        ctx.isph_step(*st, 2, use_graph=True, **CAVITY)
        ctx.sync()
        out = [x.cpu().numpy() for x in st]
        if ref is None:
            ref = out
        else:
            for a, r in zip(out, ref):
                np.testing.assert_array_equal(a, r)


@pytest.mark.gpu
def test_autotune_keeps_a_valid_tiling_and_leaves_the_state():
    torch = torch_cuda()
    b = binding()
    nx = ny = 48
    lx, ly = grid_lengths(nx, ny, True)
    ctx = b.Context(nx, ny, lx, ly, x_walls=True, batch=2, family="G8", h_over_dx=1.3, prec="f32x2")
    st = _state(torch, nx, ny, 2, 3)
    before = [x.clone() for x in st]
    r, c, ms = ctx.autotune(steps=2, **CAVITY)
    assert r in (1, 2, 4) and c in (1, 2, 4) and ms > 0
    for x, y in zip(st, before):
        assert torch.equal(x, y)
    ctx.isph_step(*st, 1, use_graph=True, **CAVITY)
    ctx.sync()
    assert all(torch.isfinite(x).all() for x in st)


@pytest.mark.gpu
def test_set_tiling_rejects_bad_shapes():
    torch_cuda()
    b = binding()
    ctx = b.Context(32, 32, 32 / 31, 1.0, batch=1)
    for bad in [(0, 1), (1, 0), (9, 1), (1, 9)]:
        with pytest.raises(b.FcsphError) as e:
            ctx.set_tiling(*bad)
        assert e.value.status == 1
    # 8 column pairs of 1024-point PPE lines exceed one CTA's shared memory
    big = b.Context(1024, 1024, 1.0, 1.0, x_walls=True, batch=1)
    with pytest.raises(b.FcsphError) as e:
        big.set_tiling(1, 8)
    assert e.value.status == 6
