"""isph_step's instance mask (fcsph_step_params.active): instances whose flag
is 0 are neither read nor written, the others advance bitwise as in a step of
the whole batch, and the mask may change between replays of the captured
graph (serving keeps empty slots in a batch this way)."""
import numpy as np
import pytest

from gpu_common import binding, grid_lengths, to_dev, torch_cuda
from paper_2606_06247_gb300 import inputs

CAVITY = dict(nu=1e-3, rho=1.0, dt=1e-3, u_top=1.0, scheme="rk3")


def _init(nx, ny, batch, seed):
    us, vs = zip(*[inputs.cavity_initial(nx, ny, seed=seed + k, sigma=1e-3) for k in range(batch)])
    return np.stack(us), np.stack(vs)


def _state(torch, u0, v0):
    u, v = to_dev(u0), to_dev(v0)
    return [u, v, torch.zeros_like(u), torch.zeros_like(u), torch.zeros_like(u)]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32x2", "f32"])
def test_masked_instances_are_left_alone_and_the_rest_match(prec):
    torch = torch_cuda()
    b = binding()
    nx, ny, batch = 36, 30, 4
    lx, ly = grid_lengths(nx, ny, True)
    ctx = b.Context(nx, ny, lx, ly, x_walls=True, batch=batch, family="G8", h_over_dx=1.3, prec=prec)
    u0, v0 = _init(nx, ny, batch, 21)
    full = _state(torch, u0, v0)
    ctx.isph_step(*full, 3, use_graph=True, **CAVITY)
    ctx.sync()
    full = [x.cpu().numpy() for x in full]

    st = _state(torch, u0, v0)
    before = [x.cpu().numpy() for x in st]
    mask = torch.tensor([1, 0, 1, 0], dtype=torch.uint8, device="cuda")
    ctx.isph_step(*st, 3, use_graph=True, active=mask, **CAVITY)
    ctx.sync()
    mid = [x.cpu().numpy() for x in st]
    for got, ref, old in zip(mid, full, before):
        np.testing.assert_array_equal(got[[0, 2]], ref[[0, 2]])
        np.testing.assert_array_equal(got[[1, 3]], old[[1, 3]])
    # the same graph with the mask flipped: the other two catch up
    mask.copy_(torch.tensor([0, 1, 0, 1], dtype=torch.uint8))
    ctx.isph_step(*st, 3, use_graph=True, active=mask, **CAVITY)
    ctx.sync()
    end = [x.cpu().numpy() for x in st]
    for got, ref, m in zip(end, full, mid):
        np.testing.assert_array_equal(got[[1, 3]], ref[[1, 3]])
        np.testing.assert_array_equal(got[[0, 2]], m[[0, 2]])
    # eager launches honour the mask as well
    mask.fill_(0)
    ctx.isph_step(*st, 1, use_graph=False, active=mask, **CAVITY)
    ctx.sync()
    for got, m in zip(st, end):
        np.testing.assert_array_equal(got.cpu().numpy(), m)


@pytest.mark.gpu
def test_mask_in_3d():
    torch = torch_cuda()
    b = binding()
    nx, nz, ny, batch = 8, 6, 20, 3
    dy = 1.0 / (ny - 1)
    ctx = b.Context(nx, ny, nx * dy, 1.0, batch=batch, family="G4", h_over_dx=1.3, prec="f32x2", nz=nz, lz=nz * dy)
    rng = np.random.default_rng(4)
    init = [1e-3 * rng.standard_normal((batch, nx, nz, ny)) for _ in range(3)]
    prm = dict(nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0, 0.1), scheme="rk3")

    def run(active):
        u, v, w = (to_dev(a) for a in init)
        p, fu, fv, fw = (torch.zeros_like(u) for _ in range(4))
        ctx.isph_step(u, v, p, fu, fv, 2, w=w, fw=fw, active=active, **prm)
        ctx.sync()
        return [x.cpu().numpy() for x in (u, v, w, p)]

    full = run(None)
    part = run(torch.tensor([0, 1, 0], dtype=torch.uint8, device="cuda"))
    for got, ref, a in zip(part, full, init + [np.zeros_like(init[0])]):
        np.testing.assert_array_equal(got[1], ref[1])
        np.testing.assert_array_equal(got[[0, 2]], a[[0, 2]])


@pytest.mark.gpu
def test_mask_is_refused_with_fp32_refinement():
    torch = torch_cuda()
    b = binding()
    ctx = b.Context(32, 32, 1.0, 1.0, x_walls=True, batch=2, prec="f32", refine=1)
    st = _state(torch, *_init(32, 32, 2, 3))
    with pytest.raises(b.FcsphError) as e:
        ctx.isph_step(*st, 1, active=torch.ones(2, dtype=torch.uint8, device="cuda"), **CAVITY)
    assert e.value.status == 6
