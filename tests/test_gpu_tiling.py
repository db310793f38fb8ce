"""Launch-shape selection (fcsph_set_tiling, fcsph_set_cta_threads,
fcsph_autotune): the tiling and the CTA width only change which CTA and which
thread carry which line and butterfly, never the arithmetic of a line, so
every launch shape gives bitwise the same results; the autotuner keeps a
valid shape and leaves the caller's state alone."""
import numpy as np
import pytest

from gpu_common import binding, grid_lengths, to_dev, torch_cuda
from paper_2606_06247_gb300 import inputs

TILINGS = [(1, 1), (2, 2), (4, 1), (1, 4), (2, 1), (4, 8)]
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
    assert r in (1, 2, 4) and c in (1, 2, 4, 8) and ms > 0
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


WIDTHS = [(32, 32), (64, 128), (128, 64), (64, 64), (128, 128)]


def _same_across_widths(ctx, run):
    ref = None
    for w in WIDTHS:
        ctx.set_cta_threads(*w)
        assert ctx.get_cta_threads() == w
        out = run()
        if ref is None:
            ref = out
        else:
            for a, r in zip(out, ref):
                np.testing.assert_array_equal(a, r, err_msg=f"widths {w}")


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f32", "f32x2", "f64"])
@pytest.mark.parametrize("nx,ny,x_walls", [(37, 30, True), (64, 256, False), (40, 512, False)])
def test_every_cta_width_gives_the_same_results(nx, ny, x_walls, prec):
    """Operators, line operator, pressure solve and RK3 steps: bitwise equal
    for every pair of CTA widths, in every precision.  The lengths cover a
    direct plan (55 = 5 * 11), Rader (281) and Bluestein (537) columns."""
    torch = torch_cuda()
    b = binding()
    batch = 2
    lx, ly = grid_lengths(nx, ny, x_walls)
    fam = "G8" if x_walls else "G4"
    ctx = b.Context(nx, ny, lx, ly, x_walls=x_walls, batch=batch, family=fam, h_over_dx=1.3, prec=prec)
    rng = np.random.default_rng(5)
    dt = torch.float32 if prec == "f32" else torch.float64
    f = torch.tensor(rng.standard_normal((batch, nx, ny)), dtype=dt, device="cuda")
    rhs = f - f.mean(dim=(1, 2), keepdim=True)

    def ops():
        outs = [torch.empty_like(f) for _ in range(4)]
        ctx.spectral_op(f, ["W", "DX", "DY", "LAP"], outs)
        lo = [torch.empty_like(f) for _ in range(2)]
        ctx.line_op(f, ["DY", "LAP"], lo)
        phi = torch.empty_like(f)
        ctx.ppe_solve(rhs, phi)
        ctx.sync()
        return [x.cpu().numpy() for x in outs + lo + [phi]]

    _same_across_widths(ctx, ops)
    prm = dict(CAVITY) if x_walls else dict(nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0), scheme="rk3")

    def steps():
        st = _state(torch, nx, ny, batch, 7)
        ctx.isph_step(*st, 2, use_graph=True, **prm)
        ctx.sync()
        return [x.cpu().numpy() for x in st]

    _same_across_widths(ctx, steps)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f32", "f32x2", "f64"])
def test_every_cta_width_gives_the_same_3d_step(prec):
    torch = torch_cuda()
    b = binding()
    nx, nz, ny = 8, 6, 20
    dy = 1.0 / (ny - 1)
    ctx = b.Context(nx, ny, nx * dy, 1.0, family="G4", h_over_dx=1.3, prec=prec, nz=nz, lz=nz * dy)
    rng = np.random.default_rng(9)
    init = [1e-3 * rng.standard_normal((1, nx, nz, ny)) for _ in range(3)]

    def steps():
        u, v, w = (to_dev(a) for a in init)
        p, fu, fv, fw = (torch.zeros_like(u) for _ in range(4))
        ctx.isph_step(u, v, p, fu, fv, 2, w=w, fw=fw, nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0, 0.1), scheme="rk3")
        ctx.sync()
        return [x.cpu().numpy() for x in (u, v, w, p)]

    _same_across_widths(ctx, steps)


@pytest.mark.gpu
def test_cta_widths_are_checked():
    """Defaults: 4-warp CTAs for passes that fill at most a quarter of the GPU
    with one-warp CTAs, 2-warp for at most half; long FP32 lines at least 64
    (row) and 128 (column); FP64 / FP32x2 passes whose shared memory fits
    fewer than 12 one-warp CTAs per SM the narrowest width reaching 12 warps."""
    torch_cuda()
    b = binding()
    for prec in ("f64", "f32x2", "f32"):
        small = b.Context(64, 64, 64 / 63, 1.0, batch=1, prec=prec)  # 32 column pairs, 45 rows
        assert small.get_cta_threads() == (128, 128)
        full = b.Context(256, 256, 1.0, 1.0, x_walls=True, batch=32, prec=prec)  # 4096 pairs, 4512 rows
        assert full.get_cta_threads() == (32, 32)
        mid = b.Context(256, 256, 1.0, 1.0, x_walls=True, batch=6, prec=prec)  # 768 pairs, 846 rows
        assert mid.get_cta_threads() == (64, 64)
        for bad in [(0, 32), (32, 96), (256, 32)]:
            with pytest.raises(b.FcsphError) as e:
                small.set_cta_threads(*bad)
            assert e.value.status == 1
        small.set_cta_threads(64, 32)
        assert small.get_cta_threads() == (64, 32)
    big = b.Context(1024, 1024, 1024 / 1023, 1.0, batch=1, prec="f32")
    assert big.get_cta_threads() == (64, 128)      # FP32, lines of >= 768 points
    # FP32-pair 540-point lines: a row CTA holds 4 lines (~35 KB), 6 fit an SM, so 2 warps reach 12; a
    # column pair holds 2 (~17 KB, its FP64 values stay in global memory), 13 fit, so one warp does
    long = b.Context(512, 512, 1.0, 1.0, x_walls=True, batch=32, n_cont=28, prec="f32x2")
    assert long.get_cta_threads() == (64, 32)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32x2", "f32"])
def test_step_groups_give_the_same_step(prec):
    """fcsph_set_step_groups splits the batch into groups whose kernels run as
    parallel branches of the step graph; every instance's arithmetic is that
    of the single chain, so the state after the steps is bitwise the same, for
    groups of unequal size (5 instances in 2 or 3 groups) and with an instance
    masked out."""
    torch = torch_cuda()
    b = binding()
    nx, ny, batch = 37, 30, 5
    lx, ly = grid_lengths(nx, ny, True)
    ctx = b.Context(nx, ny, lx, ly, x_walls=True, batch=batch, family="G8", h_over_dx=1.3, prec=prec)
    active = torch.tensor([1, 1, 0, 1, 1], dtype=torch.uint8, device="cuda")
    for mask in (None, active):
        ref = None
        for groups in (1, 2, 3, 5, 8):
            ctx.set_step_groups(groups)
            assert ctx.get_step_groups() == groups
            st = _state(torch, nx, ny, batch, 21)
            ctx.isph_step(*st, 2, use_graph=True, active=mask, **CAVITY)
            ctx.sync()
            out = [x.cpu().numpy() for x in st]
            if ref is None:
                ref = out
            else:
                for a, r in zip(out, ref):
                    np.testing.assert_array_equal(a, r, err_msg=f"groups {groups}")
        if mask is not None:
            init = [x.cpu().numpy() for x in _state(torch, nx, ny, batch, 21)]
            for a, r in zip(ref, init):
                np.testing.assert_array_equal(a[2], r[2])  # the masked instance is untouched
    with pytest.raises(b.FcsphError) as e:
        ctx.set_step_groups(0)
    assert e.value.status == 1


@pytest.mark.gpu
def test_step_groups_in_3d():
    torch = torch_cuda()
    b = binding()
    nx, ny, nz, batch = 16, 20, 8, 3
    dy = 1.0 / (ny - 1)
    ctx = b.Context(nx, ny, nx * dy, 1.0, batch=batch, family="G4", h_over_dx=1.3, prec="f32x2", nz=nz, lz=nz * dy)
    ref = None
    for groups in (1, 2, 3):
        ctx.set_step_groups(groups)
        st = [torch.zeros((batch, nx * nz, ny), dtype=torch.float64, device="cuda") for _ in range(7)]
        g0 = np.random.default_rng(9)
        for k in range(3):
            st[k].copy_(torch.tensor(1e-3 * g0.standard_normal((batch, nx * nz, ny))))
            st[k][:, :, 0] = 0
            st[k][:, :, -1] = 0
        u, v, w, p, fu, fv, fw = st
        ctx.isph_step(u, v, p, fu, fv, 2, nu=0.01, rho=1.0, dt=1e-3, force=(0.08, 0.0, 0.0), scheme="rk3",
                      use_graph=True, w=w, fw=fw)
        ctx.sync()
        out = [x.cpu().numpy() for x in (u, v, w, p)]
        if ref is None:
            ref = out
        else:
            for a, r in zip(out, ref):
                np.testing.assert_array_equal(a, r, err_msg=f"groups {groups}")
