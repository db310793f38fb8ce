"""The register-resident x pass of FP32 contexts (periodic x lines of 32 M
points, M = 2 .. 32: one warp per 32 / M rows, fcsph_warpfft.cuh) against the
FP64 oracle: spectral_op at every M with a ragged last CTA of rows,
two-input row passes (spectral_div, spectral_project), a channel RK3 step,
and a 3D channel step against the FP64 path."""
import numpy as np
import pytest

from gpu_common import binding, grid_lengths, oracle_problem, rel_l2, to_dev, torch_cuda
from oracle import ops as oops
from oracle import ppe as oppe
from oracle import step as ostep
from paper_2606_06247_gb300 import inputs


def _fields(nx, ny, batch, seed):
    return np.stack([inputs.smooth_field(nx, ny, seed=seed + k) for k in range(batch)])


@pytest.mark.gpu
@pytest.mark.parametrize("nx", [64, 128, 256, 512, 1024])
def test_fp32_register_rows_spectral_op(nx):
    torch = torch_cuda()
    b = binding()
    ny, batch = 20, 2   # 23 spectrum rows: the last CTA of rows is partly empty
    lx, ly = grid_lengths(nx, ny, False)
    ctx = b.Context(nx, ny, lx, ly, batch=batch, family="G4", h_over_dx=1.3, prec="f32")
    p = oracle_problem(nx, ny, False, "G4", 1.3)
    from oracle.symbols import symbol_closed
    mx, my = p.extended_shape()
    names = ["W", "DX", "DY", "LAP"]
    S = [symbol_closed(op, "G4", p.h, mx, my, p.dx, p.dy) for op in names]
    f = _fields(nx, ny, batch, 3)
    outs = [torch.zeros((batch, nx, ny), dtype=torch.float32, device="cuda") for _ in names]
    ctx.spectral_op(to_dev(f, "f32"), names, outs)
    ctx.sync()
    worst = 0.0
    for k in range(batch):
        refs = oops.apply_symbols(f[k].astype(np.float32).astype(np.float64), S, p.E_dir)
        for n, o, r in zip(names, outs, refs):
            worst = max(worst, rel_l2(o[k].double().cpu().numpy(), r))
    print(f"register rows nx={nx}: worst FP32 rel L2 vs FP64 oracle {worst:.2e}")
    assert worst < 1e-4


@pytest.mark.gpu
def test_fp32_register_rows_two_inputs():
    torch = torch_cuda()
    b = binding()
    nx, ny = 256, 24
    lx, ly = grid_lengths(nx, ny, False)
    ctx = b.Context(nx, ny, lx, ly, batch=1, family="G4", h_over_dx=1.3, prec="f32")
    p = oracle_problem(nx, ny, False, "G4", 1.3)
    fx, fy = _fields(nx, ny, 1, 21), _fields(nx, ny, 1, 31)
    div = torch.zeros((1, nx, ny), dtype=torch.float32, device="cuda")
    ctx.spectral_div(to_dev(fx, "f32"), to_dev(fy, "f32"), div)
    ox, oy = torch.zeros_like(div), torch.zeros_like(div)
    ctx.spectral_project(to_dev(fx, "f32"), to_dev(fy, "f32"), ox, oy)
    ctx.sync()
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    ref = oops.divergence(r32(fx[0]), r32(fy[0]), p.sym["DX"], p.sym["DY"], p.E_dir)
    e_div = rel_l2(div[0].double().cpu().numpy(), ref)
    rx, ry = oppe.extended_projection(r32(fx[0]), r32(fy[0]), p.sym["DX"], p.sym["DY"], p.E_dir)
    e_proj = max(rel_l2(ox[0].double().cpu().numpy(), rx), rel_l2(oy[0].double().cpu().numpy(), ry))
    print(f"register rows, two inputs: divergence {e_div:.2e}, projection {e_proj:.2e}")
    assert e_div < 1e-4 and e_proj < 1e-4


@pytest.mark.gpu
def test_fp32_register_rows_channel_step():
    torch = torch_cuda()
    b = binding()
    nx, ny = 128, 24
    lx, ly = grid_lengths(nx, ny, False)
    u0, v0 = inputs.channel_initial(nx, ny, seed=1, sigma=1e-3)
    prm = dict(nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0))
    ctx = b.Context(nx, ny, lx, ly, family="G4", h_over_dx=1.3, prec="f32")
    u, v = to_dev(u0[None]), to_dev(v0[None])
    p, fu, fv = torch.zeros_like(u), torch.zeros_like(u), torch.zeros_like(u)
    ctx.isph_step(u, v, p, fu, fv, 3, scheme="rk3", **prm)
    ctx.sync()
    prob = oracle_problem(nx, ny, False, "G4", 1.3, scheme="rk3", **prm)
    uo, vo, _ = ostep.isph_steps(prob, u0, v0, 3)
    eu, ev = rel_l2(u[0].cpu().numpy(), uo), rel_l2(v[0].cpu().numpy(), vo)
    print(f"register rows, channel {nx}x{ny} RK3 x3: FP32 rel L2 u {eu:.2e} v {ev:.2e}")
    assert eu < 5e-4 and ev < 1e-2


@pytest.mark.gpu
def test_fp32_register_rows_3d_channel_step():
    torch = torch_cuda()
    b = binding()
    nx, nz, ny = 64, 6, 16
    dy = 1.0 / (ny - 1)
    rng = np.random.default_rng(9)
    init = [1e-3 * rng.standard_normal((1, nx, nz, ny)) for _ in range(3)]
    res = {}
    for prec in ("f64", "f32"):
        ctx = b.Context(nx, ny, nx * dy, 1.0, family="G4", h_over_dx=1.3, prec=prec, nz=nz, lz=nz * dy)
        u, v, w = (to_dev(a) for a in init)
        p, fu, fv, fw = (torch.zeros_like(u) for _ in range(4))
        ctx.isph_step(u, v, p, fu, fv, 2, w=w, fw=fw, nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0, 0.1), scheme="rk3")
        ctx.sync()
        res[prec] = [x.cpu().numpy() for x in (u, v, w)]
    errs = [rel_l2(a, r) for a, r in zip(res["f32"], res["f64"])]
    print("register rows, 3D channel RK3 x2: FP32 vs FP64 rel L2 (u, v, w)", errs)
    assert max(errs) < 5e-4


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny,n_cont", [(16, 1024, 26), (15, 512, 28), (64, 512, 28),
                                         (16, 1024, 25), (15, 512, 25), (64, 512, 25)])
def test_fp32_register_columns_spectral_op(nx, ny, n_cont):
    """The register column FFT of FP32 contexts (fcsph_regfft.cuh: 1050 = 30 x 35
    and 540 = 20 x 27 extended points, and Bluestein's convolution on the team
    FFT for 1049 (m = 2100 = 42 x 50) and 537 (m = 1080 = 30 x 36)): forward
    pass with FC and inverse pass into FP32 outputs, against the FP64 oracle;
    an odd nx leaves the last column pair half empty."""
    torch = torch_cuda()
    b = binding()
    batch = 2
    lx, ly = grid_lengths(nx, ny, False)
    ctx = b.Context(nx, ny, lx, ly, batch=batch, n_cont=n_cont, family="G4", h_over_dx=1.3, prec="f32")
    p = oracle_problem(nx, ny, False, "G4", 1.3, n_cont=n_cont)
    from oracle.symbols import symbol_closed
    mx, my = p.extended_shape()
    names = ["W", "DX", "DY", "LAP"]
    S = [symbol_closed(op, "G4", p.h, mx, my, p.dx, p.dy) for op in names]
    f = _fields(nx, ny, batch, 5)
    outs = [torch.zeros((batch, nx, ny), dtype=torch.float32, device="cuda") for _ in names]
    ctx.spectral_op(to_dev(f, "f32"), names, outs)
    div = torch.zeros((batch, nx, ny), dtype=torch.float32, device="cuda")
    ctx.spectral_div(to_dev(f, "f32"), to_dev(f[:, ::-1].copy(), "f32"), div)
    ctx.sync()
    worst = 0.0
    for k in range(batch):
        fk = f[k].astype(np.float32).astype(np.float64)
        refs = oops.apply_symbols(fk, S, p.E_dir)
        for o, r in zip(outs, refs):
            worst = max(worst, rel_l2(o[k].double().cpu().numpy(), r))
        rd = oops.divergence(fk, fk[::-1].copy(), S[1], S[2], p.E_dir)
        worst = max(worst, rel_l2(div[k].double().cpu().numpy(), rd))
    print(f"register columns {nx}x{ny} C={n_cont}: worst FP32 rel L2 vs FP64 oracle {worst:.2e}")
    assert worst < 2e-4


@pytest.mark.gpu
@pytest.mark.parametrize("ny,n_cont", [(1024, 26), (512, 28), (1024, 25), (512, 25)])
def test_fp32_register_line_op(ny, n_cont):
    """line_op of FP32 contexts on the register team FFT (1050 and 540 extended
    points directly, 1049 and 537 by Bluestein's convolution on it), an odd
    number of lines, against the FP64 oracle."""
    torch = torch_cuda()
    b = binding()
    from oracle.symbols import symbol_closed
    from tables import gram_golden
    nl = 5
    dy = 1.0 / (ny - 1)
    ctx = b.Context(nl, ny, nl * dy, 1.0, batch=1, n_cont=n_cont, family="G4", h_over_dx=1.3, prec="f32")
    f = inputs.band_limited_lines(nl, ny, seed=3, n_modes=32).reshape(1, nl, ny)
    names = ["W", "DY", "LAP"]
    outs = [torch.zeros((1, nl, ny), dtype=torch.float32, device="cuda") for _ in names]
    ctx.line_op(to_dev(f, "f32"), names, outs)
    ctx.sync()
    E = gram_golden(5, n_cont)
    S = [symbol_closed(op, "G4", 1.3 * dy, 1, ny + n_cont, 1.0, dy) for op in names]
    worst = 0.0
    for i in range(nl):
        refs = oops.apply_symbols(f[0, i].astype(np.float32).astype(np.float64)[None, :], S, E)
        for o, r in zip(outs, refs):
            worst = max(worst, rel_l2(o[0, i].double().cpu().numpy(), r[0]))
    print(f"register line_op ny={ny} C={n_cont}: worst FP32 rel L2 {worst:.2e}")
    # Bluestein lengths run two FP32 transforms of length m ~ 2n plus two chirp
    # products per transform: about twice the rounding of a direct transform
    # (measured 1.3e-4 at 1049 points, under 1e-4 at the direct lengths)
    assert worst < (2e-4 if n_cont == 25 else 1e-4)


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny,n_cont,batch", [(128, 512, 28, 24), (40, 1024, 26, 3), (128, 512, 25, 24),
                                               (40, 1024, 25, 3)])
def test_fp32_register_columns_tma_staging_is_exact(nx, ny, n_cont, batch):
    """The output column pass with its half-spectrum rows staged by 2D bulk
    tensor copies (fcsph_set_tma, the default) gives bitwise the outputs of the
    per-thread loads, for one to several outputs and, at 128 x 24 column pairs
    of 512 nodes, more column pairs than resident CTAs (each CTA then stages
    the next pair while it transforms the current one)."""
    torch = torch_cuda()
    b = binding()
    lx, ly = grid_lengths(nx, ny, False)
    ctx = b.Context(nx, ny, lx, ly, batch=batch, n_cont=n_cont, family="G4", h_over_dx=1.3, prec="f32")
    f = to_dev(_fields(nx, ny, batch, 9), "f32")
    names = ["W", "DX", "DY", "LAP"]
    res = []
    for tma in (True, False):
        ctx.set_tma(tma)
        outs = [torch.zeros((batch, nx, ny), dtype=torch.float32, device="cuda") for _ in names]
        ctx.spectral_op(f, names, outs)
        div = torch.zeros((batch, nx, ny), dtype=torch.float32, device="cuda")
        ctx.spectral_div(f, f.flip(1).contiguous(), div)
        ctx.sync()
        res.append([o.cpu().numpy() for o in outs + [div]])
    for a, r in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, r)
