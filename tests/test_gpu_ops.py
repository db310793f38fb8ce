"""Parity of fc_extend, spectral_op and spectral_div (CUDA, through the C ABI)
with the FP64 oracle, on seeded fields.  Sizes span several CTA tiles and
leave ragged tails (odd nx -> an unpaired column; hy not a multiple of the
rows per CTA)."""
import numpy as np
import pytest

from gpu_common import binding, grid_lengths, oracle_problem, parity_tol, rel_l2, to_dev, torch_cuda, ulp_floor
from oracle import fc as ofc
from oracle import ops as oops
from paper_2606_06247_gb300 import inputs
from tables import gram_golden

CASES = [  # nx, ny, x_walls, family, h/dx, batch
    (24, 20, False, "G4", 1.3, 2),
    (17, 33, False, "G8", 2.0, 3),
    (20, 20, True, "G8", 1.3, 2),
    (13, 27, True, "G4", 1.3, 1),
    (64, 64, False, "G4", 1.3, 1),
]

TOL64 = 1e-12


def _fields(nx, ny, batch, seed):
    return np.stack([inputs.smooth_field(nx, ny, seed=seed + k) for k in range(batch)])


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
def test_fc_extend_matches_oracle(case):
    torch_cuda()
    b = binding()
    nx, ny, xw, fam, hdx, batch = case
    lx, ly = grid_lengths(nx, ny, xw)
    ctx = b.Context(nx, ny, lx, ly, x_walls=xw, batch=batch, family=fam, h_over_dx=hdx)
    f = _fields(nx, ny, batch, 1)
    mx = nx + 25 if xw else nx
    out = to_dev(np.zeros((batch, mx, ny + 25)))
    ctx.fc_extend(to_dev(f), out)
    ctx.sync()
    E = gram_golden(5, 25)
    for k in range(batch):
        ref = ofc.extend2d(f[k], E, E if xw else None)
        assert np.abs(out[k].cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_spectral_op_matches_oracle_fp64(case, bc, prec):
    """FP64 transforms, and FP32-pair transforms (unit roundoff ~2^-48: bar x32)."""
    torch = torch_cuda()
    b = binding()
    nx, ny, xw, fam, hdx, batch = case
    lx, ly = grid_lengths(nx, ny, xw)
    ctx = b.Context(nx, ny, lx, ly, x_walls=xw, batch=batch, family=fam, h_over_dx=hdx, prec=prec)
    scale = 1.0 if prec == "f64" else 32.0
    p = oracle_problem(nx, ny, xw, fam, hdx)
    from oracle.symbols import symbol_closed
    mx, my = p.extended_shape()
    S = {op: symbol_closed(op, fam, p.h, mx, my, p.dx, p.dy) for op in ("W", "DX", "DY", "LAP")}
    f = _fields(nx, ny, batch, 7)
    names = ["W", "DX", "DY", "LAP"]
    outs = [torch.zeros((batch, nx, ny), dtype=torch.float64, device="cuda") for _ in names]
    ctx.spectral_op(to_dev(f), names, outs, bc=bc)
    ctx.sync()
    E = p.E_dir
    fn = lambda x: oops.apply_symbols(x, [S[n] for n in names], E, E if xw else None)
    for k in range(batch):
        refs = fn(f[k])
        floors = ulp_floor(fn, f[k])
        for n, o, r, fl in zip(names, outs, refs, floors):
            err = rel_l2(o[k].cpu().numpy(), r)
            assert err < parity_tol(fl, base=1e-12 * scale, factor=10.0 * scale), (n, k, err, fl)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES[:3])
def test_spectral_op_fp32_error_is_reported_and_small(case):
    torch = torch_cuda()
    b = binding()
    nx, ny, xw, fam, hdx, batch = case
    lx, ly = grid_lengths(nx, ny, xw)
    ctx = b.Context(nx, ny, lx, ly, x_walls=xw, batch=batch, family=fam, h_over_dx=hdx, prec="f32")
    p = oracle_problem(nx, ny, xw, fam, hdx)
    f = _fields(nx, ny, batch, 11)
    outs = [torch.zeros((batch, nx, ny), dtype=torch.float32, device="cuda") for _ in range(3)]
    ctx.spectral_op(to_dev(f, "f32"), ["DX", "DY", "LAP"], outs)
    ctx.sync()
    refs = oops.apply_symbols(f[0].astype(np.float32).astype(np.float64), [p.sym["DX"], p.sym["DY"], p.sym["LAP"]],
                              p.E_dir, p.E_dir if xw else None)
    errs = [rel_l2(o[0].cpu().numpy(), r) for o, r in zip(outs, refs)]
    print("fp32 spectral_op rel L2 vs FP64 oracle:", errs)
    # FP32 rounding of the FC-extended line (continuation values up to ~1e2 |f|)
    # seen through a derivative (k_max ~ pi/dy): ~1e3 eps_f32
    assert max(errs) < 5e-4


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES[:4])
def test_spectral_div_matches_oracle(case):
    torch = torch_cuda()
    b = binding()
    nx, ny, xw, fam, hdx, batch = case
    lx, ly = grid_lengths(nx, ny, xw)
    ctx = b.Context(nx, ny, lx, ly, x_walls=xw, batch=batch, family=fam, h_over_dx=hdx)
    p = oracle_problem(nx, ny, xw, fam, hdx)
    fx = _fields(nx, ny, batch, 21)
    fy = _fields(nx, ny, batch, 31)
    out = torch.zeros((batch, nx, ny), dtype=torch.float64, device="cuda")
    ctx.spectral_div(to_dev(fx), to_dev(fy), out)
    ctx.sync()
    fn = lambda a, c: [oops.divergence(a, c, p.sym["DX"], p.sym["DY"], p.E_dir, p.E_dir if xw else None)]
    for k in range(batch):
        ref = fn(fx[k], fy[k])[0]
        fl = ulp_floor(fn, fx[k], fy[k])[0]
        assert rel_l2(out[k].cpu().numpy(), ref) < parity_tol(fl)


@pytest.mark.gpu
def test_caller_table_is_used():
    torch = torch_cuda()
    b = binding()
    nx, ny = 16, 18
    lx, ly = grid_lengths(nx, ny, False)
    E = ofc.paper_table(5, 25, 3)
    ctx = b.Context(nx, ny, lx, ly, table_dir=E, table_neu=E)
    np.testing.assert_array_equal(ctx.get_fc_table(0), E)
    f = _fields(nx, ny, 1, 3)
    out = to_dev(np.zeros((1, nx, ny + 25)))
    ctx.fc_extend(to_dev(f), out)
    ctx.sync()
    ref = ofc.extend_last_axis(f[0], E)
    assert np.abs(out[0].cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
