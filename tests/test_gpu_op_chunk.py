"""spectral_op chunk by chunk of instances (fcsph_set_op_chunk): the passes
take each chunk as an instance offset and count, so every chunk size gives
bitwise the outputs of the whole-batch schedule, for the generic kernels
(FP64, FP32 pairs, FP32 on a 37 x 30 box) and for the FP32 register and
bulk-copy (TMA) column passes of 540- and 537-point lines (direct and
Bluestein), with a ragged last chunk."""
import numpy as np
import pytest

from gpu_common import binding, grid_lengths, to_dev, torch_cuda
from paper_2606_06247_gb300 import inputs

NAMES = ["W", "DX", "DY", "LAP"]


def _fields(nx, ny, batch, seed):
    return np.stack([inputs.smooth_field(nx, ny, seed=seed + k) for k in range(batch)])


def _chunked_outputs(torch, ctx, f, batch, nx, ny, dtype, chunks):
    res = []
    for ch in chunks:
        ctx.set_op_chunk(ch)
        assert ctx.get_op_chunk() == ch
        outs = [torch.full((batch, nx, ny), np.nan, dtype=dtype, device="cuda") for _ in NAMES]
        ctx.spectral_op(f, NAMES, outs)
        ctx.sync()
        res.append([o.cpu().numpy() for o in outs])
    return res


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32x2", "f32"])
def test_chunked_spectral_op_is_the_whole_batch(prec):
    torch = torch_cuda()
    b = binding()
    nx, ny, batch = 37, 30, 5
    lx, ly = grid_lengths(nx, ny, True)
    ctx = b.Context(nx, ny, lx, ly, x_walls=True, batch=batch, family="G8", h_over_dx=1.3, prec=prec)
    io = "f32" if prec == "f32" else "f64"
    f = to_dev(_fields(nx, ny, batch, 21), io)
    dtype = torch.float32 if prec == "f32" else torch.float64
    res = _chunked_outputs(torch, ctx, f, batch, nx, ny, dtype, [0, 1, 2, 3, 5, 9])
    for other in res[1:]:
        for a, r in zip(other, res[0]):
            assert np.isfinite(a).all()
            np.testing.assert_array_equal(a, r)


@pytest.mark.gpu
@pytest.mark.parametrize("n_cont", [28, 25])
def test_chunked_register_and_bulk_copy_passes(n_cont):
    torch = torch_cuda()
    b = binding()
    nx, ny, batch = 64, 512, 7
    lx, ly = grid_lengths(nx, ny, False)
    ctx = b.Context(nx, ny, lx, ly, batch=batch, n_cont=n_cont, family="G4", h_over_dx=1.3, prec="f32")
    f = to_dev(_fields(nx, ny, batch, 5), "f32")
    res = _chunked_outputs(torch, ctx, f, batch, nx, ny, torch.float32, [0, 2, 3])
    for other in res[1:]:
        for a, r in zip(other, res[0]):
            assert np.isfinite(a).all()
            np.testing.assert_array_equal(a, r)


@pytest.mark.gpu
def test_op_chunk_rejects_negative():
    torch_cuda()
    b = binding()
    ctx = b.Context(32, 32, 32 / 31, 1.0, batch=2)
    with pytest.raises(b.FcsphError) as e:
        ctx.set_op_chunk(-1)
    assert e.value.status == 1
