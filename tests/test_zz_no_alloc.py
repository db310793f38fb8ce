"""fcsph_dft_noalloc, the allocation-free variant of the batched DFT (for
callers that cannot allocate device memory, such as code running during a
CUDA graph capture or under an allocator that owns all device memory).

Through the C ABI it must give the same transform as fcsph_dft on two calls in
a row (the second call reuses the shared fixed scratch left by the first), and
it must refuse lengths whose scratch does not fit.  Kept in a file that pytest
collects last, so a failure here never hides the other GPU tests."""
import numpy as np
import pytest

from gpu_common import binding, torch_cuda


@pytest.mark.gpu
@pytest.mark.parametrize("n", [89, 256, 281, 510, 1049])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_dft_matches_fcsph_dft_twice(n, prec):
    torch = torch_cuda()
    b = binding()
    rng = np.random.default_rng(n + 7)
    dt = torch.complex128 if prec == "f64" else torch.complex64
    tol = 1e-13 if prec == "f64" else 2e-6
    for call in range(2):
        x = rng.standard_normal((5, n)) + 1j * rng.standard_normal((5, n))
        xd = torch.tensor(x, dtype=dt).cuda()
        for direction in (-1, 1):
            ref = b.fcsph_dft(xd, direction)
            out = torch.empty_like(xd)
            b.fcsph_dft_noalloc(xd, out, direction)
            torch.cuda.synchronize()
            err = (torch.linalg.norm(out - ref) / torch.linalg.norm(ref)).item()
            assert err < tol, (n, prec, call, direction, err)


@pytest.mark.gpu
def test_noalloc_rejects_lengths_beyond_the_scratch():
    torch = torch_cuda()
    b = binding()
    n = 9973  # prime: Bluestein with m = 20000 needs (2m + n) * 24 bytes > 1 MiB
    x = torch.zeros((1, n), dtype=torch.complex128, device="cuda")
    with pytest.raises(b.FcsphError) as e:
        b.fcsph_dft_noalloc(x, torch.empty_like(x))
    assert e.value.status == 1
