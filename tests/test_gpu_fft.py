"""The library's FFT engine (fcsph_dft: Stockham mixed radix + Bluestein)
against numpy's FFT at every transform length the configurations use."""
import numpy as np
import pytest

from gpu_common import binding, torch_cuda

# extended lengths (n + 25), PPE even extensions 2(n-1), smooth variants and small edge cases
LENGTHS = [1, 2, 3, 4, 5, 7, 8, 9, 11, 16, 27, 31, 37, 64, 72, 81, 89, 90, 96, 126, 150, 153, 243, 254, 256, 280,
           281, 510, 512, 537, 540, 567, 576, 1000, 1022, 1049, 1050, 2046, 143, 221, 187, 289]


@pytest.mark.gpu
@pytest.mark.parametrize("n", LENGTHS)
@pytest.mark.parametrize("prec", ["f64", "f32", "f32x2"])
def test_dft_matches_numpy(n, prec):
    torch = torch_cuda()
    b = binding()
    rng = np.random.default_rng(n)
    nl = 7
    x = rng.standard_normal((nl, n)) + 1j * rng.standard_normal((nl, n))
    dt = torch.complex64 if prec == "f32" else torch.complex128
    xd = torch.tensor(x, dtype=dt).cuda()
    for direction in (-1, 1):
        y = b.fcsph_dft(xd, direction, double_float=prec == "f32x2").cpu().numpy()
        ref = np.fft.fft(x, axis=-1) if direction < 0 else np.fft.ifft(x, axis=-1) * n
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        # unit roundoff: FP64 2^-53, FP32 pairs about 2^-48 (32x), FP32 2^-24
        u = {"f64": 2e-15, "f32x2": 32 * 2e-15, "f32": 3e-7}[prec]
        tol = u * np.log2(max(n, 2)) * 4
        assert err < tol, (n, prec, direction, err)
