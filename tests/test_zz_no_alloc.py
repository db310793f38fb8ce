"""fcsph_dft_noalloc, the allocation-free variant of the batched DFT, for
callers that cannot allocate device memory (an application whose memory pool
owns all device memory, a plugin or host thread that must not call the CUDA
allocator).

Through the C ABI it must give the same transform as fcsph_dft on two calls in
a row (the second call reuses the shared fixed scratch left by the first), work
as the very first library call of a process, leave the device's free memory
unchanged, and refuse lengths whose scratch or shared-memory line does not
fit.  Kept in a file that pytest collects last, so a failure here never hides
the other GPU tests."""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_common import binding, torch_cuda

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


_FIRST_CALL = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
from paper_2606_06247_gb300 import binding as b
rng = np.random.default_rng(3)
worst = 0.0
# first library call of the process: a 256-point FP32 line needs more than the
# default 48 KB of dynamic shared memory, 89 goes through Bluestein
for n, dt, tol in ((256, torch.complex64, 2e-6), (89, torch.complex128, 1e-13), (4096, torch.complex128, 1e-13)):
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    out = torch.empty((3, n), dtype=dt, device="cuda")
    b.fcsph_dft_noalloc(torch.tensor(x, dtype=dt).cuda(), out, -1)
    torch.cuda.synchronize()
    ref = np.fft.fft(x, axis=-1)
    err = np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < tol, (n, err)
    worst = max(worst, err / tol)
print("ok", worst)
"""


@pytest.mark.gpu
def test_noalloc_as_first_call_of_a_process():
    torch_cuda()
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL.format(root=ROOT)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


@pytest.mark.gpu
def test_noalloc_leaves_free_device_memory_unchanged():
    torch = torch_cuda()
    b = binding()
    rng = np.random.default_rng(11)
    for n in (256, 281, 1049):
        x = torch.tensor(rng.standard_normal((64, n)) + 1j * rng.standard_normal((64, n))).cuda()
        out = torch.empty_like(x)
        b.fcsph_dft_noalloc(x, out, -1)  # loads the kernels' modules
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        b.fcsph_dft_noalloc(x, out, -1)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, n


@pytest.mark.gpu
def test_noalloc_rejects_lengths_beyond_the_scratch():
    torch = torch_cuda()
    b = binding()
    n = 9973  # prime: Bluestein with m = 20000 needs (2m + n) * 24 bytes > 1 MiB
    x = torch.zeros((1, n), dtype=torch.complex128, device="cuda")
    with pytest.raises(b.FcsphError) as e:
        b.fcsph_dft_noalloc(x, torch.empty_like(x))
    assert e.value.status == 1


@pytest.mark.gpu
def test_noalloc_rejects_lines_beyond_shared_memory_before_any_launch():
    torch = torch_cuda()
    b = binding()
    # 8192 points fit the scratch (8192 * 24 bytes) but an FP64 line of 8192
    # complex values (2 x 128 KB) does not fit one CTA's shared memory
    x = torch.ones((2, 8192), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(x)
    with pytest.raises(b.FcsphError) as e:
        b.fcsph_dft_noalloc(x, out)
    assert e.value.status == 1
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    assert "shared memory" in b.last_error()
    # the same length in FP32 fits and runs
    xf = torch.ones((2, 8192), dtype=torch.complex64, device="cuda")
    of = torch.empty_like(xf)
    b.fcsph_dft_noalloc(xf, of)
    torch.cuda.synchronize()
    assert abs(of[0, 0].item() - 8192) < 1e-2 and torch.abs(of[:, 1:]).max().item() < 1e-2
