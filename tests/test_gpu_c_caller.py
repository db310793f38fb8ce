"""A C program on the device side of the boundary: it allocates device memory
with the CUDA runtime, steps a channel through fcsph_create / isph_step /
fcsph_sync, serves two requests through the continuous-batching calls
(fcsph_batch_create / add / run / poll / result), and prints the results;
each must be bitwise the one the Python binding gets from the same calls."""
import os
import shutil
import subprocess
import time

import numpy as np
import pytest

from gpu_common import binding, torch_cuda

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime.h>
#include "fcsph.h"

#define N 32

static int fail(const char* what, fcsph_status st) {
  char msg[256];
  fcsph_last_error(NULL, msg, sizeof msg);
  fprintf(stderr, "%s: %d %s\n", what, (int)st, msg);
  return 3;
}

int main(void) {
  /* 1. a 32 x 32 channel, FP64, two FOP steps from rest under a body force */
  const double dy = 1.0 / (N - 1);
  fcsph_grid g = {N, N, N * dy, 1.0, 0, 1, 1, 0.0};
  fcsph_fc fc = {FCSPH_FC_GRAM, 5, 25, 0};
  fcsph_kernel k = {FCSPH_G4, 1.3};
  fcsph_precision p = {FCSPH_F64, 0};
  fcsph_ctx* ctx = NULL;
  fcsph_status st = fcsph_create(&g, &fc, &k, &p, NULL, NULL, NULL, &ctx);
  if (st != FCSPH_OK) return fail("create", st);
  double* d = NULL;
  const size_t n = (size_t)N * N;
  if (cudaMalloc((void**)&d, 5 * n * sizeof(double)) != cudaSuccess) return 4;
  cudaMemset(d, 0, 5 * n * sizeof(double));
  fcsph_state s = {d, d + n, d + 2 * n, d + 3 * n, d + 4 * n, NULL, NULL};
  fcsph_step_params prm = {0};
  prm.nu = 0.1;
  prm.rho = 1.0;
  prm.dt = 1e-3;
  prm.force_x = 0.8;
  prm.scheme = FCSPH_SCHEME_FOP;
  prm.use_graph = 1;
  if ((st = isph_step(ctx, &s, 2, &prm)) != FCSPH_OK) return fail("isph_step", st);
  if ((st = fcsph_sync(ctx)) != FCSPH_OK) return fail("sync", st);
  double* u = (double*)malloc(n * sizeof(double));
  cudaMemcpy(u, d, n * sizeof(double), cudaMemcpyDeviceToHost);
  for (size_t i = 0; i < n; ++i) printf("%.17g\n", u[i]);
  fcsph_destroy(ctx);
  cudaFree(d);

  /* 2. continuous batching: two cavity requests of different sizes */
  fcsph_batch* b = NULL;
  if ((st = fcsph_batch_create(FCSPH_F32X2, 2, 0.0, 25, &b)) != FCSPH_OK) return fail("batch_create", st);
  fcsph_request r1 = {FCSPH_REQ_CAVITY, 32, 400.0, 3}, r2 = {FCSPH_REQ_CAVITY, 48, 1000.0, 2};
  long long id1 = 0, id2 = 0;
  if ((st = fcsph_batch_add(b, &r1, &id1)) != FCSPH_OK || (st = fcsph_batch_add(b, &r2, &id2)) != FCSPH_OK)
    return fail("batch_add", st);
  for (int it = 0; it < 100000; ++it) {
    int inflight = 0;
    if ((st = fcsph_batch_run(b, 1, &inflight)) != FCSPH_OK) return fail("batch_run", st);
    fcsph_request_info i1, i2;
    fcsph_batch_poll(b, id1, &i1);
    fcsph_batch_poll(b, id2, &i2);
    if (i1.state == FCSPH_REQ_DONE && i2.state == FCSPH_REQ_DONE) break;
  }
  double* u1 = (double*)malloc(32 * 32 * sizeof(double));
  double* u2 = (double*)malloc(48 * 48 * sizeof(double));
  if ((st = fcsph_batch_result(b, id1, u1, NULL, NULL, NULL, 32 * 32)) != FCSPH_OK) return fail("result", st);
  if ((st = fcsph_batch_result(b, id2, u2, NULL, NULL, NULL, 48 * 48)) != FCSPH_OK) return fail("result", st);
  for (int i = 0; i < 32 * 32; ++i) printf("%.17g\n", u1[i]);
  for (int i = 0; i < 48 * 48; ++i) printf("%.17g\n", u2[i]);
  fcsph_batch_destroy(b);
  free(u);
  free(u1);
  free(u2);
  return 0;
}
"""


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.isdir(c):
            return c
    nvcc = shutil.which("nvcc")
    return os.path.dirname(os.path.dirname(nvcc)) if nvcc else None


@pytest.mark.gpu
def test_c_caller_steps_and_serves_like_the_binding(tmp_path):
    torch = torch_cuda()
    b = binding()
    cc, cuda = shutil.which("gcc") or shutil.which("cc"), _cuda_home()
    if cc is None or cuda is None:
        pytest.skip("no C compiler or CUDA toolkit")
    libdir = os.path.join(ROOT, "paper_2606_06247_gb300")
    src = tmp_path / "caller.c"
    src.write_text(C_SOURCE)
    exe = tmp_path / "caller"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), str(src), "-L", libdir, "-lfcsph",
                    "-Wl,-rpath," + libdir, "-L", os.path.join(cuda, "lib64"), "-lcudart",
                    "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    vals = np.array([float(x) for x in r.stdout.split()])
    n = 32
    u_c, u1_c, u2_c = vals[:n * n], vals[n * n:2 * n * n], vals[2 * n * n:]
    assert u2_c.size == 48 * 48
    # the same through the binding
    dy = 1.0 / (n - 1)
    ctx = b.Context(n, n, n * dy, 1.0, batch=1, family="G4", h_over_dx=1.3, prec="f64")
    st = [torch.zeros((1, n, n), dtype=torch.float64, device="cuda") for _ in range(5)]
    ctx.isph_step(*st, 2, nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0), scheme="fop", use_graph=True)
    ctx.sync()
    np.testing.assert_array_equal(u_c, st[0][0].cpu().numpy().ravel())
    bt = b.Batch(prec="f32x2", slots=2, mem_budget=0.0, n_cont=25)
    i1, i2 = bt.add("cavity", 32, 400.0, 3), bt.add("cavity", 48, 1000.0, 2)
    for _ in range(100000):
        bt.run(block=True)
        if bt.poll(i1)["state"] == "done" and bt.poll(i2)["state"] == "done":
            break
        time.sleep(0)
    np.testing.assert_array_equal(u1_c, bt.result(i1, "cavity", 32)["u"].ravel())
    np.testing.assert_array_equal(u2_c, bt.result(i2, "cavity", 48)["u"].ravel())
    bt.close()
