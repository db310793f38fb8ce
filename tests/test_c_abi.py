"""The boundary as a C program sees it: include/fcsph.h compiles as C99 with
warnings as errors, a C caller links libfcsph.so, builds the FC(Gram) table
through fcsph_fc_table and gets the oracle's table back, and argument errors
come back as status codes with a message (no GPU needed for these calls)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from tables import gram_golden

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <stdio.h>
#include "fcsph.h"

int main(void) {
  fcsph_fc fc = {FCSPH_FC_GRAM, 5, 25, 0};
  double E[25 * 10];
  fcsph_status st = fcsph_fc_table(&fc, FCSPH_DIRICHLET, E, 25 * 10);
  if (st != FCSPH_OK) return 10 + (int)st;
  for (int i = 0; i < 25 * 10; ++i) printf("%.17g\n", E[i]);
  /* a grid with no nodes is refused before any device work */
  fcsph_grid g = {0};
  fcsph_kernel k = {FCSPH_G4, 1.3};
  fcsph_precision p = {FCSPH_F64, 0};
  fcsph_ctx* ctx = NULL;
  st = fcsph_create(&g, &fc, &k, &p, NULL, NULL, NULL, &ctx);
  char msg[256];
  fcsph_last_error(NULL, msg, sizeof msg);
  fprintf(stderr, "%d %s\n", (int)st, msg);
  return (st == FCSPH_EINVAL && ctx == NULL) ? 0 : 2;
}
"""


@pytest.fixture(scope="module")
def libdir():
    from paper_2606_06247_gb300 import build
    build.build()
    return os.path.join(ROOT, "paper_2606_06247_gb300")


def test_c_caller_gets_the_oracle_table(libdir, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "caller.c"
    src.write_text(C_SOURCE)
    exe = tmp_path / "caller"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-lfcsph", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    E = np.array([float(x) for x in r.stdout.split()]).reshape(25, 10)
    np.testing.assert_allclose(E, gram_golden(5, 25), rtol=0, atol=1e-12 * np.abs(E).max())
    code, msg = r.stderr.strip().split(" ", 1)
    assert int(code) == 1 and "fcsph_create" in msg
