"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/fcsph.h declares, rejects bad arguments, and its host-side FC table
builder reproduces the oracle's tables (no GPU needed for these calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import fc as ofc
from tables import gram_golden

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fcsph.h")).read()
    return sorted(set(re.findall(r"^(?:fcsph_status|long long)\s+(\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_06247_gb300 import build
    build.build()
    from paper_2606_06247_gb300 import binding
    return binding


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib.lib, n), n


@pytest.mark.parametrize("n_cont", [22, 24, 25, 26])
def test_gram_table_bitwise_equal_to_oracle(lib, n_cont):
    # both sides solve the same least squares in extended precision and round once
    np.testing.assert_array_equal(lib.fc_table("gram", 5, n_cont), gram_golden(5, n_cont))


@pytest.mark.parametrize("n_cont", [28, 32])
def test_gram_table_close_to_oracle(lib, n_cont):
    G = gram_golden(5, n_cont)
    assert np.abs(lib.fc_table("gram", 5, n_cont) - G).max() < 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("m,p,c", [(5, 3, 25), (10, 5, 16), (8, 4, 12)])
@pytest.mark.parametrize("bc", [0, 1])
def test_paper_table_matches_oracle(lib, m, p, c, bc):
    O = ofc.paper_table(m, c, p, bc)
    assert np.abs(lib.fc_table("paper", m, c, bc, p) - O).max() < 1e-13 * np.abs(O).max()


def test_bad_arguments_are_rejected(lib):
    with pytest.raises(lib.FcsphError) as e:
        lib.fc_table("gram", 1, 25)
    assert e.value.status == 1
    with pytest.raises(lib.FcsphError):
        lib.fc_table("paper", 5, 25, 0, 5)  # poly_deg must be < n_match
    L = lib.lib
    # context-taking entry points reject a null context without touching a GPU
    assert L.fcsph_set_tiling(None, 1, 1) == 1
    r, c = ctypes.c_int(), ctypes.c_int()
    assert L.fcsph_get_tiling(None, ctypes.byref(r), ctypes.byref(c)) == 1
    assert L.fcsph_set_cta_threads(None, 32, 32) == 1
    assert L.fcsph_get_cta_threads(None, ctypes.byref(r), ctypes.byref(c)) == 1
    assert L.fcsph_set_step_groups(None, 2) == 1
    assert L.fcsph_get_step_groups(None, ctypes.byref(r)) == 1
    assert L.fcsph_set_step_persistent(None, 1) == 1
    assert L.fcsph_set_tma(None, 1) == 1
    assert L.fcsph_set_tracing(None, 1) == 1
    assert L.fcsph_get_step_persistent(None, ctypes.byref(r)) == 1
    prm = lib.fcsph_step_params(1e-3, 1.0, 1e-3, 0.0, 0.0, 0.0, 1.0, 1, 1, None, None)
    assert L.fcsph_autotune(None, ctypes.byref(prm), 3, None) == 1
    assert L.fcsph_sync(None) == 1


def test_create_rejects_bad_grids_before_touching_the_gpu(lib):
    """fcsph_create validates its arguments first, so these run without a GPU."""
    import ctypes as C

    def create(nx=32, ny=32, batch=1, x_walls=0, nz=1, lz=0.0, family=2, prec=0, refine=0, n_match=5, n_cont=25):
        g = lib.fcsph_grid(nx, ny, 1.0, 1.0, x_walls, batch, nz, lz)
        fc = lib.fcsph_fc(0, n_match, n_cont, 0)
        k = lib.fcsph_kernel(family, 1.3)
        p = lib.fcsph_precision(prec, refine)
        h = C.c_void_p()
        return lib.lib.fcsph_create(C.byref(g), C.byref(fc), C.byref(k), C.byref(p), None, None, None, C.byref(h))

    assert create(batch=0) == 1                    # no instances
    assert create(nx=3) == 1                       # too few x nodes
    assert create(ny=8) == 1                       # fewer than 2 * n_match wall-normal nodes
    assert create(x_walls=1, nz=4, lz=1.0) == 1    # 3D needs periodic x
    assert create(nz=4, lz=0.0) == 1               # 3D needs a z period
    assert create(prec=7) == 1                     # unknown precision
    assert create(family=0) == 1                   # unknown kernel family
    assert create(nx=9000) == 1                    # beyond the supported size
    assert create(batch=70000) == 1                # more instances than a launch grid dimension holds
    assert create(nz=4, lz=1.0, prec=1, refine=2) == 6  # PPE refinement is 2D only
