"""The smoothing length: the paper's h = 8 dx (Sec. 3.3) against the h = 1.3 dx
the library runs at, with both FC variants on the continuation lengths they
are used with (FC(Gram) d = 5, C = 25; the paper's FC with p = 5 on 10
matching points and n_cont = N/4, Sec. 6.1).

Two measurements in the FP64 oracle, G4 kernel:
  * operator error on the Sec. 6.1 test function (Eq. 35) under refinement;
  * the spectral radius of one FOP projection substep linearised about the
    fluid at rest (power iteration on the oracle's substep with 1e-8
    perturbations), on a 32 x 32 channel (nu = 0.1) and cavity (nu = 1e-3),
    dt = 1e-3.
At h = 8 dx the kernel spans about three continuation widths: the x-derivative
error is set by the kernel's smoothing (1 - W_hat of the test function's modes,
~3e-2 at N = 64), the Laplacian does not converge, and the substep amplifies
perturbations 16-7e4 fold.  At h = 1.3 dx the operators converge at 4th order
(FC(Gram)) and the substep is stable."""
import numpy as np
import pytest

from oracle import fc, norms, ops, step, symbols
from tables import gram_golden


def _test_function(N):
    dx, dy = 1.0 / N, 1.0 / (N - 1)
    X, Y = np.meshgrid(np.arange(N) * dx, np.arange(N) * dy, indexing="ij")
    g1 = Y * (1 - Y)
    g2 = g1 ** 2
    f = np.sin(2 * np.pi * X) * g1 + 0.5 * np.cos(4 * np.pi * X) * g2
    fx = 2 * np.pi * np.cos(2 * np.pi * X) * g1 - 2 * np.pi * np.sin(4 * np.pi * X) * g2
    g2pp = 2 - 12 * Y + 12 * Y ** 2
    lap = np.sin(2 * np.pi * X) * (-4 * np.pi ** 2 * g1 - 2) + 0.5 * np.cos(4 * np.pi * X) * (-16 * np.pi ** 2 * g2 + g2pp)
    return f, fx, lap, dx, dy


def _tables(variant, N):
    if variant == "gram":
        E = gram_golden(5, 25)
        return E, E, 25
    nc = N // 4
    return fc.paper_table(10, nc, 5, fc.DIRICHLET), fc.paper_table(10, nc, 5, fc.NEUMANN), nc


def _operator_errors(variant, h_over_dx, sizes=(32, 64, 128)):
    out = []
    for N in sizes:
        f, fx, lap, dx, dy = _test_function(N)
        E, _, nc = _tables(variant, N)
        S = [symbols.symbol_closed(op, "G4", h_over_dx * dy, N, N + nc, dx, dy) for op in ("DX", "LAP")]
        ox, ol = ops.apply_symbols(f, S, E)
        out.append((norms.l2_abs(ox, fx), norms.l2_abs(ol, lap)))
    return np.array(out)


@pytest.mark.parametrize("variant", ["gram", "paper"])
def test_operators_at_8dx_do_not_reach_the_fc_accuracy(variant):
    e8 = _operator_errors(variant, 8.0)
    e13 = _operator_errors(variant, 1.3)
    # gradient: smoothing-dominated at 8 dx, two to three orders worse than at 1.3 dx
    assert e8[1, 0] > 1e-2 and e8[2, 0] > 1e-3
    assert np.all(e8[:, 0] > 100 * e13[:, 0])
    # Laplacian: O(1e-1) or worse at every size at 8 dx
    assert np.all(e8[:, 1] > 0.1)
    if variant == "gram":
        rates = np.log2(e13[:-1] / e13[1:])
        assert np.all(rates > 3.7), e13


def _substep_radius(variant, h_over_dx, x_walls, nu, N=32, iters=60):
    E, En, _ = _tables(variant, N)
    dy = 1.0 / (N - 1)
    p = step.Problem(nx=N, ny=N, Lx=1.0 if x_walls else N * dy, Ly=1.0, x_walls=x_walls, family="G4",
                     h_over_dx=h_over_dx, E_dir=E, E_neu=En, nu=nu, rho=1.0, dt=1e-3, scheme="fop").build_symbols()
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal((N, N)), rng.standard_normal((N, N))
    z = np.zeros((N, N))
    eps = 1e-8
    lam = 0.0
    for _ in range(iters):
        n0 = np.sqrt((u * u).sum() + (v * v).sum())
        u, v = u / n0, v / n0
        un, vn, _, _, _ = step.substep(p, eps * u, eps * v, z, z, 1.0, 1.0, 0.0)
        u, v = un / eps, vn / eps
        lam = np.sqrt((u * u).sum() + (v * v).sum())
    return lam


@pytest.mark.parametrize("variant", ["gram", "paper"])
@pytest.mark.parametrize("x_walls,nu", [(False, 0.1), (True, 1e-3)])
def test_linearised_substep_is_unstable_at_8dx(variant, x_walls, nu):
    r8 = _substep_radius(variant, 8.0, x_walls, nu)
    assert r8 > 10.0, r8


@pytest.mark.parametrize("variant", ["gram", "paper"])
def test_linearised_channel_substep_is_stable_at_1_3dx(variant):
    assert _substep_radius(variant, 1.3, False, 0.1) < 1.0
