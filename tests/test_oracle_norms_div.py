"""Direct pins for oracle.norms (Eq. 34 and companions) and oracle.ops.divergence.

Norms: hand-computed values.  Divergence: (i) with the delta kernel (h = 0,
W_hat = 1) and no FC on band-limited periodic fields it is the textbook
Fourier divergence, checked against the closed-form derivatives; (ii) the
velocity of a stream function, u = d(psi)/dy, v = -d(psi)/dx, has zero
divergence to round-off for any kernel (the x and y symbols commute), which
fails if the two symbols are swapped or a sign is flipped; (iii) on an
FC-extended walled grid it is the sum of the DX and DY operator outputs."""
import numpy as np

from oracle import norms, ops, symbols
from tables import gram_golden


def test_l2_abs_is_eq34_rms():
    a = np.array([[1.0, 2.0], [2.0, 4.0]])
    b = np.array([[1.0, 0.0], [0.0, 0.0]])
    # differences 0, 2, 2, 4: sum of squares 24 over 4 nodes
    assert norms.l2_abs(a, b) == np.sqrt(6.0)
    assert norms.l2_abs(b, a) == np.sqrt(6.0)
    assert norms.l2_abs(a, a) == 0.0


def test_l2_rel_and_linf_hand_values():
    a = np.array([[1.0, 2.0], [2.0, 4.0]])
    b = np.array([[1.0, 0.0], [0.0, 0.0]])
    assert abs(norms.l2_rel(a, b) - np.sqrt(24.0)) < 1e-15   # ||b||_2 = 1
    assert abs(norms.l2_rel(2 * a, a) - 1.0) < 1e-15
    assert norms.l2_rel(np.array([3.0, 4.0]), np.zeros(2)) == 5.0  # zero reference: absolute 2-norm
    assert norms.linf(a, b) == 4.0
    assert norms.linf(np.array([1.0, -3.0]), np.array([2.0, 2.0])) == 5.0


def _periodic_grid(m0, m1):
    dx, dy = 1.0 / m0, 1.0 / m1
    X, Y = np.meshgrid(np.arange(m0) * dx, np.arange(m1) * dy, indexing="ij")
    return X, Y, dx, dy


def test_divergence_delta_kernel_is_fourier_divergence():
    m0, m1 = 16, 12
    X, Y, dx, dy = _periodic_grid(m0, m1)
    tp = 2 * np.pi
    fx = np.sin(tp * 3 * X + 0.2) * np.cos(tp * 2 * Y)
    fy = np.cos(tp * X) * np.sin(tp * 4 * Y - 0.7) + np.cos(tp * 5 * Y)
    div = (tp * 3 * np.cos(tp * 3 * X + 0.2) * np.cos(tp * 2 * Y)
           + tp * 4 * np.cos(tp * X) * np.cos(tp * 4 * Y - 0.7) - tp * 5 * np.sin(tp * 5 * Y))
    Sx = symbols.symbol_closed("DX", "G4", 0.0, m0, m1, dx, dy)
    Sy = symbols.symbol_closed("DY", "G4", 0.0, m0, m1, dx, dy)
    out = ops.divergence(fx, fy, Sx, Sy, None, None)
    assert np.abs(out - div).max() < 1e-11


def test_divergence_of_stream_function_velocity_vanishes():
    m0, m1 = 16, 20
    X, Y, dx, dy = _periodic_grid(m0, m1)
    tp = 2 * np.pi
    # psi = sin(2 pi (2x + 3y) + 0.4) + cos(2 pi (x - 5y)): u = psi_y, v = -psi_x
    u = tp * 3 * np.cos(tp * (2 * X + 3 * Y) + 0.4) + tp * 5 * np.sin(tp * (X - 5 * Y))
    v = -(tp * 2 * np.cos(tp * (2 * X + 3 * Y) + 0.4) - tp * np.sin(tp * (X - 5 * Y)))
    for fam, h in (("G4", 0.07), ("G8", 0.05)):
        Sx = symbols.symbol_closed("DX", fam, h, m0, m1, dx, dy)
        Sy = symbols.symbol_closed("DY", fam, h, m0, m1, dx, dy)
        out = ops.divergence(u, v, Sx, Sy, None, None)
        assert np.abs(out).max() < 1e-11 * np.abs(u).max() * tp * 5
        # swapping the velocity components (or the symbols) breaks it
        assert np.abs(ops.divergence(v, u, Sx, Sy, None, None)).max() > 1.0


def test_divergence_on_fc_grid_is_sum_of_derivative_outputs():
    nx, ny = 12, 14
    dx, dy = 1.0 / nx, 1.0 / (ny - 1)
    rng = np.random.default_rng(5)
    fx, fy = rng.standard_normal((nx, ny)), rng.standard_normal((nx, ny))
    E = gram_golden(5, 25)
    h = 1.3 * dy
    Sx = symbols.symbol_closed("DX", "G4", h, nx, ny + 25, dx, dy)
    Sy = symbols.symbol_closed("DY", "G4", h, nx, ny + 25, dx, dy)
    div = ops.divergence(fx, fy, Sx, Sy, E)
    ref = ops.apply_symbols(fx, [Sx], E)[0] + ops.apply_symbols(fy, [Sy], E)[0]
    assert np.abs(div - ref).max() < 1e-9 * np.abs(ref).max()
