"""Seeded synthetic workloads shared by the tests, the benchmark and the smoke check.

Only random draws and the shapes of the workloads live here (no step of the
method), so both the CUDA path and the FP64 oracle can be fed identical
arrays.  Shapes follow the paper's wall-bounded benchmarks (Sec. 6): a channel
periodic in x with walls at y = 0, 1 (Sec. 6.3), a square box with walls all
round, and the operator test function of Eq. 35.
"""
import numpy as np


def channel_initial(nx, ny, seed=1, sigma=1e-6):
    """u = v = 0 plus N(0, sigma^2) noise on the interior (non-wall) nodes."""
    rng = np.random.default_rng(seed)
    u = np.zeros((nx, ny))
    v = np.zeros((nx, ny))
    u[:, 1:-1] = sigma * rng.standard_normal((nx, ny - 2))
    v[:, 1:-1] = sigma * rng.standard_normal((nx, ny - 2))
    return u, v


def cavity_initial(nx, ny, seed=None, sigma=0.0):
    """Fluid at rest (the lid velocity is imposed by the wall condition)."""
    u = np.zeros((nx, ny))
    v = np.zeros((nx, ny))
    if seed is not None and sigma > 0:
        rng = np.random.default_rng(seed)
        u[1:-1, 1:-1] = sigma * rng.standard_normal((nx - 2, ny - 2))
        v[1:-1, 1:-1] = sigma * rng.standard_normal((nx - 2, ny - 2))
    return u, v


def dipole_initial(n, omega_e=299.528, r0=0.1, x1=-0.1, x2=0.1):
    """Sec. 6.5 vortex dipole on [-1, 1]^2 (walls all round, nodes on the walls):
    two monopoles of vorticity omega_e (1 - (r/r0)^2) e^{-(r/r0)^2} at (x1, 0)
    and (x2, 0) with opposite signs; the printed velocity field of each is
    (-(1/2)|omega_e| (y - y_c), (1/2)|omega_e| (x - x_c)) e^{-(r/r0)^2}, with
    the sign of the second monopole reversed.  |omega_e| = 299.528 gives a
    total kinetic energy E(0) = 2.  Returns (u, v) of shape (n, n), [i][j] =
    (x_i, y_j)."""
    x = np.linspace(-1.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    e1 = np.exp(-((X - x1) ** 2 + Y ** 2) / r0 ** 2)
    e2 = np.exp(-((X - x2) ** 2 + Y ** 2) / r0 ** 2)
    w = 0.5 * abs(omega_e)
    u = -w * Y * e1 + w * Y * e2
    v = w * (X - x1) * e1 - w * (X - x2) * e2
    return u, v


def smooth_field(nx, ny, seed=0, modes=4, poly_deg=4):
    """A smooth non-periodic field on x in [0,1), y in [0,1]: a few random
    low Fourier modes times random polynomials in y (band-limited in x)."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) / nx
    y = np.linspace(0.0, 1.0, ny)
    f = np.zeros((nx, ny))
    for _ in range(modes):
        k = rng.integers(0, 4)
        ph = rng.uniform(0, 2 * np.pi)
        c = rng.uniform(-1, 1, poly_deg + 1)
        py = sum(c[i] * y ** i for i in range(poly_deg + 1))
        f += np.cos(2 * np.pi * k * x + ph)[:, None] * py[None, :]
    return f


def band_limited_lines(nlines, n, seed=12345, n_modes=32, poly_deg=4, dtype=np.float32):
    """Lines of length n on y in [0,1]: sum_{m<=n_modes} a_m cos(2 pi m y + phi_m),
    a_m ~ N(0,1)/m, plus sum_{i<=poly_deg} c_i y^i, c_i ~ U(-1,1)."""
    rng = np.random.default_rng(seed)
    y = np.linspace(0.0, 1.0, n)
    out = np.empty((nlines, n), dtype=np.float64)
    m = np.arange(1, n_modes + 1)
    for l in range(nlines):
        a = rng.standard_normal(n_modes) / m
        ph = rng.uniform(0, 2 * np.pi, n_modes)
        c = rng.uniform(-1, 1, poly_deg + 1)
        out[l] = (a[:, None] * np.cos(2 * np.pi * m[:, None] * y[None, :] + ph[:, None])).sum(0)
        out[l] += sum(c[i] * y ** i for i in range(poly_deg + 1))
    return out.astype(dtype)


def band_limited_planes(nplanes, nx, ny, seed=12346, n_modes=64, max_mode=64, poly_deg=4, dtype=np.float32):
    """Planes periodic in x, walls in y: random (m_x, m_y) trig modes plus a
    degree-poly_deg polynomial in y per plane."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) / nx
    y = np.linspace(0.0, 1.0, ny)
    out = np.empty((nplanes, nx, ny), dtype=dtype)
    for p in range(nplanes):
        f = np.zeros((nx, ny))
        mx = rng.integers(0, max_mode + 1, n_modes)
        my = rng.integers(0, max_mode + 1, n_modes)
        a = rng.standard_normal(n_modes) / (1.0 + np.hypot(mx, my))
        ph = rng.uniform(0, 2 * np.pi, n_modes)
        for i in range(n_modes):
            f += a[i] * np.cos(2 * np.pi * mx[i] * x + ph[i])[:, None] * np.cos(2 * np.pi * my[i] * y)[None, :]
        c = rng.uniform(-1, 1, poly_deg + 1)
        f += sum(c[i] * y ** i for i in range(poly_deg + 1))[None, :]
        out[p] = f
    return out


def uneven_batch(n_instances=64, seed=2024, sizes=(64, 128, 256, 512), re_range=(100.0, 5000.0)):
    """Sizes uniform on `sizes`, Re log-uniform on re_range; even index = cavity, odd = channel."""
    rng = np.random.default_rng(seed)
    n = rng.choice(np.asarray(sizes), n_instances)
    re = np.exp(rng.uniform(np.log(re_range[0]), np.log(re_range[1]), n_instances))
    kind = ["cavity" if i % 2 == 0 else "channel" for i in range(n_instances)]
    return [dict(n=int(n[i]), re=float(re[i]), kind=kind[i]) for i in range(n_instances)]


def poisson_requests(rate=200.0, duration=10.0, seed=7, sizes=(64, 128, 256, 512, 1024), steps=(50, 500),
                     frac_3d=0.2, sizes_3d=(64, 96, 128)):
    """Arrival times of a Poisson stream and the size/steps of each request:
    a fraction frac_3d are 3D channels of n^3 (n from sizes_3d), the others
    2D cavities or channels of n^2 (n from sizes)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        st = int(rng.integers(steps[0], steps[1] + 1))
        if rng.uniform() < frac_3d:
            out.append(dict(t=t, n=int(rng.choice(np.asarray(sizes_3d))), steps=st, kind="channel3d"))
        else:
            out.append(dict(t=t, n=int(rng.choice(np.asarray(sizes))), steps=st,
                            kind="cavity" if rng.uniform() < 0.5 else "channel"))
    return out
