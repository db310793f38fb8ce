"""The 3D channel (x and z periodic, walls in y) through the C ABI: spectral
operators, the PPE and the projection step against oracle.channel3d, in FP64
and FP32 pairs, on grids with even and odd z lengths."""
import numpy as np
import pytest

from gpu_common import binding, parity_tol, rel_l2, to_dev, torch_cuda, ulp_floor
from oracle import channel3d as c3
from tables import gram_golden

E = gram_golden(5, 25)
CASES = [(8, 6, 20, 2), (6, 5, 24, 1), (12, 8, 18, 1)]  # nx, nz, ny, batch


def _lengths(nx, nz, ny):
    dy = 1.0 / (ny - 1)
    return nx * dy, nz * dy, 1.0


def _smooth3(nx, nz, ny, seed):
    rng = np.random.default_rng(seed)
    x = np.arange(nx) / nx
    z = np.arange(nz) / nz
    y = np.linspace(0, 1, ny)
    X, Z, Y = np.meshgrid(x, z, y, indexing="ij")
    f = np.zeros((nx, nz, ny))
    for _ in range(4):
        a, c = rng.integers(0, 3, size=2)
        f += rng.standard_normal() * np.cos(2 * np.pi * (a * X + c * Z) + rng.uniform(0, 6.3)) * \
            np.polyval(rng.uniform(-1, 1, 5), Y)
    return f


def _tol(floor, prec):
    scale = 1.0 if prec == "f64" else 32.0
    return parity_tol(floor, base=1e-12 * scale, factor=10.0 * scale)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_spectral_op_3d_matches_oracle(case, prec):
    torch = torch_cuda()
    b = binding()
    nx, nz, ny, batch = case
    Lx, Lz, Ly = _lengths(nx, nz, ny)
    ctx = b.Context(nx, ny, Lx, Ly, batch=batch, family="G4", h_over_dx=1.3, prec=prec, nz=nz, lz=Lz)
    f = np.stack([_smooth3(nx, nz, ny, 10 + k) for k in range(batch)])
    names = ["W", "DX", "DY", "LAP", "DZ"]
    outs = [torch.zeros((batch, nx, nz, ny), dtype=torch.float64, device="cuda") for _ in names]
    ctx.spectral_op(to_dev(f), names, outs)
    ctx.sync()
    dx, dz, dy = Lx / nx, Lz / nz, Ly / (ny - 1)
    S = [c3.symbol3(n, "G4", 1.3 * dx, nx, nz, ny + 25, dx, dz, dy) for n in names]
    fn = lambda a: c3.apply_symbols3(a, S, E)
    for k in range(batch):
        refs = fn(f[k])
        floors = ulp_floor(fn, f[k])
        for n, o, r, fl in zip(names, outs, refs, floors):
            err = rel_l2(o[k].cpu().numpy(), r)
            assert err < _tol(fl, prec), (n, k, err, fl)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_ppe_3d_matches_oracle(case, prec):
    torch = torch_cuda()
    b = binding()
    nx, nz, ny, batch = case
    Lx, Lz, Ly = _lengths(nx, nz, ny)
    ctx = b.Context(nx, ny, Lx, Ly, batch=batch, prec=prec, nz=nz, lz=Lz)
    rng = np.random.default_rng(7)
    rhs = rng.standard_normal((batch, nx, nz, ny))
    phi = torch.zeros((batch, nx, nz, ny), dtype=torch.float64, device="cuda")
    res = ctx.ppe_solve(to_dev(rhs), phi, want_resid=True)
    scale = 1.0 if prec == "f64" else 32.0
    for k in range(batch):
        ref = c3.ppe_solve3(rhs[k], Lx, Lz, Ly)
        assert rel_l2(phi[k].cpu().numpy(), ref) < 1e-12 * scale
    assert res < 1e-13 * scale


@pytest.mark.gpu
@pytest.mark.parametrize("scheme,nsteps", [("fop", 4), ("rk3", 2)])
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_channel3d_step_matches_oracle(scheme, nsteps, prec):
    torch = torch_cuda()
    b = binding()
    nx, nz, ny = 8, 6, 20
    Lx, Lz, Ly = _lengths(nx, nz, ny)
    rng = np.random.default_rng(3)
    u0, v0, w0 = (1e-3 * rng.standard_normal((nx, nz, ny)) for _ in range(3))
    for a in (u0, v0, w0):
        a[:, :, [0, -1]] = 0.0
    ctx = b.Context(nx, ny, Lx, Ly, family="G4", h_over_dx=1.3, prec=prec, nz=nz, lz=Lz)
    u, v, w = to_dev(u0[None]), to_dev(v0[None]), to_dev(w0[None])
    p, fu, fv, fw = (torch.zeros_like(u) for _ in range(4))
    prm = dict(nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0, 0.1), scheme=scheme)
    ctx.isph_step(u, v, p, fu, fv, nsteps, w=w, fw=fw, **prm)
    ctx.sync()
    prob = c3.Problem3(nx=nx, nz=nz, ny=ny, Lx=Lx, Lz=Lz, Ly=Ly, family="G4", h_over_dx=1.3, E_dir=E, E_neu=E,
                       nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0, 0.1), scheme=scheme).build_symbols()
    fn = lambda a, c, d: c3.isph_steps3(prob, a, c, d, nsteps)
    ref = fn(u0, v0, w0)
    fl = ulp_floor(fn, u0, v0, w0)
    got = [x[0].cpu().numpy() for x in (u, v, w, p)]
    errs = [rel_l2(g, r) for g, r in zip(got, ref)]
    print(f"3D channel {scheme} {prec}: parity (u, v, w, p) {errs}, floor {fl}")
    for e, f in zip(errs, fl):
        assert e < _tol(f, prec)


@pytest.mark.gpu
def test_3d_rejects_what_it_does_not_support():
    torch_cuda()
    b = binding()
    with pytest.raises(b.FcsphError):
        b.Context(8, 20, 1.0, 1.0, x_walls=True, nz=4, lz=1.0)   # 3D needs periodic x
    ctx = b.Context(8, 20, 1.0, 1.0, nz=4, lz=0.5)
    import torch
    f = torch.zeros((1, 8, 4, 20), dtype=torch.float64, device="cuda")
    with pytest.raises(b.FcsphError) as e:
        ctx.spectral_div(f, f, f)
    assert e.value.status == 6
    two = b.Context(8, 20, 1.0, 1.0)
    g = torch.zeros((1, 8, 20), dtype=torch.float64, device="cuda")
    with pytest.raises(b.FcsphError):
        two.spectral_op(g, ["DZ"], [g.clone()])
