"""Continuous batching (paper_2606_06247_gb300.serve): every request's result
is identical alone and in a mix of kinds, sizes and Reynolds numbers; the
per-instance viscosity/force path matches the oracle."""
import numpy as np
import pytest

from gpu_common import binding, oracle_problem, parity_tol, rel_l2, torch_cuda, ulp_floor
from oracle import step as ostep


def _reqs():
    from paper_2606_06247_gb300.serve import Request
    return [Request(0, "cavity", 32, 400.0, 4), Request(1, "channel", 32, 50.0, 6), Request(2, "cavity", 48, 1000.0, 3),
            Request(3, "cavity", 32, 2500.0, 5), Request(4, "channel", 40, 800.0, 2),
            Request(5, "channel3d", 16, 300.0, 3), Request(6, "channel3d", 16, 900.0, 2)]


@pytest.mark.gpu
@pytest.mark.parametrize("fc_cont", [25, "smooth"])
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_result_is_the_same_alone_and_in_the_mix(prec, fc_cont):
    torch_cuda()
    binding()
    from paper_2606_06247_gb300.serve import Server
    mix = _reqs()
    srv = Server(prec=prec, capacity=4, fc_cont=fc_cont)
    for r in mix:
        srv.submit(r)
    while not srv.idle():
        srv.tick(0.0)
    assert all(r.result is not None and r.done_steps == r.steps for r in mix)
    for r in _reqs():
        alone = Server(prec=prec, capacity=4, fc_cont=fc_cont)
        alone.submit(r)
        while not alone.idle():
            alone.tick(0.0)
        m = [x for x in mix if x.rid == r.rid][0]
        for f in r.result:
            np.testing.assert_array_equal(r.result[f], m.result[f])


@pytest.mark.gpu
@pytest.mark.parametrize("fc_cont", [25, "smooth"])
def test_per_instance_viscosity_matches_oracle(fc_cont):
    """The served results match the oracle with the class's continuation
    length (smooth: 24 for N = 32, i.e. 56-point lines instead of 57 = 3 19)."""
    torch_cuda()
    binding()
    from paper_2606_06247_gb300.serve import Request, Server, smooth_n_cont
    srv = Server(capacity=2, fc_cont=fc_cont)
    reqs = [Request(0, "cavity", 32, 400.0, 3), Request(1, "channel", 32, 50.0, 3)]
    for r in reqs:
        srv.submit(r)
    while not srv.idle():
        srv.tick(0.0)
    N = 32
    C = smooth_n_cont(N) if fc_cont == "smooth" else fc_cont
    cav = oracle_problem(N, N, True, "G8", 1.3, n_cont=C, scheme="rk3", nu=1.0 / 400.0, dt=1e-3, u_top=1.0)
    ch = oracle_problem(N, N, False, "G4", 1.3, n_cont=C, scheme="rk3", nu=1.0 / 50.0, dt=1e-3,
                        force=(8.0 / 50.0, 0.0))
    z = np.zeros((N, N))
    for r, prob, scale in ((reqs[0], cav, 1.0), (reqs[1], ch, 1.0)):
        fn = lambda a, c: ostep.isph_steps(prob, a, c, 3)
        uo, vo, po = fn(z, z)
        fl = ulp_floor(fn, z, z, scale=scale)
        assert rel_l2(r.result["u"], uo) < parity_tol(fl[0])
        assert rel_l2(r.result["v"], vo) < parity_tol(fl[1]) or np.abs(vo).max() < 1e-14
