"""The library's own continuous-batching scheduler (fcsph_batch_* through the
C ABI): each request's result is the same alone and in a mix of kinds, sizes
and Reynolds numbers (bitwise), equal to the Python server's result for the
same request, and at parity with the oracle; a request removed while it runs
frees its slot for the next one; with a budget for one class at a time,
classes are dropped and created as requests wait."""
import time

import numpy as np
import pytest

from gpu_common import binding, oracle_problem, parity_tol, rel_l2, torch_cuda, ulp_floor
from oracle import step as ostep

MIX = [("cavity", 32, 400.0, 4), ("channel", 32, 50.0, 6), ("cavity", 48, 1000.0, 3), ("cavity", 32, 2500.0, 5),
       ("channel", 40, 800.0, 2), ("channel3d", 16, 300.0, 3), ("channel3d", 16, 900.0, 2)]


def _serve(b, reqs, prec, slots=4, budget=0.0, n_cont=25):
    bt = b.Batch(prec=prec, slots=slots, mem_budget=budget, n_cont=n_cont)
    ids = [bt.add(*r) for r in reqs]
    for _ in range(100000):
        inflight = bt.run()
        if all(bt.poll(i)["state"] == "done" for i in ids):
            break
        if inflight:
            time.sleep(1e-4)
    infos = [bt.poll(i) for i in ids]
    out = [bt.result(i, r[0], r[1]) for i, r in zip(ids, reqs)]
    bt.close()
    return out, infos


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_native_batch_alone_equals_in_mix(prec):
    torch_cuda()
    b = binding()
    mix, infos = _serve(b, MIX, prec)
    assert [i["done_steps"] for i in infos] == [r[3] for r in MIX]
    assert all(i["total_step_ms"] > 0 for i in infos)
    for k, r in enumerate(MIX):
        alone, _ = _serve(b, [r], prec)
        for f in alone[0]:
            np.testing.assert_array_equal(alone[0][f], mix[k][f], err_msg=f"{r} {f}")


@pytest.mark.gpu
def test_native_batch_matches_python_server_and_oracle():
    torch_cuda()
    b = binding()
    from paper_2606_06247_gb300.serve import Request, Server
    reqs = [("cavity", 32, 400.0, 3), ("channel", 32, 50.0, 3)]
    native, _ = _serve(b, reqs, "f64", slots=2)
    srv = Server(prec="f64", capacity=2)
    py = [Request(k, *r) for k, r in enumerate(reqs)]
    for r in py:
        srv.submit(r)
    while not srv.idle():
        srv.tick(0.0)
    for n, p in zip(native, py):
        for f in ("u", "v", "p"):
            np.testing.assert_array_equal(n[f], p.result[f])
    N = 32
    cav = oracle_problem(N, N, True, "G8", 1.3, scheme="rk3", nu=1.0 / 400.0, dt=1e-3, u_top=1.0)
    z = np.zeros((N, N))
    fn = lambda a, c: ostep.isph_steps(cav, a, c, 3)
    uo, vo, po = fn(z, z)
    fl = ulp_floor(fn, z, z, scale=1.0)
    assert rel_l2(native[0]["u"], uo) < parity_tol(fl[0])


@pytest.mark.gpu
def test_native_batch_remove_frees_the_slot():
    torch_cuda()
    b = binding()
    bt = b.Batch(prec="f64", slots=1, mem_budget=0.0)
    long_id = bt.add("cavity", 32, 400.0, 1000)
    for _ in range(3):
        bt.run(block=True)
    assert bt.poll(long_id)["state"] == "running"
    nxt = bt.add("cavity", 32, 400.0, 2)
    bt.remove(long_id)
    for _ in range(10000):
        bt.run(block=True)
        if bt.poll(nxt)["state"] == "done":
            break
    assert bt.poll(long_id)["state"] == "cancelled" and bt.poll(long_id)["done_steps"] < 1000
    assert bt.poll(nxt)["done_steps"] == 2
    alone, _ = _serve(b, [("cavity", 32, 400.0, 2)], "f64", slots=1)
    np.testing.assert_array_equal(bt.result(nxt, "cavity", 32)["u"], alone[0]["u"])
    bt.close()


@pytest.mark.gpu
def test_native_batch_budget_holds_one_class_at_a_time():
    torch_cuda()
    b = binding()
    reqs = [("cavity", 32, 400.0, 2), ("channel", 32, 50.0, 2), ("cavity", 48, 1000.0, 2)]
    from paper_2606_06247_gb300.serve import footprint_bytes
    budget = 1.2 * footprint_bytes(48, 2, "f64")   # the two 32^2 classes, or the 48^2 class alone
    assert footprint_bytes(32, 2, "f64") * 2 < budget < footprint_bytes(32, 2, "f64") + footprint_bytes(48, 2, "f64")
    served, _ = _serve(b, reqs, "f64", slots=2, budget=budget)
    alone = [_serve(b, [r], "f64", slots=2)[0][0] for r in reqs]
    for s, a in zip(served, alone):
        np.testing.assert_array_equal(s["u"], a["u"])


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_per_instance_time_step(prec):
    """isph_step's dt_inst: an instance stepped with its own dt equals the same
    instance stepped with that dt for the whole batch (bitwise)."""
    torch = torch_cuda()
    b = binding()
    N = 32
    ctx = b.Context(N, N, 1.0, 1.0, x_walls=True, batch=2, family="G8", h_over_dx=1.3, prec=prec)
    rng = np.random.default_rng(4)
    init = torch.tensor(1e-3 * rng.standard_normal((2, N, N)), device="cuda")

    def run(dt, dt_inst=None):
        u, v = init.clone(), init.flip(1).clone()
        p, fu, fv = torch.zeros_like(u), torch.zeros_like(u), torch.zeros_like(u)
        ctx.isph_step(u, v, p, fu, fv, 4, nu=1.0 / 400.0, dt=dt, u_top=1.0, scheme="rk3", dt_inst=dt_inst)
        ctx.sync()
        return u.cpu().numpy(), v.cpu().numpy()

    per = run(1e-3, torch.tensor([1e-3, 5e-4], dtype=torch.float64, device="cuda"))
    big, small = run(1e-3), run(5e-4)
    for a, x, y in zip(per, big, small):
        np.testing.assert_array_equal(a[0], x[0])
        np.testing.assert_array_equal(a[1], y[1])
    assert np.abs(big[0][1] - small[0][1]).max() > 1e-9


@pytest.mark.gpu
def test_size_priorities_leave_results_unchanged():
    """fcsph_batch_set_size_priorities only reorders the classes' streams on the
    GPU: every request's result is bitwise the one without priorities."""
    torch_cuda()
    b = binding()
    reqs = [("cavity", 64, 400.0, 3), ("channel", 32, 50.0, 4), ("cavity", 48, 1000.0, 3)]
    ref, _ = _serve(b, reqs, "f32x2")
    bt = b.Batch(prec="f32x2", slots=4, mem_budget=0.0)
    bt.set_size_priorities(True)
    ids = [bt.add(*r) for r in reqs]
    for _ in range(100000):
        bt.run(block=True)
        if all(bt.poll(i)["state"] == "done" for i in ids):
            break
    for i, r, a in zip(ids, reqs, ref):
        got = bt.result(i, r[0], r[1])
        for f in got:
            np.testing.assert_array_equal(got[f], a[f])
    bt.close()
