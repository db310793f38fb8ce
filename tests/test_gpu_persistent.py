"""Persistent multi-class step (fcsph_batch_set_persistent): every tick of the
library's scheduler steps all size classes in one launch of a persistent
kernel that takes (pass, instance, tile) work items from a queue and waits,
boundedly, for the previous pass of the same instance.  Each request's result
equals the per-class graphs' result bitwise (alone and in a mix of kinds,
sizes, Reynolds numbers and precisions); a wait that runs out (a planted
count that never comes, set on the host) is reported as FCSPH_ETIMEOUT and
the batch stays usable."""
import time

import numpy as np
import pytest

from gpu_common import binding, torch_cuda

MIX2D = [("cavity", 32, 400.0, 4), ("channel", 32, 50.0, 6), ("cavity", 48, 1000.0, 3), ("cavity", 32, 2500.0, 5),
         ("channel", 40, 800.0, 2), ("cavity", 64, 300.0, 3), ("channel", 20, 120.0, 4)]


def _serve(b, reqs, prec, persistent, slots=4, n_cont=25, wait_s=1.0):
    bt = b.Batch(prec=prec, slots=slots, mem_budget=0.0, n_cont=n_cont)
    if persistent:
        bt.set_persistent(True, wait_s)
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
def test_persistent_step_equals_the_class_graphs(prec):
    torch_cuda()
    b = binding()
    pers, infos = _serve(b, MIX2D, prec, True)
    assert [i["done_steps"] for i in infos] == [r[3] for r in MIX2D]
    graphs, _ = _serve(b, MIX2D, prec, False)
    for k, r in enumerate(MIX2D):
        for f in pers[k]:
            np.testing.assert_array_equal(pers[k][f], graphs[k][f], err_msg=f"{r} {f}")
    # alone in the persistent launch equals in the mix
    for k in (0, 2, 6):
        alone, _ = _serve(b, [MIX2D[k]], prec, True)
        for f in alone[0]:
            np.testing.assert_array_equal(alone[0][f], pers[k][f], err_msg=f"{MIX2D[k]} {f}")


@pytest.mark.gpu
def test_persistent_step_with_smooth_continuation_and_removal():
    torch_cuda()
    b = binding()
    reqs = [("cavity", 64, 500.0, 3), ("channel", 64, 200.0, 2), ("cavity", 32, 900.0, 4)]
    pers, _ = _serve(b, reqs, "f32x2", True, n_cont=0)
    graphs, _ = _serve(b, reqs, "f32x2", False, n_cont=0)
    for p, g in zip(pers, graphs):
        for f in p:
            np.testing.assert_array_equal(p[f], g[f])
    bt = b.Batch(prec="f64", slots=1, mem_budget=0.0)
    bt.set_persistent(True)
    long_id = bt.add("cavity", 32, 400.0, 1000)
    for _ in range(3):
        bt.run(block=True)
    nxt = bt.add("cavity", 32, 400.0, 2)
    bt.remove(long_id)
    for _ in range(10000):
        bt.run(block=True)
        if bt.poll(nxt)["state"] == "done":
            break
    assert bt.poll(long_id)["state"] == "cancelled"
    alone, _ = _serve(b, [("cavity", 32, 400.0, 2)], "f64", False, slots=1)
    np.testing.assert_array_equal(bt.result(nxt, "cavity", 32)["u"], alone[0]["u"])
    bt.close()


@pytest.mark.gpu
def test_persistent_wait_that_runs_out_is_reported_and_the_batch_stays_usable():
    """The host plants a dependency count that never comes (the last work item
    of the next launch waits for it); the bounded wait gives up after 50 ms,
    the launch drains, fcsph_batch_run returns FCSPH_ETIMEOUT once, and the
    next requests are served correctly."""
    torch_cuda()
    b = binding()
    bt = b.Batch(prec="f32x2", slots=2, mem_budget=0.0)
    bt.set_persistent(True, 0.05)
    first = bt.add("cavity", 32, 400.0, 2)
    bt.inject_stall()
    bt.run()
    t0 = time.perf_counter()
    with pytest.raises(b.FcsphError) as e:
        for _ in range(1000):
            bt.run(block=True)
    assert e.value.status == 4  # FCSPH_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    for _ in range(1000):
        bt.run(block=True)
        if bt.poll(first)["state"] == "done":
            break
    nxt = bt.add("cavity", 32, 400.0, 3)
    for _ in range(1000):
        bt.run(block=True)
        if bt.poll(nxt)["state"] == "done":
            break
    ref, _ = _serve(b, [("cavity", 32, 400.0, 3)], "f32x2", False, slots=2)
    got = bt.result(nxt, "cavity", 32)
    for f in got:
        np.testing.assert_array_equal(got[f], ref[0][f])
    bt.close()


@pytest.mark.gpu
def test_persistent_mode_refuses_3d_and_fp32():
    torch_cuda()
    b = binding()
    bt = b.Batch(prec="f32x2", slots=2, mem_budget=0.0)
    bt.set_persistent(True)
    with pytest.raises(b.FcsphError) as e:
        bt.add("channel3d", 16, 300.0, 2)
    assert e.value.status == 6
    bt.close()
    bt = b.Batch(prec="f32", slots=2, mem_budget=0.0)
    with pytest.raises(b.FcsphError) as e:
        bt.set_persistent(True)
    assert e.value.status == 6
    bt.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32x2"])
def test_persistent_isph_step_equals_the_graph(prec):
    """fcsph_set_step_persistent: isph_step as one persistent launch per step
    gives bitwise the graph's state, with and without an instance mask, and a
    change of the state pointers re-records the step."""
    from gpu_common import grid_lengths, to_dev
    from paper_2606_06247_gb300 import inputs
    torch = torch_cuda()
    b = binding()
    nx, ny, batch = 37, 30, 5
    lx, ly = grid_lengths(nx, ny, True)
    prm = dict(nu=1e-3, rho=1.0, dt=1e-3, u_top=1.0, scheme="rk3")

    def state(seed):
        us, vs = [], []
        for k in range(batch):
            u0, v0 = inputs.cavity_initial(nx, ny, seed=seed + k, sigma=1e-3)
            us.append(u0)
            vs.append(v0)
        u, v = to_dev(np.stack(us)), to_dev(np.stack(vs))
        return [u, v, torch.zeros_like(u), torch.zeros_like(u), torch.zeros_like(u)]

    active = torch.tensor([1, 0, 1, 1, 1], dtype=torch.uint8, device="cuda")
    for mask in (None, active):
        outs = []
        for pers in (False, True, True):
            ctx = b.Context(nx, ny, lx, ly, x_walls=True, batch=batch, family="G8", h_over_dx=1.3, prec=prec)
            ctx.set_step_persistent(pers)
            assert ctx.get_step_persistent() == pers
            st = state(31)
            ctx.isph_step(*st, 2, use_graph=True, active=mask, **prm)
            st2 = [x.clone() for x in st]      # new pointers: the step is recorded again
            ctx.isph_step(*st2, 1, use_graph=True, active=mask, **prm)
            ctx.sync()
            outs.append([x.cpu().numpy() for x in st2])
        for o in outs[1:]:
            for a, r in zip(o, outs[0]):
                np.testing.assert_array_equal(a, r)
    ctx3 = b.Context(16, 20, 16 / 19, 1.0, nz=8, lz=8 / 19)
    with pytest.raises(b.FcsphError) as e:
        ctx3.set_step_persistent(True)
    assert e.value.status == 6
