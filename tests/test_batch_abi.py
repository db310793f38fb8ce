"""fcsph_batch_* argument checks on the CPU: creating a batch with an explicit
memory budget and queueing requests touch no device, so bad arguments, unknown
handles and unfinished results are rejected here without a GPU."""
import pytest

b = pytest.importorskip("paper_2606_06247_gb300.binding")


def test_create_and_add_validate_arguments():
    with pytest.raises(b.FcsphError) as e:
        b.Batch(prec="f32x2", slots=0, mem_budget=1e9)
    assert e.value.status == 1
    bt = b.Batch(prec="f32x2", slots=4, mem_budget=1e9, n_cont="smooth")
    rid = bt.add("cavity", 64, 1000.0, 10)
    assert rid > 0 and bt.add("channel3d", 32, 100.0, 5) == rid + 1
    for bad in [("cavity", 8, 100.0, 1), ("channel", 64, 0.0, 1), ("channel", 64, 100.0, 0), ("channel3d", 512, 10.0, 1)]:
        with pytest.raises(b.FcsphError) as e:
            bt.add(*bad)
        assert e.value.status == 1
    assert bt.poll(rid) == {"state": "queued", "done_steps": 0, "last_step_ms": 0.0, "total_step_ms": 0.0}
    with pytest.raises(b.FcsphError):
        bt.poll(12345)
    with pytest.raises(b.FcsphError) as e:
        bt.result(rid, "cavity", 64)
    assert "not finished" in str(e.value)
    bt.remove(rid)
    assert bt.poll(rid)["state"] == "cancelled"
    assert bt.info() == {"classes": 0, "queued": 1, "used_bytes": 0.0}
    bt.close()


def test_persistent_mode_arguments_are_checked_before_any_device_call():
    bt = b.Batch(prec="f32x2", slots=2, mem_budget=1e9)
    for bad in (0.0, -1.0, 61.0):
        with pytest.raises(b.FcsphError) as e:
            bt.set_persistent(True, bad)
        assert e.value.status == 1
    with pytest.raises(b.FcsphError) as e:
        bt.inject_stall()   # persistent mode only
    assert e.value.status == 1
    bt.add("channel3d", 32, 100.0, 5)
    with pytest.raises(b.FcsphError) as e:
        bt.set_persistent(True)   # a 3D request is queued
    assert e.value.status == 6
    bt.set_persistent(False)
    bt.close()
    f32 = b.Batch(prec="f32", slots=2, mem_budget=1e9)
    with pytest.raises(b.FcsphError) as e:
        f32.set_persistent(True)
    assert e.value.status == 6
    f32.close()
    L = b.lib
    assert L.fcsph_batch_set_persistent(None, 1, 1.0) == 1
    assert L.fcsph_batch_inject_stall(None) == 1
    assert L.fcsph_batch_set_size_priorities(None, 1) == 1
