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
