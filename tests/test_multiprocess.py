"""The replica path of bench.py on the CPU: world size 2 over gloo.  Each
rank times its own batch; every rank must see the slowest rank's time, the
whole-job rate counts the units of all ranks, and the reference arm runs on
rank 0 only."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = [30.0, 50.0][rank]
    t_max = bench.max_over_ranks(local_ms, ws)
    dist.barrier()
    out[rank] = (t_max, bench.job_rate(1000, ws, t_max))
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_all_units_count():
    import torch.multiprocessing as mp
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        t_max, rate = res[r]
        assert t_max == 50.0
        assert rate == pytest.approx(1000 * 2 / 0.05)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup, batch = 1, 0, 32

    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
