"""Serving across ranks on the CPU (world size 2 over gloo, no device work):
requests are placed by device footprint, each rank serves its share with its
own server, and rank 0 gets every finished request back exactly once, with
its own result."""
import os
import socket

import numpy as np
import pytest

serve = pytest.importorskip("paper_2606_06247_gb300.serve")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _requests():
    sizes = [64, 512, 128, 256, 64, 1024, 128, 64, 256, 512]
    return [serve.Request(i, "cavity" if i % 2 == 0 else "channel", n, 100.0 + 10 * i, 1 + i % 3, 0.0)
            for i, n in enumerate(sizes)]


def test_placement_balances_footprint():
    reqs = _requests()
    parts, load = serve.place_requests(reqs, 2, prec="f32x2")
    assert sorted(r.rid for p in parts for r in p) == list(range(len(reqs)))
    one = {r.rid: serve.footprint_bytes(r.n, 1, "f32x2", False, 25) for r in reqs}
    assert [sum(one[r.rid] for r in p) for p in parts] == load
    # greedy placement: the two loads differ by at most the largest single request
    assert abs(load[0] - load[1]) <= max(one.values())
    parts1, load1 = serve.place_requests(reqs, 1)
    assert len(parts1[0]) == len(reqs)


class _InstantClass:
    """SizeClass stand-in whose step finishes at once; a request's result
    carries its id so that the gathered results can be checked."""

    def __init__(self, key, capacity, prec, device, n_cont=25):
        self.key, self.kind, self.n, self.capacity, self.prec = key, key[0], key[1], capacity, prec
        self.n_cont, self.d3 = n_cont, key[0] == "channel3d"
        self.slots = [None] * capacity
        self.pending_event = False

        class _Ev:
            @staticmethod
            def query():
                return True
        self.ev1 = _Ev()

    def free_slots(self):
        return [i for i, r in enumerate(self.slots) if r is None]

    def active(self):
        return [i for i, r in enumerate(self.slots) if r is not None]

    def admit(self, slot, req):
        self.slots[slot] = req

    def step(self):
        self.pending_event = True

    def finish_tick(self, now):
        retired = []
        self.pending_event = False
        for i in self.active():
            r = self.slots[i]
            r.done_steps += 1
            r.latencies_ms.append(1.0)
            if r.done_steps >= r.steps:
                r.result = {"u": np.full((2, 2), float(r.rid))}
                self.slots[i] = None
                retired.append(r)
        return retired


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    serve.SizeClass = _InstantClass
    done, walls = serve.serve_on_ranks(_requests(), rank, ws,
                                       lambda: serve.Server(prec="f32x2", capacity=2, mem_budget=1 << 40, device="cpu"))
    if rank == 0:
        out["rids"] = [r.rid for r in done]
        out["ok"] = all(r.done_steps == r.steps and r.result["u"][0, 0] == r.rid for r in done)
        out["ranks"] = sorted({r.rank for r in done})
        out["walls"] = len(walls)
    else:
        out["other"] = done is None and walls is None
    dist.destroy_process_group()


def test_two_ranks_serve_and_gather_on_rank_zero():
    import torch.multiprocessing as mp
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    assert res["rids"] == list(range(10))
    assert res["ok"] and res["ranks"] == [0, 1] and res["walls"] == 2 and res["other"]
