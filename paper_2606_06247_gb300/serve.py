"""Continuous batching of independent wall-bounded solves on one GPU.

Requests of different sizes and kinds (lid-driven cavity / channel / 3D
channel of n^3) arrive over time; each asks for a number of RK3 projection
steps.  A size class (kind, n, kernel family) owns one fcsph context with a
fixed number of slots
(its batch) and device-resident state for every slot; the class advances all
its slots with one CUDA-graph step at a time on its own stream, so classes
overlap on the GPU.  Classes run independently: the host polls each class's
end-of-step event and, when a class's step is done, retires its finished
requests (state copied to the host), admits queued requests into the freed
slots and launches its next step, without waiting for the other classes.
The step runs only the occupied slots (isph_step's instance mask): an empty
slot costs its CTAs an early return.  New classes are admitted only while the estimated device footprint of all
classes fits the memory budget.

Every slot is an independent instance of the step: its result does not
depend on which slot it occupies or on what the other slots hold, so a
request's result is the same alone and in the mix (bitwise, same precision).

The per-request Reynolds number enters through per-instance viscosity (and,
for the channels, body force): cavity nu = 1/Re (lid speed 1, side 1);
channel (2D and 3D) u_max = 1, nu = 1/Re, F = 8 nu.

FC continuation length: 25 points for every size (fc_cont=25), or per size
the length nearest 25 in [20, 40] whose extended line n + C the FFT engine
transforms directly (fc_cont="smooth"; see smooth_n_cont).  The continuation
length is a free parameter of FC(Gram) (Sec. 4: the Gram fit sets the
accuracy, C the period); with 25, sizes such as 512 (537 = 3 * 179) or 1024
(1049, prime) need Bluestein transforms of about twice the length.
"""
import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as b

DT = 1e-3


@dataclass
class Request:
    rid: int
    kind: str          # "cavity", "channel" or "channel3d"
    n: int             # n x n (3D: n x n x n) particles
    re: float
    steps: int
    arrival: float = 0.0
    # filled by the server
    done_steps: int = 0
    latencies_ms: list = field(default_factory=list)
    result: dict = None
    t_admit: float = None
    t_done: float = None


# Radices the FFT engine runs as register butterflies.
_DIRECT_PRIMES = (2, 3, 5, 7, 11, 13, 17)


def _factors_over(m, primes):
    for q in primes:
        while m % q == 0:
            m //= q
    return m == 1


def smooth_n_cont(n, base=25, lo=20, hi=40):
    """FC continuation length for n wall-normal nodes: `base` if n + base
    factors into the engine's register radices (2..17); else the length in
    [lo, hi] nearest `base` (the smaller on a tie) with n + C 7-smooth; else
    `base`."""
    if _factors_over(n + base, _DIRECT_PRIMES):
        return base
    for d in range(1, max(base - lo, hi - base) + 1):
        for c in (base - d, base + d):
            if lo <= c <= hi and _factors_over(n + c, (2, 3, 5, 7)):
                return c
    return base


def request_dt(req):
    """Time step of a request: dt = min(1e-3, 0.25 dx^2 Re).  The explicit
    viscous limit of the smoothed Laplacian at h = 1.3 dx is about
    0.6 dx^2 / nu (RK3), so low-Re requests on fine grids need less than
    1e-3."""
    dx = 1.0 / (req.n - 1)
    return min(DT, 0.25 * dx * dx * req.re)


def family_for(kind, re):
    """Kernel family per the paper's guidance: G4 at low Re, G8 at high Re (cavity always G8)."""
    if kind == "cavity":
        return "G8"
    return "G4" if re < 625 else "G8"


def class_key(req):
    return (req.kind, req.n, family_for(req.kind, req.re))


def particles(req):
    return req.n ** 3 if req.kind == "channel3d" else req.n ** 2


def footprint_bytes(n, capacity, prec, d3=False, n_cont=25):
    """Device bytes of one class: state, workspace and spectra per slot
    (2D: 5 + 6 fields, 8 spectra; 3D: 7 + 7 fields, 15 spectra)."""
    my = n + n_cont
    hy = my // 2 + 1
    rows = max(hy, n)
    cb = 8 if prec == "f32" else 16
    ncol = n * n if d3 else n
    fields, specs = (14, 15) if d3 else (11, 8)
    return capacity * (fields * ncol * n * 8 + specs * rows * ncol * cb + rows * ncol * 16)


class SizeClass:
    def __init__(self, key, capacity, prec, device, n_cont=25):
        kind, n, fam = key
        self.key, self.kind, self.n, self.capacity, self.prec = key, kind, n, capacity, prec
        self.n_cont = n_cont
        self.d3 = kind == "channel3d"
        x_walls = kind == "cavity"
        dy = 1.0 / (n - 1)
        lx = 1.0 if x_walls else n * dy
        self.stream = torch.cuda.Stream(device=device)
        with torch.cuda.stream(self.stream):
            self.ctx = b.Context(n, n, lx, 1.0, x_walls=x_walls, batch=capacity, n_cont=n_cont, family=fam,
                                 h_over_dx=1.3, prec=prec, stream=self.stream.cuda_stream, nz=n if self.d3 else 1,
                                 lz=n * dy if self.d3 else 0.0)
            shape = (capacity, n, n, n) if self.d3 else (capacity, n, n)
            z = torch.zeros(shape, dtype=torch.float64, device=device)
            self.u, self.v, self.p, self.fu, self.fv = [z.clone() for _ in range(5)]
            self.w, self.fw = (z.clone(), z.clone()) if self.d3 else (None, None)
            self.nu = torch.full((capacity,), 1e-2, dtype=torch.float64, device=device)
            self.fx = torch.zeros((capacity,), dtype=torch.float64, device=device)
            self.dt = torch.full((capacity,), DT, dtype=torch.float64, device=device)
            # slots holding a request; empty slots are skipped by the step's kernels
            self.active_mask = torch.zeros((capacity,), dtype=torch.uint8, device=device)
        self.slots = [None] * capacity
        self.ev0 = torch.cuda.Event(enable_timing=True)
        self.ev1 = torch.cuda.Event(enable_timing=True)
        self.pending_event = False

    def free_slots(self):
        return [i for i, r in enumerate(self.slots) if r is None]

    def active(self):
        return [i for i, r in enumerate(self.slots) if r is not None]

    def admit(self, slot, req):
        nu = 1.0 / req.re
        with torch.cuda.stream(self.stream):
            for t in (self.u, self.v, self.p, self.fu, self.fv, self.w, self.fw):
                if t is not None:
                    t[slot].zero_()
            self.nu[slot] = nu
            self.fx[slot] = 8.0 * nu if self.kind in ("channel", "channel3d") else 0.0
            self.dt[slot] = request_dt(req)
            self.active_mask[slot] = 1
        self.slots[slot] = req

    def step(self):
        """Queue one RK3 step of every slot on this class's stream."""
        with torch.cuda.stream(self.stream):
            self.ev0.record(self.stream)
            self.ctx.isph_step(self.u, self.v, self.p, self.fu, self.fv, 1, nu=1e-2, rho=1.0, dt=DT,
                               u_top=1.0 if self.kind == "cavity" else 0.0, scheme="rk3", use_graph=True,
                               nu_inst=self.nu, fx_inst=self.fx, w=self.w, fw=self.fw, active=self.active_mask,
                               dt_inst=self.dt)
            self.ev1.record(self.stream)
        self.pending_event = True

    def finish_tick(self, now):
        """Wait for this tick's step, account latency, retire finished requests."""
        retired = []
        if not self.pending_event:
            return retired
        self.ev1.synchronize()
        ms = self.ev0.elapsed_time(self.ev1)
        self.pending_event = False
        for i in self.active():
            r = self.slots[i]
            r.done_steps += 1
            r.latencies_ms.append(ms)
            if r.done_steps >= r.steps:
                r.result = {"u": self.u[i].cpu().numpy(), "v": self.v[i].cpu().numpy(), "p": self.p[i].cpu().numpy()}
                if self.d3:
                    r.result["w"] = self.w[i].cpu().numpy()
                r.t_done = now
                self.slots[i] = None
                with torch.cuda.stream(self.stream):
                    self.active_mask[i] = 0
                retired.append(r)
        return retired


class Server:
    def __init__(self, prec="f64", capacity=8, mem_budget=None, device=None, fc_cont=25):
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.prec = prec
        self.capacity = capacity
        assert fc_cont == "smooth" or isinstance(fc_cont, int)
        self.fc_cont = fc_cont
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            mem_budget = int(0.8 * free)
        self.mem_budget = mem_budget
        self.classes = collections.OrderedDict()
        self.queue = collections.deque()
        self.done = []

    def n_cont(self, n):
        return smooth_n_cont(n) if self.fc_cont == "smooth" else self.fc_cont

    def used_bytes(self):
        return sum(footprint_bytes(c.n, c.capacity, c.prec, c.d3, c.n_cont) for c in self.classes.values())

    def submit(self, req):
        self.queue.append(req)

    def _admit(self, now):
        waiting = collections.deque()
        while self.queue:
            req = self.queue.popleft()
            key = class_key(req)
            cls = self.classes.get(key)
            if cls is None:
                need = footprint_bytes(req.n, self.capacity, self.prec, req.kind == "channel3d", self.n_cont(req.n))
                if self.used_bytes() + need > self.mem_budget:
                    waiting.append(req)
                    continue
                cls = SizeClass(key, self.capacity, self.prec, self.device, self.n_cont(req.n))
                self.classes[key] = cls
            free = cls.free_slots()
            if not free or cls.pending_event:
                # a class in flight takes new requests when its step is done
                waiting.append(req)
                continue
            req.t_admit = now
            cls.admit(free[0], req)
        self.queue = waiting

    def _evict_idle(self):
        """Drop classes with no active slot and no queued request, freeing their memory."""
        wanted = {class_key(r) for r in self.queue}
        for key in list(self.classes):
            c = self.classes[key]
            if not c.active() and not c.pending_event and key not in wanted:
                del self.classes[key]

    def tick(self, now, block=False):
        """Retire the classes whose step is done, admit queued requests, and
        launch the next step of every idle class with active slots.  With
        block=True it first waits for every class in flight.  Returns the
        number of classes in flight after the call."""
        for c in self.classes.values():
            if c.pending_event and (block or c.ev1.query()):
                self.done.extend(c.finish_tick(now))
        self._admit(now)
        for c in self.classes.values():
            if not c.pending_event and c.active():
                c.step()
        if self.queue:
            self._evict_idle()
            self._admit(now)
        return sum(1 for c in self.classes.values() if c.pending_event)

    def idle(self):
        return not self.queue and not any(c.active() or c.pending_event for c in self.classes.values())

    def run(self, requests, time_scale=1.0, max_wall=None):
        """Drive arrivals in (scaled) real time until every request finishes."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        k = 0
        while k < len(pending) or not self.idle():
            now = (time.perf_counter() - t0) / time_scale
            while k < len(pending) and pending[k].arrival <= now:
                self.submit(pending[k])
                k += 1
            inflight = self.tick(now)
            if inflight == 0 and k < len(pending) and not self.queue:
                time.sleep(max(0.0, (pending[k].arrival - now) * time_scale))
            elif inflight:
                time.sleep(5e-5)  # poll the classes' events again shortly
            if max_wall and time.perf_counter() - t0 > max_wall:
                break
        return time.perf_counter() - t0


class NativeServer:
    """The same serving loop run by the library's own scheduler (fcsph_batch_*
    in include/fcsph.h): size classes, slots, admission by footprint and the
    per-class streams live in C++; this class only submits requests, ticks
    the batch and collects results and step latencies (same interface as
    Server)."""

    def __init__(self, prec="f64", capacity=8, mem_budget=None, device=None, fc_cont=25, persistent=False,
                 size_priorities=False):
        """persistent: every tick steps all classes in one persistent launch (2D requests; FP64 / FP32x2).
        size_priorities: larger classes step on higher-priority streams."""
        self.prec = prec
        self.capacity = capacity
        self.fc_cont = fc_cont
        self.batch = b.Batch(prec=prec, slots=capacity, mem_budget=0.0 if mem_budget is None else mem_budget,
                             n_cont=fc_cont)
        if persistent:
            self.batch.set_persistent(True)
        if size_priorities:
            self.batch.set_size_priorities(True)
        self.live = {}     # library id -> Request
        self.done = []

    def submit(self, req):
        rid = self.batch.add(req.kind, req.n, req.re, req.steps)
        req.t_admit = None
        self.live[rid] = req

    def tick(self, now, block=False):
        inflight = self.batch.run(block=block)
        for rid in list(self.live):
            req = self.live[rid]
            info = self.batch.poll(rid)
            while req.done_steps < info["done_steps"]:
                req.done_steps += 1
                req.latencies_ms.append(info["last_step_ms"])
            if req.t_admit is None and info["state"] != "queued":
                req.t_admit = now
            if info["state"] == "done":
                req.result = self.batch.result(rid, req.kind, req.n)
                req.t_done = now
                self.done.append(req)
                del self.live[rid]
        return inflight

    def idle(self):
        return not self.live

    def run(self, requests, time_scale=1.0, max_wall=None):
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        k = 0
        while k < len(pending) or not self.idle():
            now = (time.perf_counter() - t0) / time_scale
            while k < len(pending) and pending[k].arrival <= now:
                self.submit(pending[k])
                k += 1
            inflight = self.tick(now)
            if inflight == 0 and k < len(pending) and self.idle():
                time.sleep(max(0.0, (pending[k].arrival - now) * time_scale))
            elif inflight:
                time.sleep(5e-5)
            if max_wall and time.perf_counter() - t0 > max_wall:
                break
        return time.perf_counter() - t0

    def close(self):
        self.batch.close()


def summarize(requests, wall_s):
    lat = np.concatenate([np.asarray(r.latencies_ms) for r in requests if r.latencies_ms]) if requests else np.zeros(0)
    updates = sum(particles(r) * r.done_steps for r in requests)
    return {"requests": len(requests), "finished": sum(1 for r in requests if r.result is not None),
            "particle_updates": updates, "wall_s": wall_s, "particle_updates_per_s": updates / wall_s if wall_s else None,
            "step_latency_ms_p50": float(np.percentile(lat, 50)) if lat.size else None,
            "step_latency_ms_p99": float(np.percentile(lat, 99)) if lat.size else None}


# ---------------------------------------------------------------- several GPUs
def place_requests(requests, world_size, prec="f64", fc_cont=25):
    """Placement of independent requests on `world_size` ranks (one GPU each):
    in arrival order, each request goes to the rank whose placed device
    footprint (one slot of the request's size class per request) is
    smallest, the lower rank on a tie.  Returns (per-rank request lists,
    per-rank footprint bytes).  The solves are independent, so ranks
    exchange nothing while they run."""
    load = [0] * world_size
    out = [[] for _ in range(world_size)]
    for r in sorted(requests, key=lambda q: (q.arrival, q.rid)):
        nc = smooth_n_cont(r.n) if fc_cont == "smooth" else fc_cont
        need = footprint_bytes(r.n, 1, prec, r.kind == "channel3d", nc)
        k = min(range(world_size), key=lambda i: (load[i], i))
        out[k].append(r)
        load[k] += need
    return out, load


def serve_on_ranks(requests, rank, world_size, make_server, time_scale=1.0):
    """Serves this rank's share of `requests` (place_requests) with its own
    Server (make_server() builds it on this rank's device) and gathers every
    rank's finished requests on rank 0 through torch.distributed (host
    objects, once at the end).  Rank 0 returns (all requests ordered by rid,
    per-rank wall seconds); the other ranks return (None, None)."""
    import torch.distributed as dist
    srv = make_server()
    parts, _ = place_requests(requests, world_size, srv.prec, srv.fc_cont)
    mine = parts[rank]
    wall = srv.run(mine, time_scale=time_scale) if mine else 0.0
    payload = {"wall_s": wall,
               "requests": [dict(rid=r.rid, kind=r.kind, n=r.n, re=r.re, steps=r.steps, arrival=r.arrival,
                                 done_steps=r.done_steps, latencies_ms=list(r.latencies_ms), result=r.result,
                                 rank=rank) for r in mine]}
    gathered = [None] * world_size if rank == 0 else None
    dist.gather_object(payload, gathered, dst=0)
    if rank != 0:
        return None, None
    done = []
    for g in gathered:
        for d in g["requests"]:
            r = Request(d["rid"], d["kind"], d["n"], d["re"], d["steps"], d["arrival"])
            r.done_steps, r.latencies_ms, r.result = d["done_steps"], d["latencies_ms"], d["result"]
            r.rank = d["rank"]
            done.append(r)
    return sorted(done, key=lambda r: r.rid), [g["wall_s"] for g in gathered]
