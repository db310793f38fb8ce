"""Benchmark of the FC spectral ISPH hot path on GB300 (one JSON line).

Workload: 2D lid-driven square cavity, 256 x 256 particles, walls on all four
sides with FC(Gram) d=5, C=25 continuation in x and y (281 x 281 extended
grid), Re = 1000 (lid velocity 1, nu = 1e-3), G8 kernel with h = 1.3 dx,
low-storage RK3 (3 projection substeps per step), dt = 1e-3, fluid at rest at
t = 0.  A batch of B independent instances is advanced together (device
resident state, one CUDA graph per step).  One bench step = one RK3 ISPH step
of every instance.  The metric is particle-updates/s = B * 256^2 * steps / s.

The headline path is the mixed one at equal L2: transforms, symbols and FC
sums in FP32 pairs (FP32x2, 48-bit significand, FP32 units), state and
epilogues in FP64.  Beside it: the plain FP64 path batched and as a single
solve (batch 1), and FP32 transforms, each with its L2 against the FP64 path
on the cavity and against the analytic start-up series on the 64^2 channel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--prec f32x2|f64|f32]
  python bench.py --impl reference ...   # the FP64 CPU oracle (numpy) on the same workload

Under torchrun each rank runs its own batch on its own GPU (independent
instances, no data-path collective; weak scaling); rank 0 prints the line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/s per ISPH step, served-mixed vs plain FP64 at equal L2; p50/p99"
N = 256
NU, DT, LID = 1e-3, 1e-3, 1.0
FAMILY, HDX = "G8", 1.3
N_MATCH, N_CONT = 5, 25
PROF_KINDS = ["col_fwd", "row_mom", "row_div", "row_grad", "row_op", "col_mom", "col_div", "col_corr", "col_out",
              "row_ppe", "col_ppe", "other"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--prec", default="f32x2", choices=["f32", "f64", "f32x2"])
    ap.add_argument("--refine", type=int, default=0)
    ap.add_argument("--tiling", default=None,
                    help="rows,pairs per CTA for the headline context instead of the autotuner (profiling runs)")
    ap.add_argument("--cta-threads", default=None,
                    help="with --tiling: row,column CTA widths of the headline context (profiling runs)")
    ap.add_argument("--groups", type=int, default=None,
                    help="with --tiling: instance groups of the step graph (profiling runs)")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--workload", default="cavity", choices=["cavity", "uneven", "serve", "planes", "lines", "dipole", "channel3d"],
                    help="cavity: the 256^2 lid cavity (default); uneven: 64 solves of sizes 64^2..512^2 "
                         "submitted together; serve: a Poisson request stream (2D part)")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--slots", type=int, default=8, help="uneven/serve: slots (batch) per size class")
    ap.add_argument("--server", default="native", choices=["native", "python"],
                    help="uneven/serve: the library's scheduler (fcsph_batch_*) or the Python one")
    ap.add_argument("--size-priorities", action="store_true",
                    help="uneven/serve (native scheduler): larger size classes on higher-priority streams")
    ap.add_argument("--persistent", action="store_true",
                    help="uneven/serve (native scheduler, 2D requests): every tick steps all size classes in one "
                         "persistent launch instead of one graph per class; with --profile-case: two cavity "
                         "steps as persistent launches")
    ap.add_argument("--fc-cont", default="25",
                    help="uneven/serve: FC continuation length of every size class, an integer or 'smooth' (per size "
                         "the length nearest 25 in [20, 40] whose extended line the engine transforms directly)")
    ap.add_argument("--plane-cont", type=int, default=26,
                    help="--profile-case --workload planes: FC continuation length (26: n_e = 1050; 25: 1049)")
    ap.add_argument("--profile-case", action="store_true",
                    help="no timing: 2 eager RK3 steps of the cavity, or (--workload planes) 3 spectral_op calls "
                         "on --batch planes of 1024^2, for ncu captures on a small batch")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-microbench", action="store_true",
                    help="skip the plane and line operator microbenchmarks of the default run")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def max_over_ranks(x, ws, device="cpu"):
    """The largest per-rank value (the slowest rank's time) on every rank."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ws, t_max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * ws / (t_max_ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- byte model
def kernel_bytes(kind, nx, ny, hy, cb, batch):
    """Algorithmic bytes one launch of each kernel kind must move (whole batch):
    its spectra in/out at the context's complex size cb and the FP64 fields it
    reads/writes.  Intermediates kept on chip inside the kernel do not count."""
    S = hy * nx * cb        # one half-spectrum (rows ky < hy)
    P = ny * nx * cb        # one PPE (DCT-y) spectrum (rows l < ny)
    F = nx * ny * 8         # one FP64 field
    per = {
        "col_fwd": 2 * F + 2 * S,
        "row_mom": 8 * S,
        "row_div": 3 * S,
        "row_grad": 3 * S,
        "col_mom": 6 * S + 4 * F + 4 * F + 2 * S,
        "col_div": S + F + P,
        "col_corr": 2 * S + 2 * F + 2 * F + 2 * S,
        "row_ppe": 2 * P,
        "col_ppe": P + F + S,
    }
    return per.get(kind, 0) * batch


def kernel_flops(kind, nx, ny, my, mx, hy, px, batch, split_fields=True):
    """Algorithmic flops of one launch (whole batch): 5 n log2 n per complex
    length-n transform (the textbook FFT count, whatever algorithm realises
    it), for the line transforms each kernel kind performs.  Column kernels
    transform packed pairs of columns (nx/2 lines per field), row kernels hy
    rows per spectrum; PPE lines have length 2(ny-1) (y) and px (x)."""
    F = lambda n: 5.0 * n * math.log2(n) if n > 1 else 0.0
    pairs = (nx + 1) // 2
    my_p = 2 * (ny - 1)
    per = {
        "col_fwd": 2 * pairs * F(my),
        "row_mom": (1 + 3) * hy * F(mx) if split_fields else (2 + 6) * hy * F(mx),
        "row_div": 3 * hy * F(mx),
        "row_grad": 3 * hy * F(mx),
        "col_mom": 8 * pairs * F(my),
        "col_div": pairs * (F(my) + F(my_p)),
        "col_corr": 4 * pairs * F(my),
        "row_ppe": 2 * ny * F(px),
        "col_ppe": pairs * (F(my_p) + F(my)),
    }
    return per.get(kind, 0.0) * batch


def _startup_series(y, t, F, nu, nterms=199):
    """Channel flow from rest under body force F (walls at y = 0, 1): the
    Poiseuille profile minus its decaying sine series."""
    import numpy as np
    u = F / (2 * nu) * y * (1 - y)
    for n in range(1, nterms, 2):
        u = u - 4 * F / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * y) * np.exp(-nu * n * n * np.pi ** 2 * t)
    return u


def channel_analytic_l2(b, torch, dev):
    """64^2 Poiseuille channel (G4, h = 1.3 dx, nu = 0.1, F = 0.8, FOP, dt = 1e-3,
    100 steps from rest with 1e-6 seeded noise): relative L2 error of u against
    the analytic start-up series, for each transform precision."""
    import numpy as np
    from paper_2606_06247_gb300 import inputs
    n = 64
    u0, v0 = inputs.channel_initial(n, n, seed=1, sigma=1e-6)
    ua = np.tile(_startup_series(np.linspace(0, 1, n), 0.1, 0.8, 0.1), (n, 1))
    out = {}
    for pr in ("f64", "f32x2", "f32"):
        ctx = b.Context(n, n, n / (n - 1), 1.0, family="G4", h_over_dx=1.3, prec=pr)
        u = torch.tensor(u0[None], dtype=torch.float64, device=dev)
        v = torch.tensor(v0[None], dtype=torch.float64, device=dev)
        p, fu, fv = torch.zeros_like(u), torch.zeros_like(u), torch.zeros_like(u)
        ctx.isph_step(u, v, p, fu, fv, 100, nu=0.1, rho=1.0, dt=1e-3, force=(0.8, 0.0), scheme="fop")
        ctx.sync()
        uh = u[0].cpu().numpy()
        out[pr] = float(np.linalg.norm(uh - ua) / np.linalg.norm(ua))
    return out


def fp64_peak_tflops(sm_mhz=2070.0):
    """GB300 FP64 issue rate: 152 SMs x 2 FP64 FMA lanes x 2 flops x clock."""
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


def fp32_peak_tflops(sm_mhz=2070.0):
    """GB300 FP32 FMA rate: 152 SMs x 128 FP32 lanes x 2 flops x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# FP32 instructions per algorithmic flop of FP32-pair arithmetic, counted on
# the radix-2 butterfly (1 complex multiply + 2 complex adds = 10 flops): a
# pair add is 11 FP32 instructions (TwoSum 6, low-part adds 2, Fast2Sum 3), a
# pair multiply 7 (product, 3 FMAs, Fast2Sum 3); 4 multiplies + 6 adds = 94.
# Used only for the issue-efficiency figure (FP32 instructions the achieved
# pair-flop rate implies, over the FP32 lane issue rate), not as a peak.
FF_INST_PER_FLOP = 94 / 10


def fp32_lane_inst_rate(sm_mhz=2070.0):
    """FP32 instructions per second over all lanes: 152 SMs x 128 lanes x clock."""
    return 152 * 128 * sm_mhz * 1e6


# Algorithmic bytes per particle-update of one FOP substep (the four fused
# passes u,v -> u*,v*; u*,v* -> b; b -> phi; phi,u*,v* -> u,v, each reading
# and writing its fields once): 72 B with FP32 transforms and spectra held
# on chip, 112 B for plain FP64.  An RK3 step is three substeps.
STEP_BYTES_PER_UPDATE = {"f32": 72, "f32x2": 72, "f64": 112}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a kernel kind, from one ncu
# capture of `bench.py --profile-case --batch B --prec P` (first RK3 substep; command and table in
# profiles/), keyed by (precision, kind, batch).  Valid only for the device code they were taken on:
# KERNEL_SOURCES_SHA256 is kernel_sources_sha256() at capture time, and a different hash reports null.
MEASURED_TRAFFIC = {
    ("f32x2", "row_mom", 32): 91674880, ("f32x2", "col_mom", 32): 238897152,
    ("f64", "row_mom", 32): 84284928, ("f64", "col_mom", 32): 248863232,
    ("f32", "row_mom", 32): 21544448, ("f32", "col_mom", 32): 164872960,
}
KERNEL_SOURCES_SHA256 = "19a1f5682d47932420e19b5ae1d03b2570af3564fdbb409813b5a647a3d0ff08"


def kernel_sources_sha256():
    """SHA-256 of the device code in csrc/ (.cu, .cuh, .h) with comments and
    blank space removed, so that a comment edit keeps the recorded counters."""
    import hashlib
    import re
    d = os.path.join(ROOT, "paper_2606_06247_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(d, name)) as f:
                src = f.read()
            src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
            src = re.sub(r"//[^\n]*", " ", src)
            h.update(name.encode() + b"\0" + " ".join(src.split()).encode())
    return h.hexdigest()


def measured_traffic(prec, kind, batch):
    """(bytes per launch or None, note)."""
    v = MEASURED_TRAFFIC.get((prec, kind, batch))
    if v is None:
        return None, "no ncu capture for this precision, kernel and batch"
    if kernel_sources_sha256() != KERNEL_SOURCES_SHA256:
        return None, "kernel sources changed since the ncu capture"
    return v, "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------- CPU oracle
class OracleCavity:
    """The FP64 oracle (numpy) on one 256^2 cavity instance; built once, stepped on demand."""

    def __init__(self, n=N):
        import numpy as np
        from oracle import fc as ofc
        from oracle import step as ostep
        self.ostep = ostep
        E = ofc.gram_table(N_MATCH, N_CONT)
        self.p = ostep.Problem(nx=n, ny=n, Lx=1.0, Ly=1.0, x_walls=True, family=FAMILY, h_over_dx=HDX, E_dir=E,
                               E_neu=E, nu=NU, rho=1.0, dt=DT, u_top=LID, scheme="rk3").build_symbols()
        self.u = np.zeros((n, n))
        self.v = np.zeros((n, n))

    def step(self):
        t0 = time.perf_counter()
        self.u, self.v, _ = self.ostep.isph_steps(self.p, self.u, self.v, 1)
        return time.perf_counter() - t0


def oracle_rate(seconds, n=N):
    """Particle-updates/s of the oracle over >= 1 step and about `seconds` of stepping."""
    oc = OracleCavity(n)
    oc.step()  # first step outside the timing
    el, steps = 0.0, 0
    while steps == 0 or el < seconds:
        el += oc.step()
        steps += 1
    return n * n * steps / el, steps, el


def cpu_cores():
    """Host cores this process may run on: the oracle's dense DFT products go
    through numpy's BLAS, whose thread pool spans them."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


# ---------------------------------------------------------------- main (ours)
def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    from paper_2606_06247_gb300 import binding as b

    B = args.batch
    dy = 1.0 / (N - 1)
    stream = torch.cuda.current_stream()

    def make(prec, refine):
        return b.Context(N, N, 1.0, 1.0, x_walls=True, batch=B, n_match=N_MATCH, n_cont=N_CONT, family=FAMILY,
                         h_over_dx=HDX, prec=prec, refine=refine)

    def state():
        z = torch.zeros((B, N, N), dtype=torch.float64, device=dev)
        return [z.clone() for _ in range(5)]

    prm = dict(nu=NU, rho=1.0, dt=DT, u_top=LID, scheme="rk3")

    def timed(ctx, st, steps, warmup):
        u, v, p, fu, fv = st
        ctx.isph_step(u, v, p, fu, fv, warmup, use_graph=True, **prm)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        n0 = ctx.launch_count
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            ev[0].record(stream)
            for k in range(steps):
                ctx.isph_step(u, v, p, fu, fv, 1, use_graph=True, **prm)
                ev[k + 1].record(stream)
            torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        launches = ctx.launch_count - n0
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
        total = ev[0].elapsed_time(ev[steps])
        return total, per, launches, clk.summary()

    # ---- headline: the chosen precision, batched, device resident
    ctx = make(args.prec, args.refine if args.prec == "f32" else 0)
    if args.tiling:
        ctx.set_tiling(*[int(x) for x in args.tiling.split(",")])
        if args.cta_threads:
            ctx.set_cta_threads(*[int(x) for x in args.cta_threads.split(",")])
        if args.groups:
            ctx.set_step_groups(args.groups)
    else:
        ctx.autotune(steps=4, **prm)
    dtype_name = {"f64": "f64", "f32x2": "f32x2", "f32": "f32"}[args.prec]
    st = state()
    total_ms, per_ms, launches, clocks = timed(ctx, st, args.steps, args.warmup)
    t_max = max_over_ranks(total_ms, ws, dev)
    value = job_rate(B * N * N * args.steps, ws, t_max)

    # ---- per-kernel durations (eager launches, events on the launching stream)
    ctx.set_profiling(True)
    u, v, p, fu, fv = st
    ctx.isph_step(u, v, p, fu, fv, max(2, min(args.steps, 5)), use_graph=False, **prm)
    prof = ctx.get_profile()
    ctx.set_profiling(False)
    cb = 8 if args.prec == "f32" else 16
    hy = (N + N_CONT) // 2 + 1
    kinds = {k: dict(ms=v_[0], launches=v_[1], avg_ms=v_[0] / v_[1]) for k, v_ in prof.items()}
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    peaks, peak_src = load_peaks()
    for k, d in kinds.items():
        by = kernel_bytes(k, N, N, hy, cb, B)
        d["alg_bytes"] = by
        d["gbs"] = by / (d["avg_ms"] * 1e-3) / 1e9 if by else None
    my, mx = N + N_CONT, N + N_CONT
    px = 2 * (N - 1)
    # the momentum row pass runs once per field when one row set exceeds the shared-memory budget
    split = kinds.get("row_mom", {}).get("launches", 0) > kinds.get("row_div", {}).get("launches", 0)
    for k, d in kinds.items():
        fl = kernel_flops(k, N, N, my, mx, hy, px, B, split)
        d["alg_gflop"] = fl / 1e9
        d["gflops"] = fl / (d["avg_ms"] * 1e-3) / 1e9 if fl else None
    traffic, traffic_note = measured_traffic(args.prec, dom, B)
    clk_mhz = peaks.get("sm_max_mhz", 2070.0)
    if args.prec in ("f64", "f32x2"):
        if args.prec == "f64":
            pk = fp64_peak_tflops(clk_mhz) * 1e3
            src = "derived: 152 SMs x 2 FP64 FMA lanes x 2 flop x max SM clock"
        else:
            pk = fp32_peak_tflops(clk_mhz) * 1e3
            src = ("derived: 152 SMs x 128 FP32 FMA lanes x 2 flop x max SM clock (FP32-pair flops counted as "
                   "flops, 5 n log2 n per transform)")
        roof = {"kernel": dom, "bound": "alu", "achieved": kinds[dom]["gflops"], "peak": pk, "unit": "GFLOP/s",
                "frac": (kinds[dom]["gflops"] or 0) / pk, "traffic": traffic, "traffic_source": traffic_note,
                "peak_source": src,
                "alg_gflop_per_launch": kinds[dom]["alg_gflop"], "avg_launch_ms": kinds[dom]["avg_ms"],
                "hbm_gbs_alg": kinds[dom]["gbs"], "hbm_frac_of_measured": (kinds[dom]["gbs"] or 0) / peaks["hbm_gbs"]}
        if args.prec == "f32x2":
            roof["issue_efficiency"] = ((kinds[dom]["gflops"] or 0) * 1e9 * FF_INST_PER_FLOP
                                        / fp32_lane_inst_rate(clk_mhz))
            roof["issue_efficiency_note"] = (f"FP32 instructions implied by the achieved pair-flop rate at "
                                             f"{FF_INST_PER_FLOP} per flop (radix-2 butterfly count), over 152 x 128 "
                                             "FP32 lanes x max SM clock")
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": kinds[dom]["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": (kinds[dom]["gbs"] or 0) / peaks["hbm_gbs"], "traffic": traffic, "traffic_source": traffic_note,
                "peak_source": peak_src + " hbm_gbs", "alg_bytes_per_launch": kinds[dom]["alg_bytes"],
                "avg_launch_ms": kinds[dom]["avg_ms"]}
    step_bytes = B * N * N * 3 * STEP_BYTES_PER_UPDATE[args.prec]
    step_gbs = step_bytes / (t_max / args.steps * 1e-3) / 1e9
    roof["step"] = {"alg_bytes_per_particle_update": 3 * STEP_BYTES_PER_UPDATE[args.prec],
                    "alg_bytes_per_step": step_bytes, "alg_GBps": step_gbs, "frac_of_hbm": step_gbs / peaks["hbm_gbs"],
                    "note": (f"{STEP_BYTES_PER_UPDATE[args.prec]} B per particle-update per FOP substep x 3 RK3 "
                             "substeps over ms_per_step, against the measured HBM copy rate")}
    prof_total = sum(d["ms"] for d in kinds.values())
    for d in kinds.values():
        d["share"] = d["ms"] / prof_total

    # ---- e2e through the C ABI with host buffers (pinned), copies inside the timed region
    hu = torch.zeros((B, N, N), dtype=torch.float64).pin_memory()
    hv = torch.zeros_like(hu).pin_memory()
    hu.copy_(st[0].cpu())
    hv.copy_(st[1].cpu())
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        u.copy_(hu, non_blocking=True)
        v.copy_(hv, non_blocking=True)
        ctx.isph_step(u, v, p, fu, fv, 1, use_graph=True, **prm)
        hu.copy_(u, non_blocking=True)
        hv.copy_(v, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e = {"value": B * N * N / (e2e_ms / 1e3), "unit": "particle-updates/s",
           "h2d_bytes_per_step": 2 * B * N * N * 8, "d2h_bytes_per_step": 2 * B * N * N * 8}

    # ---- the other precisions on the same workload: throughput (plain FP64
    # batched and as a single solve, FP32), and each path's relative L2 against
    # the FP64 path after 20 steps from the same start; then the 64^2 channel's
    # L2 error against the analytic start-up series for every precision
    compare = None
    if not args.no_compare:
        compare = {}
        nsteps_cmp = 20
        rel = lambda a, r: float(torch.sqrt(((a - r) ** 2).sum() / (r ** 2).sum().clamp_min(1e-300)).item())
        finals = {}
        for pr in ("f64", "f32x2", "f32"):
            c2 = ctx if pr == args.prec else make(pr, 0)
            if pr != args.prec:
                c2.autotune(steps=4, **prm)
                st2 = state()
                n2 = max(2, args.steps // 2)
                t2, _, _, _ = timed(c2, st2, n2, 1)
                compare[f"{pr}_value"] = B * N * N * n2 / (t2 / 1e3)
                compare[f"{pr}_ms_per_step"] = t2 / n2
                compare[f"{pr}_tiling"] = list(c2.get_tiling())
                compare[f"{pr}_cta_threads"] = list(c2.get_cta_threads())
                compare[f"{pr}_step_groups"] = c2.get_step_groups()
            sa = state()
            c2.isph_step(*sa, nsteps_cmp, use_graph=True, **prm)
            torch.cuda.synchronize()
            finals[pr] = sa
            if c2 is not ctx:
                del c2
        # plain FP64 single solve: one instance per context
        c1 = b.Context(N, N, 1.0, 1.0, x_walls=True, batch=1, n_match=N_MATCH, n_cont=N_CONT, family=FAMILY,
                       h_over_dx=HDX, prec="f64")
        c1.autotune(steps=3, **prm)
        z1 = torch.zeros((1, N, N), dtype=torch.float64, device=dev)
        st1 = [z1.clone() for _ in range(5)]
        n1 = max(5, args.steps)
        t1, _, _, _ = timed(c1, st1, n1, 2)
        compare["f64_single_value"] = N * N * n1 / (t1 / 1e3)
        compare["f64_single_ms_per_step"] = t1 / n1
        compare["speedup_vs_f64_single"] = value / compare["f64_single_value"]
        del c1, st1
        uv = lambda s_: torch.stack([s_[0], s_[1]])
        for pr in ("f32x2", "f32"):
            lu, lv = rel(finals[pr][0], finals["f64"][0]), rel(finals[pr][1], finals["f64"][1])
            compare[f"rel_l2_u_{pr}_vs_f64_after_{nsteps_cmp}_steps"] = lu
            compare[f"rel_l2_v_{pr}_vs_f64_after_{nsteps_cmp}_steps"] = lv
            compare[f"rel_l2_velocity_{pr}_vs_f64_after_{nsteps_cmp}_steps"] = rel(uv(finals[pr]), uv(finals["f64"]))
        del finals
        ch = channel_analytic_l2(b, torch, dev)
        compare["channel64_l2_vs_analytic"] = ch
        for pr in ("f32x2", "f32"):
            cav = compare[f"rel_l2_velocity_{pr}_vs_f64_after_{nsteps_cmp}_steps"] < 1e-6
            chan = abs(ch[pr] - ch["f64"]) <= 1e-6 * ch["f64"]
            compare[f"{pr}_equal_l2"] = bool(cav and chan)
        compare["equal_l2_bar"] = ("cavity: velocity relative L2 against the FP64 path < 1e-6 after 20 steps; "
                                   "channel 64^2 (FOP, 100 steps): L2 error against the analytic start-up series "
                                   "equal to the FP64 path's to 1e-6 relative")
        compare["note"] = ("FP32 transforms of the doubly FC-extended lid-corner data lose accuracy; FP32-pair "
                           "transforms keep a 48-bit significand")
        if args.prec != "f64":
            compare["headline_equal_l2"] = compare.get(f"{args.prec}_equal_l2")

    # ---- the operator microbenchmarks (FP32 fields) at full size, rank 0 at N = 1:
    # 256 planes of 1024^2 (spectral_op DX+DY+LAP, per-pass algorithmic GB/s) and
    # 4096 lines of 512 (line_op DY+LAP, one fused kernel)
    micro = None
    if rank == 0 and ws == 1 and not args.no_microbench:
        torch.cuda.empty_cache()
        planes, _ = measure_planes(max(3, min(args.steps, 5)), 3)
        lines, _ = measure_lines(max(8, args.steps), 3, precs=(("f32", 25), ("f32", 28)))
        micro = {"planes_256x1024x1024_f32": planes, "lines_4096x512_f32": lines,
                 "peak": peaks["hbm_gbs"], "peak_source": peak_src + " hbm_gbs",
                 "note": ("algorithmic bytes: planes 4 B in + 3 x 4 B out per node per call and each pass's own "
                          "reads and writes; lines 4 B in + 2 x 4 B out per node")}

    # ---- CPU baseline (oracle), rank 0 only
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, nst, el = oracle_rate(args.cpu_seconds)
        cpu = {"value": rate, "unit": "particle-updates/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"FP64 numpy oracle, 1 instance x {nst} RK3 steps of the 256^2 cavity ({el:.1f} s)"}

    if rank == 0:
        per_sorted = sorted(per_ms)
        line = {
            "metric": METRIC, "value": value, "unit": "particle-updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_name, "data": "synthetic",
            "path": {"f64": "plain FP64", "f32x2": "FP32-pair transforms (48-bit significand), FP64 state",
                     "f32": "mixed (FP32 transforms)"}[args.prec],
            "config": dict(cavity_config(B, ws),
                           precision={"f32": ("FP32 FFT/symbols, FP32-pair FC sums, FP64 state and PPE residual, "
                                              f"{args.refine} refinement sweeps"),
                                      "f32x2": "FP32-pair (double-float) FFT/symbols/FC sums, FP64 state",
                                      "f64": "FP64"}[args.prec],
                           tiling=list(ctx.get_tiling()), cta_threads=list(ctx.get_cta_threads()),
                           step_groups=ctx.get_step_groups(), step_persistent=ctx.get_step_persistent()),
            "latency_ms": {"p50": per_sorted[len(per_sorted) // 2], "p99": per_sorted[min(len(per_sorted) - 1, int(0.99 * len(per_sorted)))]},
            "roofline": roof,
            "kernels": kinds,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "compare": compare,
            "operator_microbench": micro,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def cavity_config(B, ws):
    """The headline workload's config, shared by both arms."""
    return {"workload": f"lid-driven cavity {N}x{N} Re=1000, FC(Gram) d=5 C=25 on x and y, "
                        f"G8 h=1.3dx, RK3 dt=1e-3, batch of {B} instances", "batch": B, "nx": N, "ny": N,
            "l2": f"inputs larger than L2 (state + workspace {B * N * N * 8 * 11 / 2**20:.0f} MiB)",
            "parallelism": f"replicas x{ws}"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    oc = OracleCavity()
    for _ in range(args.warmup):
        oc.step()
    times = [oc.step() for _ in range(args.steps)]
    total = sum(times)
    value = N * N * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cavity_config(args.batch, ws), precision="FP64 numpy oracle on the host cores"),
            "cpu_baseline": {"value": value, "unit": "particle-updates/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": (f"bounded sample: each step advances 1 of the {args.batch} instances by one RK3 "
                                        f"step ({args.steps} steps after {args.warmup} warm-up); rate per "
                                        "particle-update")},
            "e2e": {"value": value, "unit": "particle-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_serving(args):
    """The uneven batch and the Poisson request stream through the continuous-
    batching server, and the same requests run one at a time on the plain FP64
    path (batch 1), both with the same FC continuation lengths."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06247_gb300 import inputs
    from paper_2606_06247_gb300.serve import NativeServer, Request, Server, summarize
    ServerCls = NativeServer if args.server == "native" else Server
    steps = args.steps
    if args.workload == "uneven":
        spec = inputs.uneven_batch(64, seed=2024)
        reqs = lambda: [Request(i, d["kind"], d["n"], d["re"], steps, 0.0) for i, d in enumerate(spec)]
        desc = (f"64 independent solves, sizes uniform on 64^2..512^2, Re log-uniform [100, 5000], even index cavity "
                f"(G8) / odd channel (G4 if Re < 625 else G8), {steps} RK3 steps each, submitted together")
    else:
        spec = inputs.poisson_requests(rate=200.0, duration=args.serve_seconds, seed=7, sizes=(64, 128, 256, 512, 1024),
                                       steps=(50, 500))
        reqs = lambda: [Request(i, d["kind"], d["n"], float(np.exp(np.random.default_rng(i).uniform(np.log(100), np.log(5000)))),
                                max(1, d["steps"] * steps // 500), d["t"]) for i, d in enumerate(spec)]
        desc = (f"Poisson arrivals 200/s for {args.serve_seconds} s, 80% 2D cavity/channel of 64^2..1024^2, "
                f"20% 3D channel of 64^3..128^3, each 50-500 RK3 steps scaled by {steps}/500")
    fc_cont = args.fc_cont if args.fc_cont == "smooth" else int(args.fc_cont)
    torch.cuda.synchronize()
    if args.persistent:
        if args.server != "native":
            raise SystemExit("--persistent needs the native scheduler")
        srv = ServerCls(prec=args.prec, capacity=args.slots, fc_cont=fc_cont, persistent=True)
    elif args.size_priorities:
        srv = ServerCls(prec=args.prec, capacity=args.slots, fc_cont=fc_cont, size_priorities=True)
    else:
        srv = ServerCls(prec=args.prec, capacity=args.slots, fc_cont=fc_cont)
    rs = reqs()
    wall = srv.run(rs)
    torch.cuda.synchronize()
    served = summarize(rs, wall)
    # serial baseline: plain FP64, one request at a time, batch 1
    base = reqs()
    t0 = time.perf_counter()
    for r in base:
        s1 = ServerCls(prec="f64", capacity=1, fc_cont=fc_cont)
        r.arrival = 0.0
        s1.submit(r)
        while not s1.idle():
            s1.tick(0.0)
    torch.cuda.synchronize()
    serial = summarize(base, time.perf_counter() - t0)
    # per-instance error of the served (mixed) result against the same request
    # on the plain FP64 path (which is at parity with the FP64 oracle): relative
    # L2 and L-infinity of the velocity
    per_inst = []
    for r, r0 in zip(rs, base):
        if r.result is None or r0.result is None:
            continue
        comps = ("u", "v", "w") if "w" in r.result else ("u", "v")
        a = np.stack([r.result[c] for c in comps])
        ref = np.stack([r0.result[c] for c in comps])
        nrm = max(float(np.linalg.norm(ref)), 1e-300)
        per_inst.append({"rid": r.rid, "kind": r.kind, "n": r.n, "re": r.re, "steps": r.steps,
                         "rel_l2_velocity": float(np.linalg.norm(a - ref)) / nrm,
                         "linf_velocity": float(np.abs(a - ref).max())})
    errs = sorted(d["rel_l2_velocity"] for d in per_inst)
    err_summary = {"instances": len(errs), "max_rel_l2": errs[-1] if errs else None,
                   "median_rel_l2": errs[len(errs) // 2] if errs else None,
                   "max_linf": max((d["linf_velocity"] for d in per_inst), default=None),
                   "reference": "the same request run alone on the plain FP64 path (batch 1)"}
    print(json.dumps({
        "metric": METRIC, "value": served["particle_updates_per_s"], "unit": "particle-updates/s", "n_gpus": 1,
        "steps": steps, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
        "config": {"workload": desc, "precision": args.prec, "slots_per_size_class": args.slots, "fc_cont": args.fc_cont,
                   "scheduler": args.server + (" persistent" if args.persistent else "")
                   + (" size-priorities" if args.size_priorities else "")},
        "latency_ms": {"p50": served["step_latency_ms_p50"], "p99": served["step_latency_ms_p99"]},
        "served": served, "serial_plain_fp64": serial,
        "error_vs_fp64": err_summary, "per_instance": per_inst,
        "speedup_vs_serial": served["particle_updates_per_s"] / serial["particle_updates_per_s"]}))


WIDTH_SWEEP = [(r, c) for r in (32, 64, 128) for c in (32, 64, 128)]


def plane_kernel_bytes(kind, P, nx, ny, hy, nout=3):
    """Algorithmic bytes of one launch of each pass of the FP32 plane operator
    (whole batch of P planes): the FP32 field in (col_fwd), the half-spectrum
    (hy rows of nx complex FP32) out of the y pass, into and nout spectra out
    of the x pass, and nout spectra in and FP32 fields out of the inverse y
    pass."""
    S = P * hy * nx * 8
    F = P * nx * ny * 4
    return {"col_fwd": F + S, "row_op": S + nout * S, "col_out": nout * S + nout * F}.get(kind, 0)


def measure_planes(steps, warmup, sweep_widths=True):
    """FC-extended operator microbench on 256 planes of 1024 x 1024 (x periodic,
    walls in y), FP32 fields, d/dx, d/dy and the Laplacian per call, for
    n_cont = 25 (n_e = 1049, Bluestein) and 26 (n_e = 1050).  Algorithmic bytes
    per call: 4 B in + 3 x 4 B out per node; per pass: each kernel's own
    reads and writes (plane_kernel_bytes), from CUDA events on the launching
    stream around every eager launch."""
    import numpy as np
    import torch
    from paper_2606_06247_gb300 import binding as b
    from paper_2606_06247_gb300 import inputs
    P, n = 256, 1024
    base = inputs.band_limited_planes(4, n, n, seed=12346, n_modes=64, max_mode=64)
    f = torch.tensor(np.tile(base, (P // 4, 1, 1)), dtype=torch.float32, device="cuda")
    outs = [torch.empty_like(f) for _ in range(3)]
    peaks, src = load_peaks()
    res = {}

    def call_ms(ctx, calls):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(calls):
            ctx.spectral_op(f, ["DX", "DY", "LAP"], outs)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / calls

    for n_cont in (25, 26):
        ctx = b.Context(n, n, n / (n - 1), 1.0, batch=P, n_cont=n_cont, family="G4", h_over_dx=1.3, prec="f32")
        sweep = {}
        if sweep_widths:  # CTA widths: a short sweep (row, column threads), then the timed calls at the fastest
            for w in WIDTH_SWEEP:
                ctx.set_cta_threads(*w)
                call_ms(ctx, 1)
                sweep[f"{w[0]},{w[1]}"] = call_ms(ctx, 2)
            best_w = min(sweep, key=sweep.get)
            ctx.set_cta_threads(*[int(x) for x in best_w.split(",")])
        call_ms(ctx, max(3, warmup))
        ms = call_ms(ctx, max(3, steps))
        gbs = P * n * n * 16 / (ms * 1e-3) / 1e9
        # per-pass durations (eager, events on the launching stream)
        ctx.set_profiling(True)
        for _ in range(3):
            ctx.spectral_op(f, ["DX", "DY", "LAP"], outs)
        prof = ctx.get_profile()
        ctx.set_profiling(False)
        hy = (n + n_cont) // 2 + 1
        passes = {}
        for k, (tms, cnt) in prof.items():
            by = plane_kernel_bytes(k, P, n, n, hy)
            avg = tms / cnt
            passes[k] = {"avg_ms": avg, "alg_bytes": by, "alg_GBps": by / (avg * 1e-3) / 1e9,
                         "frac_of_hbm": by / (avg * 1e-3) / 1e9 / peaks["hbm_gbs"]}
        res[f"n_cont={n_cont} (n_e={n + n_cont})"] = {
            "ms_per_call": ms, "alg_GBps": gbs, "frac_of_hbm": gbs / peaks["hbm_gbs"], "launches_per_call": 3,
            "cta_threads": list(ctx.get_cta_threads()), "width_sweep_ms": sweep, "passes": passes}
        del ctx
        torch.cuda.empty_cache()
    del f, outs
    torch.cuda.empty_cache()
    return res, src


def run_planes(args):
    import __graft_entry__
    __graft_entry__.build()
    lines, src = measure_planes(args.steps, args.warmup)
    best = max(v["alg_GBps"] for v in lines.values())
    print(json.dumps({"metric": "FC-extended spectral operator throughput (algorithmic HBM GB/s)", "value": best,
                      "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                      "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "256 planes of 1024x1024, x periodic, FC(Gram) d=5 in y, G4 h=1.3dx, "
                                             "spectral_op DX+DY+LAP, FP32 fields", "peak_source": src},
                      "variants": lines}))


def measure_lines(steps, warmup, precs=(("f32", 25), ("f32", 28), ("f32x2", 25), ("f64", 25))):
    """Line-operator microbench: 4096 independent wall-normal lines of 512 nodes
    (walls at both ends), band-limited trig sums plus degree-4 polynomials,
    d/dy and d^2/dy^2 per call through line_op (one fused kernel).
    Algorithmic bytes: 4 B in + 2 x 4 B out per node (FP32 fields; 8 B for
    FP64 I/O).  One call moves 25 MB, which fits in L2, so the timed calls
    rotate through 8 input/output sets (200 MB)."""
    import torch
    from paper_2606_06247_gb300 import binding as b
    from paper_2606_06247_gb300 import inputs
    L, n, sets = 4096, 512, 8
    base = inputs.band_limited_lines(L, n, seed=12345)
    peaks, src = load_peaks()
    variants = {}
    for prec, n_cont in precs:
        dt = torch.float32 if prec == "f32" else torch.float64
        dy = 1.0 / (n - 1)
        ctx = b.Context(L, n, L * dy, 1.0, batch=1, n_cont=n_cont, family="G4", h_over_dx=1.3, prec=prec)
        fs = [torch.tensor(base, dtype=dt, device="cuda").reshape(1, L, n) for _ in range(sets)]
        outs = [[torch.empty_like(fs[0]) for _ in range(2)] for _ in range(sets)]

        def call_ms(calls):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for k in range(calls):
                ctx.line_op(fs[k % sets], ["DY", "LAP"], outs[k % sets])
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / calls

        sweep = {}
        if prec == "f32":  # CTA width of the line kernel: a short sweep, then the timed calls at the fastest
            for w in (32, 64, 128):
                ctx.set_cta_threads(32, w)
                call_ms(sets)
                sweep[w] = call_ms(2 * sets)
            ctx.set_cta_threads(32, min(sweep, key=sweep.get))
        call_ms(max(3, warmup, sets))
        calls = max(steps, sets)
        ms = call_ms(calls)
        es = 4 if prec == "f32" else 8
        gbs = L * n * 3 * es / (ms * 1e-3) / 1e9
        variants[f"{prec} n_cont={n_cont} (n_e={n + n_cont})"] = {
            "ms_per_call": ms, "alg_GBps": gbs, "frac_of_hbm": gbs / peaks["hbm_gbs"], "launches_per_call": 1,
            "lines_per_s": L / (ms * 1e-3), "cta_threads": ctx.get_cta_threads()[1], "width_sweep_ms": sweep}
        del ctx, fs, outs
        torch.cuda.empty_cache()
    return variants, src


def run_lines(args):
    import __graft_entry__
    __graft_entry__.build()
    variants, src = measure_lines(args.steps, args.warmup)
    peaks, _ = load_peaks()
    head = variants["f32 n_cont=25 (n_e=537)"]
    print(json.dumps({"metric": "FC-extended line operator throughput (algorithmic HBM GB/s)", "value": head["alg_GBps"],
                      "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                      "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "4096 lines of 512 nodes, walls at both ends, FC(Gram) d=5 C=25, G4 "
                                             "h=1.3dy, line_op DY+LAP, FP32 fields, 8 rotating buffer sets",
                                 "peak_source": src},
                      "roofline": {"bound": "hbm", "achieved": head["alg_GBps"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                   "frac": head["frac_of_hbm"], "traffic": None},
                      "variants": variants}))


def run_dipole(args):
    """Sec. 6.5 vortex dipole rebound, Re = 100: 161^2 particles on [-1, 1]^2,
    walls all round (FC in x and y), G4 h = 1.3 dx, RK3 dt = 1.25e-3.  Reports
    the batched throughput (B independent dipoles, one graph per step) and one
    dipole run to t = 10 with E(t) = 1/2 int |u|^2 and Z(t) = 1/2 int omega^2
    (trapezoidal rule; omega from the library's spectral d/dx, d/dy)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06247_gb300 import binding as b
    from paper_2606_06247_gb300 import inputs
    n, dt, nu = 161, 1.25e-3, 0.01
    prm = dict(nu=nu, rho=1.0, dt=dt, scheme="rk3")
    u0, v0 = inputs.dipole_initial(n)
    h = 2.0 / (n - 1)
    wq = torch.ones(n, dtype=torch.float64, device="cuda")
    wq[0] = wq[-1] = 0.5
    W2 = (wq[:, None] * wq[None, :]) * (0.5 * h * h)
    B = args.batch
    out = {}
    for prec in (args.prec, "f64"):
        ctx = b.Context(n, n, 2.0, 2.0, x_walls=True, batch=B, family="G4", h_over_dx=1.3, prec=prec)
        ctx.autotune(steps=2, **prm)
        st = [torch.tensor(np.broadcast_to(a, (B, n, n)).copy(), dtype=torch.float64, device="cuda") for a in (u0, v0)]
        st += [torch.zeros_like(st[0]) for _ in range(3)]
        ctx.isph_step(*st, max(3, args.warmup), use_graph=True, **prm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.isph_step(*st, args.steps, use_graph=True, **prm)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[prec] = {"ms_per_step": ms, "particle_updates_per_s": B * n * n / (ms * 1e-3), "tiling": list(ctx.get_tiling())}
        del ctx, st
    # one dipole to t = 10 with the energy and enstrophy history
    ctx = b.Context(n, n, 2.0, 2.0, x_walls=True, batch=1, family="G4", h_over_dx=1.3, prec=args.prec)
    u = torch.tensor(u0[None], dtype=torch.float64, device="cuda")
    v = torch.tensor(v0[None], dtype=torch.float64, device="cuda")
    p, fu, fv = torch.zeros_like(u), torch.zeros_like(u), torch.zeros_like(u)
    vx, uy = torch.empty_like(u), torch.empty_like(u)
    hist = []
    marks = [0.0, 0.25, 0.5, 1.0, 2.0, 3.0, 5.0, 7.5, 10.0]
    t, k = 0.0, 0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for tm in marks:
        nst = int(round((tm - t) / dt))
        if nst > 0:
            ctx.isph_step(u, v, p, fu, fv, nst, use_graph=True, **prm)
            t += nst * dt
        ctx.spectral_op(v, ["DX"], [vx])
        ctx.spectral_op(u, ["DY"], [uy])
        E = float((W2 * (u[0] ** 2 + v[0] ** 2)).sum())
        Z = float((W2 * (vx[0] - uy[0]) ** 2).sum())
        hist.append({"t": round(t, 6), "E": E, "Z": Z})
    e1.record()
    torch.cuda.synchronize()
    run_s = e0.elapsed_time(e1) / 1e3
    head = out[args.prec]
    print(json.dumps({
        "metric": METRIC, "value": head["particle_updates_per_s"], "unit": "particle-updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "dtype": args.prec, "data": "synthetic",
        "config": {"workload": f"vortex dipole rebound Re=100, 161x161 on [-1,1]^2 walls all round, G4 h=1.3dx, "
                               f"RK3 dt=1.25e-3, batch of {B} dipoles", "batch": B},
        "variants": out,
        "history": {"precision": args.prec, "run_seconds": run_s, "steps": int(round(10.0 / dt)), "E_Z": hist}}))


def run_channel3d(args):
    """3D channel (the 3D requests of the serving mix): n^3 particles, x and z periodic
    (lx = lz = n dy), walls at y = 0, 1, G4 h = 1.3 dx, Re = 100 (u_max = 1:
    nu = 0.01, body force 0.08 in x), RK3 dt = 1e-3, a batch of B channels at
    rest.  Reports the throughput per precision and, after 100 steps, each
    precision's L2 error of u against the analytic start-up series (the flow
    stays one-dimensional).  (At nu = 0.1 the explicit step is past its
    viscous stability limit on a 128^3 lattice.)"""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06247_gb300 import binding as b
    n = int(os.environ.get("FCSPH_BENCH_N3", "128"))
    B = max(1, min(args.batch, 4))
    dy = 1.0 / (n - 1)
    prm = dict(nu=0.01, rho=1.0, dt=1e-3, force=(0.08, 0.0, 0.0), scheme="rk3")
    ua = torch.tensor(_startup_series(np.linspace(0, 1, n), 0.1, 0.08, 0.01), dtype=torch.float64, device="cuda")
    out = {}
    for prec in ("f32x2", "f64"):
        ctx = b.Context(n, n, n * dy, 1.0, batch=B, family="G4", h_over_dx=1.3, prec=prec, nz=n, lz=n * dy)
        z = torch.zeros((B, n, n, n), dtype=torch.float64, device="cuda")
        u, v, w, p, fu, fv, fw = [z.clone() for _ in range(7)]
        st = dict(w=w, fw=fw)
        ctx.isph_step(u, v, p, fu, fv, max(3, args.warmup), **st, **prm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.isph_step(u, v, p, fu, fv, args.steps, **st, **prm)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        for q in (u, v, w, p, fu, fv, fw):
            q.zero_()
        ctx.isph_step(u, v, p, fu, fv, 100, **st, **prm)
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(u[0] - ua) / torch.linalg.vector_norm(ua.expand_as(u[0])))
        out[prec] = {"ms_per_step": ms, "particle_updates_per_s": B * n ** 3 / (ms * 1e-3),
                     "l2_u_vs_analytic_after_100_steps": err, "max_abs_w": float(w.abs().max())}
        del ctx, z, u, v, w, p, fu, fv, fw
        torch.cuda.empty_cache()
    head = out["f32x2"]
    print(json.dumps({
        "metric": METRIC, "value": head["particle_updates_per_s"], "unit": "particle-updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "dtype": "f32x2", "data": "synthetic",
        "config": {"workload": f"3D channel {n}^3 (x, z periodic, walls in y), FC(Gram) d=5 C=25 in y, G4 h=1.3dx, "
                               f"Re=100, RK3 dt=1e-3, batch of {B}", "batch": B, "n": n},
        "variants": out,
        "equal_l2": abs(out["f32x2"]["l2_u_vs_analytic_after_100_steps"] - out["f64"]["l2_u_vs_analytic_after_100_steps"])
                    <= 1e-6 * out["f64"]["l2_u_vs_analytic_after_100_steps"]}))


def run_profile_case(args):
    """Two eager RK3 steps of the workload with every kernel launched on its own
    (no graph), for kernel-level captures, in the launch shape --tiling /
    --cta-threads give (else the context's default); prints the launch count.  With
    --workload planes: three spectral_op calls (DX, DY, LAP) on `batch` planes
    of 1024^2 (n_cont --plane-cont, FP32, default CTA widths)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06247_gb300 import binding as b
    B = args.batch
    if args.workload == "planes":
        import numpy as np
        from paper_2606_06247_gb300 import inputs
        n = 1024
        base = inputs.band_limited_planes(4, n, n, seed=12346, n_modes=64, max_mode=64)
        f = torch.tensor(np.tile(base, ((B + 3) // 4, 1, 1))[:B], dtype=torch.float32, device="cuda")
        outs = [torch.empty_like(f) for _ in range(3)]
        ctx = b.Context(n, n, n / (n - 1), 1.0, batch=B, n_cont=args.plane_cont, family="G4", h_over_dx=1.3,
                        prec="f32")
        for _ in range(3):
            ctx.spectral_op(f, ["DX", "DY", "LAP"], outs)
        ctx.sync()
        print(json.dumps({"profile_case": "planes", "batch": B, "cta_threads": ctx.get_cta_threads(),
                          "launches": ctx.launch_count}))
        return
    ctx = b.Context(N, N, 1.0, 1.0, x_walls=True, batch=B, n_match=N_MATCH, n_cont=N_CONT, family=FAMILY,
                    h_over_dx=HDX, prec=args.prec, refine=args.refine if args.prec == "f32" else 0)
    if args.tiling:  # the launch shape of the bench line being profiled
        ctx.set_tiling(*[int(x) for x in args.tiling.split(",")])
    if args.cta_threads:
        ctx.set_cta_threads(*[int(x) for x in args.cta_threads.split(",")])
    z = torch.zeros((B, N, N), dtype=torch.float64, device="cuda")
    u, v, p, fu, fv = [z.clone() for _ in range(5)]
    if args.persistent:  # two steps, each one launch of the persistent kernel
        ctx.set_step_persistent(True)
        ctx.isph_step(u, v, p, fu, fv, 2, nu=NU, rho=1.0, dt=DT, u_top=LID, scheme="rk3", use_graph=True)
        ctx.sync()
        print(json.dumps({"profile_case": "persistent", "prec": args.prec, "batch": B, "launches": ctx.launch_count}))
        return
    ctx.isph_step(u, v, p, fu, fv, 2, nu=NU, rho=1.0, dt=DT, u_top=LID, scheme="rk3", use_graph=False)
    ctx.sync()
    print(json.dumps({"profile_case": True, "prec": args.prec, "batch": B, "launches": ctx.launch_count}))


if __name__ == "__main__":
    a = parse()
    if a.profile_case:
        run_profile_case(a)
    elif a.workload in ("uneven", "serve") and a.impl == "ours":
        run_serving(a)
    elif a.workload == "planes" and a.impl == "ours":
        run_planes(a)
    elif a.workload == "lines" and a.impl == "ours":
        run_lines(a)
    elif a.workload == "dipole" and a.impl == "ours":
        run_dipole(a)
    elif a.workload == "channel3d" and a.impl == "ours":
        run_channel3d(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
