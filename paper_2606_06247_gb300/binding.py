"""Thin ctypes binding of libfcsph (include/fcsph.h), same names as the C ABI.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Device arrays are torch CUDA tensors (their data_ptr() is passed);
the stream is torch's current CUDA stream unless given.  Importing this module
loads libfcsph.so and raises if it has not been built -- there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfcsph.so")

F64, F32, F32X2 = 0, 1, 2
PREC = {"f64": F64, "f32": F32, "f32x2": F32X2}
FC_GRAM, FC_PAPER = 0, 1
DIRICHLET, NEUMANN = 0, 1
FAMILY = {"G2": 1, "G4": 2, "G6": 3, "G8": 4, "G10": 5}
OP_W, OP_DX, OP_DY, OP_LAP, OP_DZ = 1, 2, 4, 8, 16
OPS = {"W": OP_W, "DX": OP_DX, "DY": OP_DY, "LAP": OP_LAP, "DZ": OP_DZ}
SCHEME = {"fop": 0, "rk3": 1}
PROF_KINDS = ["col_fwd", "row_mom", "row_div", "row_grad", "row_op", "col_mom", "col_div", "col_corr", "col_out",
              "row_ppe", "col_ppe", "other"]
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENONFINITE", 6: "EUNSUPPORTED"}


class FcsphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fcsph {STATUS.get(status, status)}: {msg}")
        self.status = status


class fcsph_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("x_walls", ctypes.c_int), ("batch", ctypes.c_int), ("nz", ctypes.c_int), ("lz", ctypes.c_double)]


class fcsph_fc(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("n_match", ctypes.c_int), ("n_cont", ctypes.c_int), ("poly_deg", ctypes.c_int)]


class fcsph_kernel(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("h_over_dx", ctypes.c_double)]


class fcsph_precision(ctypes.Structure):
    _fields_ = [("fft_prec", ctypes.c_int), ("ppe_refine_iters", ctypes.c_int)]


class fcsph_state(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("u", "v", "p", "fu", "fv", "w", "fw")]


class fcsph_step_params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("rho", ctypes.c_double), ("dt", ctypes.c_double),
                ("force_x", ctypes.c_double), ("force_y", ctypes.c_double),
                ("u_bottom", ctypes.c_double), ("u_top", ctypes.c_double),
                ("scheme", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("nu_inst", ctypes.c_void_p), ("fx_inst", ctypes.c_void_p), ("force_z", ctypes.c_double),
                ("active", ctypes.c_void_p), ("dt_inst", ctypes.c_void_p)]


class fcsph_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("re", ctypes.c_double), ("steps", ctypes.c_int)]


class fcsph_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("done_steps", ctypes.c_int), ("last_step_ms", ctypes.c_double),
                ("total_step_ms", ctypes.c_double)]


REQ_KIND = {"cavity": 0, "channel": 1, "channel3d": 2}
REQ_STATE = {0: "queued", 1: "running", 2: "done", 3: "cancelled"}


def torch_uint8():
    import torch
    return torch.uint8


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it first (python -m paper_2606_06247_gb300.build)")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, U, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint, ctypes.c_size_t
    sig = {
        "fcsph_create": [ctypes.POINTER(fcsph_grid), ctypes.POINTER(fcsph_fc), ctypes.POINTER(fcsph_kernel),
                         ctypes.POINTER(fcsph_precision), P, P, P, ctypes.POINTER(P)],
        "fcsph_destroy": [P],
        "fcsph_get_fc_table": [P, I, P, S],
        "fcsph_fc_table": [ctypes.POINTER(fcsph_fc), I, P, S],
        "fc_extend": [P, P, P, I],
        "spectral_op": [P, P, U, I, P],
        "spectral_div": [P, P, P, P],
        "spectral_project": [P, P, P, P, P],
        "line_op": [P, P, U, I, P],
        "ppe_solve": [P, P, P, ctypes.POINTER(D)],
        "isph_step": [P, ctypes.POINTER(fcsph_state), I, ctypes.POINTER(fcsph_step_params)],
        "fcsph_sync": [P],
        "fcsph_dft": [I, I, I, I, P, P, P],
        "fcsph_dft_noalloc": [I, I, I, I, P, P, P],
        "fcsph_launch_count": [P],
        "fcsph_last_error": [P, ctypes.c_char_p, S],
        "fcsph_set_profiling": [P, I],
        "fcsph_get_profile": [P, P, P, I],
        "fcsph_set_tiling": [P, I, I],
        "fcsph_get_tiling": [P, ctypes.POINTER(I), ctypes.POINTER(I)],
        "fcsph_set_cta_threads": [P, I, I],
        "fcsph_get_cta_threads": [P, ctypes.POINTER(I), ctypes.POINTER(I)],
        "fcsph_set_step_groups": [P, I],
        "fcsph_set_step_persistent": [P, I],
        "fcsph_set_tma": [P, I],
        "fcsph_set_tracing": [P, I],
        "fcsph_get_step_persistent": [P, ctypes.POINTER(I)],
        "fcsph_get_step_groups": [P, ctypes.POINTER(I)],
        "fcsph_autotune": [P, ctypes.POINTER(fcsph_step_params), I, ctypes.POINTER(D)],
        "fcsph_batch_create": [I, I, D, I, ctypes.POINTER(P)],
        "fcsph_batch_destroy": [P],
        "fcsph_batch_add": [P, ctypes.POINTER(fcsph_request), ctypes.POINTER(ctypes.c_longlong)],
        "fcsph_batch_remove": [P, ctypes.c_longlong],
        "fcsph_batch_run": [P, I, ctypes.POINTER(I)],
        "fcsph_batch_poll": [P, ctypes.c_longlong, ctypes.POINTER(fcsph_request_info)],
        "fcsph_batch_result": [P, ctypes.c_longlong, P, P, P, P, S],
        "fcsph_batch_info": [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)],
        "fcsph_batch_last_error": [P, ctypes.c_char_p, S],
        "fcsph_batch_set_persistent": [P, I, D],
        "fcsph_batch_inject_stall": [P],
        "fcsph_batch_set_size_priorities": [P, I],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_longlong if name == "fcsph_launch_count" else ctypes.c_int
    return L


lib = _load()


def last_error(ctx=None):
    buf = ctypes.create_string_buffer(512)
    lib.fcsph_last_error(ctx, buf, 512)
    return buf.value.decode()


def _check(st, ctx=None):
    if st != 0:
        raise FcsphError(st, last_error(ctx))


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def fc_table(variant="gram", n_match=5, n_cont=25, bc=DIRICHLET, poly_deg=0):
    """Host-built FC table [n_cont][2*n_match] (fcsph_fc_table)."""
    fc = fcsph_fc(FC_GRAM if variant == "gram" else FC_PAPER, n_match, n_cont, poly_deg)
    out = np.zeros((n_cont, 2 * n_match))
    _check(lib.fcsph_fc_table(ctypes.byref(fc), bc, out.ctypes.data_as(ctypes.c_void_p), out.size))
    return out


def fcsph_dft(x, direction=-1, stream=None, double_float=False):
    """Batched DFT over the last axis of a complex CUDA tensor (engine test entry).
    double_float: complex128 in and out, arithmetic in FP32 pairs (FCSPH_F32X2)."""
    import torch
    assert x.is_cuda and x.is_complex() and x.is_contiguous()
    prec = F64 if x.dtype == torch.complex128 else F32
    if double_float:
        assert prec == F64
        prec = F32X2
    n = x.shape[-1]
    out = torch.empty_like(x)
    _check(lib.fcsph_dft(n, x.numel() // n if n else 0, direction, prec, _ptr(x), _ptr(out), _stream(stream)))
    return out


def fcsph_dft_noalloc(x, out, direction=-1, stream=None):
    """fcsph_dft into a caller-provided `out`, with no allocation on the library
    side (scratch in a fixed per-device array; see include/fcsph.h)."""
    import torch
    assert x.is_cuda and x.is_complex() and x.is_contiguous() and out.shape == x.shape and out.dtype == x.dtype
    prec = F64 if x.dtype == torch.complex128 else F32
    n = x.shape[-1]
    _check(lib.fcsph_dft_noalloc(n, x.numel() // n if n else 0, direction, prec, _ptr(x), _ptr(out),
                                 _stream(stream)))
    return out


def load_tune_cache(path):
    """{key: launch shape} from the autotune cache file (empty if absent or unreadable)."""
    import json
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_tune_cache(path, key, state):
    """Adds or replaces one entry of the autotune cache file (written whole, through a temporary file)."""
    import json
    import os
    d = load_tune_cache(path)
    d[key] = state
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Context:
    """fcsph_create/destroy plus the per-call entry points."""

    def __init__(self, nx, ny, lx, ly, x_walls=False, batch=1, n_match=5, n_cont=25, variant="gram", poly_deg=0,
                 family="G4", h_over_dx=1.3, prec="f64", refine=0, table_dir=None, table_neu=None, stream=None,
                 nz=1, lz=0.0):
        """nz > 1: a 3D channel (x and z periodic, walls in y), fields [batch][nx][nz][ny]."""
        self.grid = fcsph_grid(nx, ny, lx, ly, 1 if x_walls else 0, batch, nz, lz)
        self.fc = fcsph_fc(FC_GRAM if variant == "gram" else FC_PAPER, n_match, n_cont, poly_deg)
        self.kernel = fcsph_kernel(FAMILY[family], h_over_dx)
        self.prec = fcsph_precision(PREC[prec], refine)
        self.prec_name = prec
        self._tabs = []
        tp = []
        for t in (table_dir, table_neu):
            if t is None:
                tp.append(None)
            else:
                a = np.ascontiguousarray(t, dtype=np.float64)
                assert a.shape == (n_cont, 2 * n_match)
                self._tabs.append(a)
                tp.append(a.ctypes.data_as(ctypes.c_void_p))
        self.stream = _stream(stream)
        h = ctypes.c_void_p()
        _check(lib.fcsph_create(ctypes.byref(self.grid), ctypes.byref(self.fc), ctypes.byref(self.kernel),
                                ctypes.byref(self.prec), tp[0], tp[1], self.stream, ctypes.byref(h)))
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib.fcsph_destroy(h)
            self.h = None

    def close(self):
        self.__del__()

    def _ck(self, st):
        _check(st, self.h)

    def get_fc_table(self, bc=DIRICHLET):
        out = np.zeros((self.fc.n_cont, 2 * self.fc.n_match))
        self._ck(lib.fcsph_get_fc_table(self.h, bc, out.ctypes.data_as(ctypes.c_void_p), out.size))
        return out

    def fc_extend(self, f, f_ext, bc=DIRICHLET):
        self._ck(lib.fc_extend(self.h, _ptr(f), _ptr(f_ext), bc))

    def spectral_op(self, f, ops, outs, bc=DIRICHLET):
        """outs[k] for ops[k]; the C call takes them in its bit order W, DX, DY, LAP, DZ."""
        assert len(ops) == len(outs) and len(set(ops)) == len(ops)
        mask = 0
        for o in ops:
            mask |= OPS[o]
        order = [o for o in ("W", "DX", "DY", "LAP", "DZ") if mask & OPS[o]]
        assert len(order) == len(ops)
        by_name = dict(zip(ops, outs))
        arr = (ctypes.c_void_p * len(order))(*[by_name[o].data_ptr() for o in order])
        self._ck(lib.spectral_op(self.h, _ptr(f), mask, bc, arr))

    def line_op(self, f, ops, outs, bc=DIRICHLET):
        """Wall-normal operators of every column as an independent line (line_op)."""
        mask = 0
        for o in ops:
            mask |= OPS[o]
        order = [o for o in ("W", "DX", "DY", "LAP", "DZ") if mask & OPS[o]]
        assert len(order) == len(ops) and len(outs) == len(ops)
        by_name = dict(zip(ops, outs))
        arr = (ctypes.c_void_p * len(order))(*[by_name[o].data_ptr() for o in order])
        self._ck(lib.line_op(self.h, _ptr(f), mask, bc, arr))

    def spectral_div(self, fx, fy, out):
        self._ck(lib.spectral_div(self.h, _ptr(fx), _ptr(fy), _ptr(out)))

    def spectral_project(self, fx, fy, out_x, out_y):
        """Projection on the FC-extended grid (see include/fcsph.h)."""
        for t in (fx, fy, out_x, out_y):
            assert t.is_cuda and t.is_contiguous()
        assert out_x.data_ptr() not in (fx.data_ptr(), fy.data_ptr()) and out_y.data_ptr() not in (fx.data_ptr(), fy.data_ptr())
        self._ck(lib.spectral_project(self.h, _ptr(fx), _ptr(fy), _ptr(out_x), _ptr(out_y)))

    def ppe_solve(self, rhs, phi, want_resid=False):
        r = ctypes.c_double(0.0)
        self._ck(lib.ppe_solve(self.h, _ptr(rhs), _ptr(phi), ctypes.byref(r) if want_resid else None))
        return r.value if want_resid else None

    @staticmethod
    def _params(nu, rho, dt, force, u_bottom, u_top, scheme, use_graph, nu_inst, fx_inst, active=None, dt_inst=None):
        fz = force[2] if len(force) > 2 else 0.0
        if active is not None:
            assert active.is_cuda and active.dtype == torch_uint8() and active.is_contiguous()
        return fcsph_step_params(nu, rho, dt, force[0], force[1], u_bottom, u_top, SCHEME[scheme], 1 if use_graph else 0,
                                 nu_inst.data_ptr() if nu_inst is not None else None,
                                 fx_inst.data_ptr() if fx_inst is not None else None, fz,
                                 active.data_ptr() if active is not None else None,
                                 dt_inst.data_ptr() if dt_inst is not None else None)

    def isph_step(self, u, v, p, fu, fv, nsteps, nu, rho=1.0, dt=1e-3, force=(0.0, 0.0), u_bottom=0.0, u_top=0.0,
                  scheme="fop", use_graph=True, nu_inst=None, fx_inst=None, w=None, fw=None, active=None,
                  dt_inst=None):
        """nu_inst / fx_inst / dt_inst: optional CUDA float64 tensors [batch] of
        per-instance viscosity, x body force and time step (override nu /
        force[0] / dt).  3D grids: w, fw (z velocity and its F^{k-1}) and force =
        (fx, fy, fz).  active: optional CUDA uint8 tensor [batch]; only instances
        with a nonzero flag advance."""
        st = fcsph_state(u.data_ptr(), v.data_ptr(), p.data_ptr(), fu.data_ptr(), fv.data_ptr(),
                         w.data_ptr() if w is not None else None, fw.data_ptr() if fw is not None else None)
        prm = self._params(nu, rho, dt, force, u_bottom, u_top, scheme, use_graph, nu_inst, fx_inst, active, dt_inst)
        self._ck(lib.isph_step(self.h, ctypes.byref(st), nsteps, ctypes.byref(prm)))

    def set_tiling(self, row_lines, col_pairs):
        self._ck(lib.fcsph_set_tiling(self.h, row_lines, col_pairs))

    def get_tiling(self):
        r, c = ctypes.c_int(), ctypes.c_int()
        self._ck(lib.fcsph_get_tiling(self.h, ctypes.byref(r), ctypes.byref(c)))
        return r.value, c.value

    def set_cta_threads(self, row_threads, col_threads):
        """fcsph_set_cta_threads: threads per CTA of the row and column passes (32, 64, 128; FP32 only > 32)."""
        self._ck(lib.fcsph_set_cta_threads(self.h, row_threads, col_threads))

    def get_cta_threads(self):
        r, c = ctypes.c_int(), ctypes.c_int()
        self._ck(lib.fcsph_get_cta_threads(self.h, ctypes.byref(r), ctypes.byref(c)))
        return r.value, c.value

    def set_step_groups(self, groups):
        """fcsph_set_step_groups: instance groups run as parallel branches of the step graph (1..16)."""
        self._ck(lib.fcsph_set_step_groups(self.h, groups))

    def get_step_groups(self):
        g = ctypes.c_int()
        self._ck(lib.fcsph_get_step_groups(self.h, ctypes.byref(g)))
        return g.value

    def set_step_persistent(self, on=True):
        """fcsph_set_step_persistent: each graph step as one persistent launch (2D FP64 / FP32x2)."""
        self._ck(lib.fcsph_set_step_persistent(self.h, 1 if on else 0))

    def set_tracing(self, on=True):
        """fcsph_set_tracing: NVTX ranges around every call and pass."""
        self._ck(lib.fcsph_set_tracing(self.h, 1 if on else 0))

    def set_tma(self, on=True):
        """fcsph_set_tma: bulk-copy (TMA) staging of the FP32 register column passes."""
        self._ck(lib.fcsph_set_tma(self.h, 1 if on else 0))

    def get_step_persistent(self):
        v = ctypes.c_int()
        self._ck(lib.fcsph_get_step_persistent(self.h, ctypes.byref(v)))
        return bool(v.value)

    def tune_key(self, scheme="rk3", device_name=""):
        """The autotune cache key of this context: grid, FC, kernel, precision, scheme and device."""
        g, f, k, p = self.grid, self.fc, self.kernel, self.prec
        return (f"{device_name}|{g.nx}x{g.ny}x{max(g.nz, 1)}|xw{g.x_walls}|b{g.batch}|fc{f.variant},{f.n_match},"
                f"{f.n_cont},{f.poly_deg}|k{k.family},{k.h_over_dx}|p{p.fft_prec},{p.ppe_refine_iters}|{scheme}")

    def tune_state(self):
        """The launch shape the autotuner sets (tiling, CTA widths, step groups, persistent step)."""
        return {"tiling": list(self.get_tiling()), "cta_threads": list(self.get_cta_threads()),
                "groups": self.get_step_groups(), "persistent": self.get_step_persistent()}

    def apply_tune_state(self, st):
        self.set_tiling(*st["tiling"])
        self.set_cta_threads(*st["cta_threads"])
        self.set_step_groups(st["groups"])
        self.set_step_persistent(st["persistent"])

    def autotune(self, steps=3, nu=1e-3, rho=1.0, dt=1e-3, force=(0.0, 0.0), u_bottom=0.0, u_top=0.0, scheme="rk3",
                 use_graph=True, nu_inst=None, fx_inst=None, cache=None, device_name=""):
        """fcsph_autotune: keeps the fastest tiling, then CTA widths, then step groups, then (2D FP64 / FP32x2)
        the persistent step; returns (row_lines, col_pairs, ms per step).  cache: path of a JSON file of launch
        shapes by tune_key; a hit applies the stored shape without timing (ms None), a miss tunes and stores."""
        key = self.tune_key(scheme, device_name)
        if cache is not None:
            hit = load_tune_cache(cache).get(key)
            if hit is not None:
                self.apply_tune_state(hit)
                r, c = self.get_tiling()
                return r, c, None
        prm = self._params(nu, rho, dt, force, u_bottom, u_top, scheme, use_graph, nu_inst, fx_inst)
        ms = ctypes.c_double()
        self._ck(lib.fcsph_autotune(self.h, ctypes.byref(prm), steps, ctypes.byref(ms)))
        if cache is not None:
            store_tune_cache(cache, key, self.tune_state())
        r, c = self.get_tiling()
        return r, c, ms.value

    def sync(self):
        self._ck(lib.fcsph_sync(self.h))

    @property
    def launch_count(self):
        return lib.fcsph_launch_count(self.h)

    def set_profiling(self, on=True):
        self._ck(lib.fcsph_set_profiling(self.h, 1 if on else 0))

    def get_profile(self):
        """{kind: (total_ms, launches)} since the last call (eager launches only)."""
        ms = np.zeros(len(PROF_KINDS))
        cnt = np.zeros(len(PROF_KINDS), dtype=np.int64)
        self._ck(lib.fcsph_get_profile(self.h, ms.ctypes.data_as(ctypes.c_void_p),
                                       cnt.ctypes.data_as(ctypes.c_void_p), len(PROF_KINDS)))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROF_KINDS) if cnt[i] > 0}


class Batch:
    """fcsph_batch_*: continuous batching of independent solves in the
    library (argument marshalling only; the scheduler is native)."""

    def __init__(self, prec="f32x2", slots=8, mem_budget=0.0, n_cont=25):
        """n_cont: continuation length of every class, or "smooth" (per-size choice)."""
        h = ctypes.c_void_p()
        nc = 0 if n_cont == "smooth" else int(n_cont)
        st = lib.fcsph_batch_create(PREC[prec], slots, float(mem_budget), nc, ctypes.byref(h))
        if st != 0:
            raise FcsphError(st, self._err(None))
        self.h = h
        self.prec = prec

    @staticmethod
    def _err(h):
        buf = ctypes.create_string_buffer(512)
        lib.fcsph_batch_last_error(h, buf, 512)
        return buf.value.decode()

    def _ck(self, st):
        if st != 0:
            raise FcsphError(st, self._err(self.h))

    def add(self, kind, n, re, steps):
        req = fcsph_request(REQ_KIND[kind], n, re, steps)
        rid = ctypes.c_longlong()
        self._ck(lib.fcsph_batch_add(self.h, ctypes.byref(req), ctypes.byref(rid)))
        return rid.value

    def remove(self, rid):
        self._ck(lib.fcsph_batch_remove(self.h, rid))

    def run(self, block=False):
        """One scheduling tick; returns the number of classes in flight."""
        k = ctypes.c_int()
        self._ck(lib.fcsph_batch_run(self.h, 1 if block else 0, ctypes.byref(k)))
        return k.value

    def set_persistent(self, on=True, wait_limit_s=1.0):
        """fcsph_batch_set_persistent: every tick steps all classes in one persistent launch."""
        self._ck(lib.fcsph_batch_set_persistent(self.h, 1 if on else 0, float(wait_limit_s)))

    def set_size_priorities(self, on=True):
        """fcsph_batch_set_size_priorities: larger classes on higher-priority streams."""
        self._ck(lib.fcsph_batch_set_size_priorities(self.h, 1 if on else 0))

    def inject_stall(self):
        """fcsph_batch_inject_stall: the next persistent launch has one wait that runs out (tests)."""
        self._ck(lib.fcsph_batch_inject_stall(self.h))

    def poll(self, rid):
        info = fcsph_request_info()
        self._ck(lib.fcsph_batch_poll(self.h, rid, ctypes.byref(info)))
        return {"state": REQ_STATE[info.state], "done_steps": info.done_steps, "last_step_ms": info.last_step_ms,
                "total_step_ms": info.total_step_ms}

    def result(self, rid, kind, n):
        shape = (n, n, n) if kind == "channel3d" else (n, n)
        out = {k: np.zeros(shape) for k in (("u", "v", "w", "p") if kind == "channel3d" else ("u", "v", "p"))}
        ptr = lambda k: out[k].ctypes.data_as(ctypes.c_void_p) if k in out else None
        self._ck(lib.fcsph_batch_result(self.h, rid, ptr("u"), ptr("v"), ptr("w"), ptr("p"), out["u"].size))
        return out

    def info(self):
        c, q, u = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._ck(lib.fcsph_batch_info(self.h, ctypes.byref(c), ctypes.byref(q), ctypes.byref(u)))
        return {"classes": c.value, "queued": q.value, "used_bytes": u.value}

    def close(self):
        if self.h:
            lib.fcsph_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
