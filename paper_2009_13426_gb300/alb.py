"""Thin Python binding of the C ABI in include/alb.h (libalb.so).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. The functions keep the C names. Host arrays are numpy float64
(or int8) arrays; device arrays are torch CUDA tensors (torch is used for
device memory and streams only). There is no CPU fallback: if libalb.so is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libalb.so")

ALB_OK = 0
ALB_EINVAL = -1
ALB_ENOMEM = -2
ALB_EUNSUPPORTED = -3
ALB_ENEWTON = -4
ALB_EUNREALIZABLE = -5
ALB_ETIMEDOUT = -6
ALB_EBUSY = -7
ALB_ECUDA = -8
ALB_ENOTFOUND = -9

ALB_D2Q21 = 21
ALB_D2Q49 = 49
ALB_FP64_PLAIN = 0
ALB_FP32_FORM = 1
ALB_PERIODIC = 0
ALB_ZERO_GRADIENT = 1
ALB_HOST = 0
ALB_DEVICE = 1
ALB_START_AUTO = 0
ALB_START_MAXWELLIAN = 1
ALB_START_PREVIOUS = 2
ALB_RULE_HISTORY = 0
ALB_RULE_NEIGHBOURS = 1
Q = 21


class AlbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("alb error %d: %s" % (code, msg))
        self.code = code


class alb_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("stencil", ctypes.c_int),
        ("u_max", ctypes.c_int), ("nu", ctypes.c_double), ("gamma", ctypes.c_double),
        ("n0", ctypes.c_double), ("precision", ctypes.c_int), ("bc_x", ctypes.c_int),
        ("bc_y", ctypes.c_int), ("sensor", ctypes.c_int),
        ("sensor_eps", ctypes.c_double * 3), ("sensor_alpha", ctypes.c_double * 3),
        ("newton_tol", ctypes.c_double), ("newton_maxit", ctypes.c_int),
        ("newton_start", ctypes.c_int), ("shift_overlap", ctypes.c_double),
        ("shift_rule", ctypes.c_int), ("moments", ctypes.c_int), ("prandtl", ctypes.c_double),
        ("stream", ctypes.c_void_p),
    ]


class alb_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "steps", "node_updates", "newton_iterations", "newton_failures", "reconstructions",
        "reconstruction_failures", "newton_calls", "fp64_evaluations", "fp32_iterations",
        "fp64_updates")]


class alb_batch_tuning(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("tile_w", ctypes.c_int * 3),
                ("dynamic", ctypes.c_int), ("blocks_per_sm", ctypes.c_int)]


class alb_server_config(ctypes.Structure):
    _fields_ = [("hbm_fraction", ctypes.c_double), ("chunk_ms", ctypes.c_double),
                ("max_chunk", ctypes.c_int), ("max_flows", ctypes.c_int),
                ("batch_nodes", ctypes.c_longlong), ("tune", ctypes.c_int)]


FILL_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double))


class alb_request(ctypes.Structure):
    _fields_ = [("cfg", alb_config), ("nsteps", ctypes.c_int),
                ("rho", ctypes.c_void_p), ("rhoux", ctypes.c_void_p), ("rhouy", ctypes.c_void_p),
                ("rhoE", ctypes.c_void_p), ("fill", FILL_FN), ("user", ctypes.c_void_p),
                ("keep_result", ctypes.c_int)]


class alb_result(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_void_p), ("rhoux", ctypes.c_void_p), ("rhouy", ctypes.c_void_p),
                ("rhoE", ctypes.c_void_p), ("status", ctypes.c_int), ("steps", ctypes.c_uint64),
                ("stats", alb_stats), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class alb_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "submitted", "admitted", "completed", "failed", "queued", "running", "node_updates",
        "chunks", "steps", "resident_bytes", "budget_bytes")] + [
        ("busy_seconds", ctypes.c_double), ("elapsed_seconds", ctypes.c_double),
        ("ns_per_update", ctypes.c_double * 2)]


ALB_QUEUED, ALB_RUNNING, ALB_DONE, ALB_FAILED = 0, 1, 2, 3

_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "alb_config_default": (ctypes.c_int, [ctypes.POINTER(alb_config)]),
    "alb_create": (ctypes.c_int, [ctypes.POINTER(alb_config), ctypes.POINTER(ctypes.c_void_p)]),
    "alb_init": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [ctypes.c_int]),
    "alb_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "alb_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "alb_moments": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [ctypes.c_int]),
    "alb_shifts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "alb_stats_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(alb_stats)]),
    "alb_totals": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "alb_totals_noalloc": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_longlong,
                                                                  ctypes.c_void_p, ctypes.c_void_p]),
    "alb_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "alb_last_error": (ctypes.c_char_p, []),
    "alb_equilibrium": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_double,
                                                                ctypes.c_int, ctypes.c_int]
                        + [ctypes.c_void_p] * 5),
    "alb_exp_neg_refine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "alb_exp_neg": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "alb_select_shift": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "alb_velocities": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "alb_stencil_velocities": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "alb_equilibrium13": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_double,
                                                                  ctypes.c_int]
                          + [ctypes.c_void_p] * 5),
    "alb_next_shifts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int]),
    "alb_populations": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int]),
    "alb_primitives": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_int]),
    "alb_checkpoint_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "alb_checkpoint_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "alb_checkpoint_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "alb_batch_variants": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "alb_batch_create": (ctypes.c_int, [ctypes.POINTER(alb_config), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "alb_batch_flow": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "alb_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "alb_batch_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "alb_batch_tune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "alb_batch_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(alb_batch_tuning)]),
    "alb_batch_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(alb_batch_tuning)]),
    "alb_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "alb_server_config_default": (ctypes.c_int, [ctypes.POINTER(alb_server_config)]),
    "alb_server_create": (ctypes.c_int, [ctypes.POINTER(alb_server_config),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "alb_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(alb_request),
                                  ctypes.POINTER(ctypes.c_uint64)]),
    "alb_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(alb_result)]),
    "alb_server_drain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "alb_server_stats_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(alb_server_stats)]),
    "alb_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
}


def lib():
    """Load libalb.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libalb.so not built: run `python -c \"import __graft_entry__ as g; "
                               "g.build()\"` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    return sorted(_SIGS)


def alb_last_error() -> str:
    return lib().alb_last_error().decode()


def _check(rc):
    if rc != ALB_OK:
        raise AlbError(rc, alb_last_error())
    return rc


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError("expected numpy array or torch tensor, got %r" % type(a))


def _where(a):
    return ALB_DEVICE if (hasattr(a, "is_cuda") and a.is_cuda) else ALB_HOST


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def alb_config_default(**kw) -> alb_config:
    c = alb_config()
    _check(lib().alb_config_default(ctypes.byref(c)))
    for k, v in kw.items():
        if k in ("sensor_eps", "sensor_alpha"):
            arr = getattr(c, k)
            for j in range(3):
                arr[j] = v[j]
        elif k == "stream":
            c.stream = _stream(v)
        else:
            setattr(c, k, v)
    return c


def alb_create(cfg: alb_config):
    h = ctypes.c_void_p()
    _check(lib().alb_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def alb_init(h, rho, rhoux, rhouy, rhoE):
    where = _where(rho)
    arrs = [rho, rhoux, rhouy, rhoE]
    if where == ALB_HOST:
        arrs = [np.ascontiguousarray(a, np.float64) for a in arrs]
    return _check(lib().alb_init(h, *[_ptr(a) for a in arrs], where))


def alb_step(h, nsteps: int):
    return _check(lib().alb_step(h, int(nsteps)))


def alb_sync(h, timeout_ms: int = -1):
    return _check(lib().alb_sync(h, int(timeout_ms)))


def alb_moments(h, out):
    """out: 4 arrays (numpy float64 or torch float64 CUDA tensors) of nx*ny."""
    return _check(lib().alb_moments(h, *[_ptr(a) for a in out], _where(out[0])))


def alb_shifts(h, ux, uy):
    return _check(lib().alb_shifts(h, _ptr(ux), _ptr(uy), _where(ux)))


def alb_next_shifts(h, ux, uy):
    return _check(lib().alb_next_shifts(h, _ptr(ux), _ptr(uy), _where(ux)))


def alb_populations(h, f, g):
    """f, g: 21 * nx * ny float64 each (plane i at [i * n, (i + 1) * n))."""
    return _check(lib().alb_populations(h, _ptr(f), _ptr(g), _where(f)))


def alb_primitives(h, out):
    """out: 4 arrays (rho, ux, uy, T) of nx * ny float64."""
    return _check(lib().alb_primitives(h, *[_ptr(a) for a in out], _where(out[0])))


def alb_checkpoint_save(h) -> np.ndarray:
    n = ctypes.c_size_t()
    _check(lib().alb_checkpoint_size(h, ctypes.byref(n)))
    buf = np.empty(n.value, np.uint8)
    _check(lib().alb_checkpoint_save(h, buf.ctypes.data))
    return buf


def alb_checkpoint_load(h, buf: np.ndarray):
    buf = np.ascontiguousarray(buf, np.uint8)
    return _check(lib().alb_checkpoint_load(h, buf.ctypes.data))


def alb_stats_get(h) -> dict:
    s = alb_stats()
    _check(lib().alb_stats_get(h, ctypes.byref(s)))
    return {k: int(getattr(s, k)) for k, _ in alb_stats._fields_}


def alb_destroy(h):
    return _check(lib().alb_destroy(h))


def alb_totals(h):
    """Sums of rho, rho*ux, rho*uy, rho*E over the grid (numpy array of 4)."""
    out = np.zeros(4)
    _check(lib().alb_totals(h, out.ctypes.data))
    return out


def alb_totals_noalloc(rho, rhoux, rhouy, rhoE, n, out, stream=None):
    """Totals of four device fields into the device array `out` (4 doubles)
    without allocating: for callers that cannot allocate device memory."""
    return _check(lib().alb_totals_noalloc(_ptr(rho), _ptr(rhoux), _ptr(rhouy), _ptr(rhoE),
                                           int(n), _ptr(out), _stream(stream)))


def alb_equilibrium(rho, ubx, uby, T, n, tol, maxit, feq, lam=None, iters=None, status=None,
                    stream=None, precision=ALB_FP64_PLAIN):
    """All arrays are torch CUDA tensors (float64; iters/status int32)."""
    return _check(lib().alb_equilibrium(_ptr(rho), _ptr(ubx), _ptr(uby), _ptr(T), int(n),
                                        float(tol), int(maxit), int(precision), _ptr(feq),
                                        _ptr(lam), _ptr(iters), _ptr(status), _stream(stream)))


def alb_exp_neg_refine(s, n, out, stream=None):
    """out = exp(-s) by the FP32 form's cheaper FP64 exponential (CUDA tensors)."""
    return _check(lib().alb_exp_neg_refine(_ptr(s), int(n), _ptr(out), _stream(stream)))


def alb_exp_neg(s, n, out, stream=None):
    """out = exp(-s) by the library's table-driven FP64 exponential (CUDA tensors)."""
    return _check(lib().alb_exp_neg(_ptr(s), int(n), _ptr(out), _stream(stream)))


def alb_select_shift(rho, rhou, n, n0, u_max, out, stream=None):
    return _check(lib().alb_select_shift(_ptr(rho), _ptr(rhou), int(n), float(n0), int(u_max),
                                         _ptr(out), _stream(stream)))


def alb_velocities():
    x = np.zeros(Q, np.int32)
    y = np.zeros(Q, np.int32)
    _check(lib().alb_velocities(x.ctypes.data, y.ctypes.data))
    return x, y


def alb_stencil_velocities(stencil):
    q = 49 if stencil == ALB_D2Q49 else Q
    x = np.zeros(q, np.int32)
    y = np.zeros(q, np.int32)
    _check(lib().alb_stencil_velocities(int(stencil), x.ctypes.data, y.ctypes.data))
    return x, y


def alb_equilibrium13(rho, ubx, uby, T, n, tol, maxit, feq, lam, iters, status, stream=None):
    """D2Q49 13-moment equilibria; torch CUDA tensors (float64; iters/status int32)."""
    return _check(lib().alb_equilibrium13(_ptr(rho), _ptr(ubx), _ptr(uby), _ptr(T), int(n),
                                          float(tol), int(maxit), _ptr(feq), _ptr(lam),
                                          _ptr(iters), _ptr(status), _stream(stream)))


def alb_batch_variants(precision):
    """[(block, min_blocks), ...] of the compiled batched-kernel variants."""
    n = ctypes.c_int()
    block = np.zeros(8, np.int32)
    minb = np.zeros(8, np.int32)
    _check(lib().alb_batch_variants(int(precision), ctypes.byref(n), block.ctypes.data,
                                    minb.ctypes.data))
    return [(int(block[v]), int(minb[v])) for v in range(n.value)]


def alb_batch_create(cfgs, stream=None):
    arr = (alb_config * len(cfgs))(*cfgs)
    b = ctypes.c_void_p()
    _check(lib().alb_batch_create(arr, len(cfgs), _stream(stream), ctypes.byref(b)))
    return b


def alb_batch_flow(b, i):
    h = ctypes.c_void_p()
    _check(lib().alb_batch_flow(b, int(i), ctypes.byref(h)))
    return h


def alb_batch_step(b, nsteps):
    return _check(lib().alb_batch_step(b, int(nsteps)))


def alb_batch_sync(b, timeout_ms=-1):
    return _check(lib().alb_batch_sync(b, int(timeout_ms)))


def alb_batch_tune(b, trials=3):
    return _check(lib().alb_batch_tune(b, int(trials)))


def alb_batch_get_tuning(b, precision) -> dict:
    t = alb_batch_tuning()
    _check(lib().alb_batch_get_tuning(b, int(precision), ctypes.byref(t)))
    return {"variant": t.variant, "tile_w": list(t.tile_w), "dynamic": t.dynamic,
            "blocks_per_sm": t.blocks_per_sm}


def alb_batch_set_tuning(b, precision, variant=0, tile_w=(64, 128, 128), dynamic=1,
                         blocks_per_sm=0):
    t = alb_batch_tuning(variant, (ctypes.c_int * 3)(*tile_w), dynamic, blocks_per_sm)
    return _check(lib().alb_batch_set_tuning(b, int(precision), ctypes.byref(t)))


def alb_batch_destroy(b):
    return _check(lib().alb_batch_destroy(b))


class Flow:
    """One flow on the GPU. Fields are (ny, nx) arrays. Owns its alb_handle,
    unless it wraps a flow of a batch (`handle` given), which the batch owns."""

    def __init__(self, nx, ny, handle=None, **cfg):
        self.cfg = alb_config_default(nx=nx, ny=ny, **cfg)
        self.nx, self.ny = nx, ny
        self.owned = handle is None
        self.h = alb_create(self.cfg) if handle is None else handle

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value and self.owned:
            alb_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, rhoux, rhouy, rhoE):
        return alb_init(self.h, rho, rhoux, rhouy, rhoE)

    def step(self, n):
        return alb_step(self.h, n)

    def sync(self, timeout_ms=-1):
        return alb_sync(self.h, timeout_ms)

    def moments(self):
        n = self.nx * self.ny
        out = [np.empty(n) for _ in range(4)]
        alb_moments(self.h, out)
        return [a.reshape(self.ny, self.nx) for a in out]

    def shifts(self):
        n = self.nx * self.ny
        ux = np.empty(n, np.int8)
        uy = np.empty(n, np.int8)
        alb_shifts(self.h, ux, uy)
        return ux.reshape(self.ny, self.nx), uy.reshape(self.ny, self.nx)

    def next_shifts(self):
        n = self.nx * self.ny
        ux = np.empty(n, np.int8)
        uy = np.empty(n, np.int8)
        alb_next_shifts(self.h, ux, uy)
        return ux.reshape(self.ny, self.nx), uy.reshape(self.ny, self.nx)

    def populations(self):
        """(f, g), each (Q, ny, nx) float64: the post-collision populations
        (Q = 21, or 49 on D2Q49)."""
        n, q = self.nx * self.ny, (49 if self.cfg.stencil == ALB_D2Q49 else 21)
        f = np.empty(q * n)
        g = np.empty(q * n)
        alb_populations(self.h, f, g)
        return f.reshape(q, self.ny, self.nx), g.reshape(q, self.ny, self.nx)

    def primitives(self):
        n = self.nx * self.ny
        out = [np.empty(n) for _ in range(4)]
        alb_primitives(self.h, out)
        return [a.reshape(self.ny, self.nx) for a in out]

    def checkpoint(self):
        return alb_checkpoint_save(self.h)

    def restore(self, buf):
        return alb_checkpoint_load(self.h, buf)

    def stats(self):
        return alb_stats_get(self.h)

    def totals(self):
        return alb_totals(self.h)


class Batch:
    """Many flows advanced together (alb_batch_*). specs: list of dicts with
    nx, ny and alb_config fields; flows[i] is a Flow wrapping flow i."""

    def __init__(self, specs, stream=None):
        cfgs = [alb_config_default(**sp) for sp in specs]
        self.b = alb_batch_create(cfgs, stream)
        self.flows = [Flow(sp["nx"], sp["ny"], handle=alb_batch_flow(self.b, i),
                           **{k: v for k, v in sp.items() if k not in ("nx", "ny")})
                      for i, sp in enumerate(specs)]

    def step(self, n):
        return alb_batch_step(self.b, n)

    def sync(self, timeout_ms=-1):
        return alb_batch_sync(self.b, timeout_ms)

    def tune(self, trials=3):
        return alb_batch_tune(self.b, trials)

    def tuning(self, precision):
        return alb_batch_get_tuning(self.b, precision)

    def set_tuning(self, precision, **kw):
        return alb_batch_set_tuning(self.b, precision, **kw)

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            for f in self.flows:
                f.h = None
            alb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop (alb_server_*, alb_submit, alb_poll). submit() takes host
    fields (copied at once) or a fill(rho, rhoux, rhouy, rhoE) callable that
    writes (ny, nx) float64 views at admission on the worker thread."""

    def __init__(self, **kw):
        c = alb_server_config()
        _check(lib().alb_server_config_default(ctypes.byref(c)))
        for k, v in kw.items():
            setattr(c, k, v)
        self.s = ctypes.c_void_p()
        _check(lib().alb_server_create(ctypes.byref(c), ctypes.byref(self.s)))
        self._meta = {}  # id -> (nx, ny, keep, callback keep-alive)

    def submit(self, nsteps, fields=None, fill=None, keep_result=True, **cfg):
        c = alb_config_default(**cfg)
        r = alb_request()
        r.cfg = c
        r.nsteps = int(nsteps)
        r.keep_result = 1 if keep_result else 0
        keep_alive = None
        if fields is not None:
            arrs = [np.ascontiguousarray(a, np.float64).ravel() for a in fields]
            r.rho, r.rhoux, r.rhouy, r.rhoE = [a.ctypes.data for a in arrs]
            keep_alive = arrs
        else:
            nx, ny = c.nx, c.ny

            def _fill(user, a, b, cc, d):
                try:
                    outs = [np.ctypeslib.as_array(p, shape=(ny, nx)) for p in (a, b, cc, d)]
                    fill(*outs)
                    return 0
                except Exception:
                    return 1
            keep_alive = FILL_FN(_fill)
            r.fill = keep_alive
        rid = ctypes.c_uint64()
        _check(lib().alb_submit(self.s, ctypes.byref(r), ctypes.byref(rid)))
        self._meta[rid.value] = (c.nx, c.ny, keep_result,
                                 keep_alive if fields is None else None)
        return rid.value

    def poll(self, rid):
        """(state, result) with result a dict once DONE or FAILED, else None."""
        if rid not in self._meta:  # collected already or never submitted
            st = ctypes.c_int()
            _check(lib().alb_poll(self.s, ctypes.c_uint64(rid), ctypes.byref(st), None))
        nx, ny, keep, _ = self._meta[rid]
        st = ctypes.c_int()
        res = alb_result()
        outs = None
        if keep:
            outs = [np.empty((ny, nx)) for _ in range(4)]
            res.rho, res.rhoux, res.rhouy, res.rhoE = [a.ctypes.data for a in outs]
        _check(lib().alb_poll(self.s, ctypes.c_uint64(rid), ctypes.byref(st), ctypes.byref(res)))
        if st.value not in (ALB_DONE, ALB_FAILED):
            return st.value, None
        del self._meta[rid]
        out = {"status": res.status, "steps": int(res.steps), "t_submit": res.t_submit,
               "t_admit": res.t_admit, "t_done": res.t_done,
               "stats": {k: int(getattr(res.stats, k)) for k, _ in alb_stats._fields_}}
        if keep:
            out["moments"] = outs
        return st.value, out

    def drain(self, timeout_ms=-1):
        return _check(lib().alb_server_drain(self.s, int(timeout_ms)))

    def stats(self):
        st = alb_server_stats()
        _check(lib().alb_server_stats_get(self.s, ctypes.byref(st)))
        out = {k: getattr(st, k) for k, _ in alb_server_stats._fields_}
        out["ns_per_update"] = list(st.ns_per_update)
        return out

    def close(self):
        if getattr(self, "s", None) is not None and self.s.value:
            alb_server_destroy_(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alb_server_destroy_(s):
    return _check(lib().alb_server_destroy(s))
