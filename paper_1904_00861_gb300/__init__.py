"""Python binding of the DTSPH GB300 library (include/dtsph.h).

The functions below carry the C entry points' names and only marshal
arguments: numpy arrays for host pointers, torch CUDA tensors (or raw integer
addresses) for device pointers. Every step of the method runs in the CUDA
library ``_build/libdtsph.so``; there is no other code path. Importing this
package never builds or loads anything; the first call loads the library and
raises if it has not been built (``python -m paper_1904_00861_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdtsph.so")

DTSPH_OK = 0
ERRORS = {
    -1: "DTSPH_E_ARG", -2: "DTSPH_E_STATE", -3: "DTSPH_E_CUDA", -4: "DTSPH_E_OOM",
    -5: "DTSPH_E_CAPACITY", -6: "DTSPH_E_DOMAIN", -7: "DTSPH_E_UNSUPPORTED", -8: "DTSPH_E_TIMEOUT",
    -9: "DTSPH_E_SKIN",
}
for _code, _name in ERRORS.items():
    globals()[_name] = _code
DTSPH_FP64, DTSPH_FP32C = 0, 1
FIELD_POS, FIELD_VEL, FIELD_P, FIELD_VEL_PREV = 0, 1, 2, 3
REASONS = {0: "converged", 1: "stagnated", 2: "max_iter", 3: "nonfinite", 4: "fixed"}


class DtsphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class dtsph_params(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("precision", C.c_int32), ("periodic", C.c_int32 * 3), ("pad0", C.c_int32),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("h", C.c_double), ("m", C.c_double), ("rho0", C.c_double), ("beta", C.c_double), ("v_ref", C.c_double),
        ("nu", C.c_double), ("dt", C.c_double), ("eta", C.c_double), ("alpha", C.c_double),
        ("g", C.c_double * 3), ("eps", C.c_double), ("stag_tol", C.c_double),
        ("stag_window", C.c_int32), ("max_iter", C.c_int32), ("edac", C.c_int32), ("edac_h2_literal", C.c_int32),
        ("fixed_iters", C.c_int32), ("max_neighbors", C.c_int32), ("graph", C.c_int32), ("lanes", C.c_int32),
        ("stages", C.c_int32), ("shifting", C.c_int32), ("steady", C.c_int32), ("free_surface", C.c_int32),
        ("moving", C.c_int32), ("form", C.c_int32), ("skin", C.c_double), ("cell_scale", C.c_double),
        ("list_skin", C.c_double),
    ]


class dtsph_step_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("reason", C.c_int32), ("rp", C.c_double), ("rv", C.c_double),
                ("vmax", C.c_double), ("form", C.c_int32), ("pad", C.c_int32)]


_lib = None

# (name, restype, argtypes) of every exported entry point
_VP, _DP, _I64P = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)
_SIGS = [
    ("dtsph_version", C.c_char_p, []),
    ("dtsph_last_error", C.c_char_p, [_VP]),
    ("dtsph_create", C.c_int, [C.POINTER(dtsph_params), _VP, C.POINTER(_VP)]),
    ("dtsph_destroy", None, [_VP]),
    ("dtsph_set_boundary", C.c_int, [_VP, C.c_int64, _VP, _VP]),
    ("dtsph_set_particles", C.c_int, [_VP, C.c_int64, _VP, _VP, _VP, _VP]),
    ("dtsph_set_particles_device", C.c_int, [_VP, C.c_int64, _VP, _VP, _VP, _VP]),
    ("dtsph_step", C.c_int, [_VP, C.c_int32]),
    ("dtsph_sync", C.c_int, [_VP]),
    ("dtsph_step_count", C.c_int64, [_VP]),
    ("dtsph_read_stats", C.c_int, [_VP, C.c_int64, C.c_int32, C.POINTER(dtsph_step_stats)]),
    ("dtsph_read_field", C.c_int, [_VP, C.c_int32, _VP]),
    ("dtsph_read_field_device", C.c_int, [_VP, C.c_int32, _VP]),
    ("dtsph_read_state", C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    ("dtsph_eval_rates", C.c_int, [_VP, _VP, _VP]),
    ("dtsph_build_neighbors", C.c_int, [_VP]),
    ("dtsph_get_neighbors", C.c_int, [_VP, C.c_int64, _I64P, C.c_int64, _I64P]),
    ("dtsph_probe_iterate", C.c_int, [_VP, C.c_int32, C.POINTER(C.c_float), _DP, _I64P]),
    ("dtsph_tuning", C.c_int, [_VP, C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    ("dtsph_form_stats", C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("dtsph_loop_times", C.c_int, [_VP, C.c_int64, C.c_int32, C.POINTER(C.c_float)]),
    ("dtsph_tuning_candidates", C.c_int, [_VP, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_float), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("dtsph_batch_create", C.c_int, [C.c_int32, C.POINTER(dtsph_params), _VP, C.POINTER(_VP)]),
    ("dtsph_batch_set_boundary", C.c_int, [_VP, C.c_int32, C.c_int64, _VP, _VP]),
    ("dtsph_batch_set_particles", C.c_int, [_VP, _I64P, _VP, _VP, _VP, _VP]),
    ("dtsph_batch_read_stats", C.c_int, [_VP, C.c_int32, C.c_int64, C.c_int32, C.POINTER(dtsph_step_stats)]),
    ("dtsph_kernel_launches", C.c_int64, [_VP]),
    ("dtsph_fma_peak", C.c_int, [C.c_int32, C.POINTER(C.c_double)]),
    ("dtsph_eval_rates_noalloc", C.c_int, [C.POINTER(dtsph_params), C.c_int64, _VP, _VP, _VP, C.c_int64, _VP, _VP,
                                           _VP, _VP, _VP, _VP]),
]


def lib():
    """Loads the CUDA library; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"DTSPH CUDA library not built: {LIB_PATH} is missing "
                              "(run python -m paper_1904_00861_gb300.build)")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return [s[0] for s in _SIGS]


def _check(ctx, rc):
    if rc != DTSPH_OK:
        msg = lib().dtsph_last_error(ctx).decode() if ctx else ""
        raise DtsphError(rc, msg)


def _host(a, dim=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptr(a):
    """Address of a numpy array, a torch tensor, or an integer address."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(f"cannot take the address of {type(a)}")


def make_params(cfg: dict, precision: int = DTSPH_FP64, graph: int = 1, **over) -> dtsph_params:
    """Fill dtsph_params from a plain dict (the keys of ``synth`` configs).
    With moving = 2 and no skin given, the skin is h / 2."""
    d = dict(periodic=(0, 0, 0), lo=(0, 0, 0), hi=(1, 1, 1), rho0=1.0, beta=10.0, v_ref=1.0, eta=0.01, alpha=0.0,
             g=(0, 0, 0), eps=1e-3, stag_tol=0.05, stag_window=4, max_iter=1000, edac=1, edac_h2_literal=0,
             fixed_iters=0, max_neighbors=0, lanes=0, stages=0, shifting=0, steady=0, free_surface=0, moving=0,
             skin=0.0, form=0, cell_scale=0.0, list_skin=0.0)
    d.update(cfg)
    d.update(over)
    p = dtsph_params()
    p.dim = int(d["dim"])
    p.precision = int(d.get("precision", precision))
    p.graph = int(d.get("graph", graph))
    for a in range(3):
        p.periodic[a] = int(d["periodic"][a]) if a < len(d["periodic"]) else 0
        p.lo[a] = float(d["lo"][a]) if a < len(d["lo"]) else 0.0
        p.hi[a] = float(d["hi"][a]) if a < len(d["hi"]) else 1.0
        p.g[a] = float(d["g"][a]) if a < len(d["g"]) else 0.0
    for k in ("h", "m", "rho0", "beta", "v_ref", "nu", "dt", "eta", "alpha", "eps", "stag_tol"):
        setattr(p, k, float(d[k]))
    for k in ("stag_window", "max_iter", "edac", "edac_h2_literal", "fixed_iters", "max_neighbors", "lanes",
              "stages", "shifting", "steady", "free_surface", "moving", "form"):
        setattr(p, k, int(d[k]))
    p.skin = float(d["skin"])
    p.cell_scale = float(d["cell_scale"])
    p.list_skin = float(d["list_skin"])
    if p.moving == 2 and p.skin == 0.0:
        p.skin = 0.5 * p.h
    return p


# ------------------------------------------------------------ entry points

def dtsph_version() -> str:
    return lib().dtsph_version().decode()


def dtsph_create(params: dtsph_params, stream=None) -> int:
    """Returns the context handle (an integer). stream: cudaStream_t address,
    a torch.cuda.Stream, or None."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    out = C.c_void_p()
    _check(None, lib().dtsph_create(C.byref(params), stream, C.byref(out)))
    return out.value


def dtsph_batch_create(params_list, stream=None) -> int:
    """Context of len(params_list) independent instances advanced together."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    arr = (dtsph_params * len(params_list))(*params_list)
    out = C.c_void_p()
    _check(None, lib().dtsph_batch_create(len(params_list), arr, stream, C.byref(out)))
    return out.value


def dtsph_batch_set_boundary(ctx, inst, x, v_wall=None) -> None:
    x = _host(x)
    vw = None if v_wall is None else _host(v_wall)
    _check(ctx, lib().dtsph_batch_set_boundary(ctx, int(inst), x.shape[0], _ptr(x), _ptr(vw)))


def dtsph_batch_set_particles(ctx, nf, x, v, p, v_prev=None) -> None:
    nf = np.ascontiguousarray(nf, dtype=np.int64)
    x, v, p = _host(x), _host(v), _host(p)
    vp = None if v_prev is None else _host(v_prev)
    _check(ctx, lib().dtsph_batch_set_particles(ctx, nf.ctypes.data_as(_I64P), _ptr(x), _ptr(v), _ptr(p), _ptr(vp)))


def dtsph_batch_read_stats(ctx, inst: int, first: int, count: int):
    buf = (dtsph_step_stats * max(count, 1))()
    _check(ctx, lib().dtsph_batch_read_stats(ctx, int(inst), int(first), int(count), buf))
    return [dict(iters=b.iters, reason=b.reason, rp=b.rp, rv=b.rv, vmax=b.vmax, form=b.form) for b in buf[:count]]


def dtsph_destroy(ctx) -> None:
    lib().dtsph_destroy(ctx)


def dtsph_set_boundary(ctx, x, v_wall=None) -> None:
    x = _host(x)
    vw = None if v_wall is None else _host(v_wall)
    _check(ctx, lib().dtsph_set_boundary(ctx, x.shape[0], _ptr(x), _ptr(vw)))


def dtsph_set_particles(ctx, x, v, p, v_prev=None) -> None:
    x, v, p = _host(x), _host(v), _host(p)
    vp = None if v_prev is None else _host(v_prev)
    _check(ctx, lib().dtsph_set_particles(ctx, x.shape[0], _ptr(x), _ptr(v), _ptr(p), _ptr(vp)))


def dtsph_set_particles_device(ctx, nf, x, v, p, v_prev=None) -> None:
    _check(ctx, lib().dtsph_set_particles_device(ctx, int(nf), _ptr(x), _ptr(v), _ptr(p), _ptr(v_prev)))


def dtsph_step(ctx, nsteps: int = 1) -> None:
    _check(ctx, lib().dtsph_step(ctx, int(nsteps)))


def dtsph_sync(ctx) -> None:
    _check(ctx, lib().dtsph_sync(ctx))


def dtsph_step_count(ctx) -> int:
    return lib().dtsph_step_count(ctx)


def dtsph_read_stats(ctx, first: int, count: int):
    buf = (dtsph_step_stats * max(count, 1))()
    _check(ctx, lib().dtsph_read_stats(ctx, int(first), int(count), buf))
    return [dict(iters=b.iters, reason=b.reason, rp=b.rp, rv=b.rv, vmax=b.vmax, form=b.form) for b in buf[:count]]


def dtsph_read_field(ctx, field: int, n: int, comps: int, out=None) -> np.ndarray:
    """One field of the n fluid particles, into `out` (a C-contiguous float64
    host array of n * comps values, e.g. pinned) or a new array."""
    if out is None:
        out = np.empty((n, comps) if comps > 1 else n, np.float64)
    elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size != n * comps:
        raise ValueError("out must be a C-contiguous float64 array of n * comps values")
    _check(ctx, lib().dtsph_read_field(ctx, int(field), _ptr(out)))
    return out


def dtsph_read_state(ctx, n: int, dim: int, out=None):
    """(r^n, V^n, p^n, V^{n-1}) of the n fluid particles in one call, into the
    four C-contiguous float64 host arrays of `out` (e.g. pinned) or new ones."""
    if out is None:
        out = (np.empty((n, dim)), np.empty((n, dim)), np.empty(n), np.empty((n, dim)))
    for a, size in zip(out, (n * dim, n * dim, n, n * dim)):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != size:
            raise ValueError("out must hold C-contiguous float64 arrays of n*dim, n*dim, n, n*dim values")
    _check(ctx, lib().dtsph_read_state(ctx, *[_ptr(a) for a in out]))
    return out


def dtsph_read_field_device(ctx, field: int, out) -> None:
    _check(ctx, lib().dtsph_read_field_device(ctx, int(field), _ptr(out)))


def dtsph_eval_rates(ctx, nf: int, dim: int):
    ap = np.empty(nf, np.float64)
    F = np.empty((nf, dim), np.float64)
    _check(ctx, lib().dtsph_eval_rates(ctx, _ptr(ap), _ptr(F)))
    return ap, F


def dtsph_build_neighbors(ctx) -> None:
    _check(ctx, lib().dtsph_build_neighbors(ctx))


def dtsph_get_neighbors(ctx, i: int, cap: int = 512) -> np.ndarray:
    out = np.zeros(cap, np.int64)
    cnt = C.c_int64()
    _check(ctx, lib().dtsph_get_neighbors(ctx, int(i), out.ctypes.data_as(_I64P), cap, C.byref(cnt)))
    if cnt.value > cap:
        return dtsph_get_neighbors(ctx, i, int(cnt.value))
    return out[: cnt.value].copy()


def dtsph_probe_iterate(ctx, launches: int = 20):
    """Mean duration (ms) of the pseudo-iteration kernel, its algorithmic bytes
    per launch, and the number of cached fluid pairs."""
    ms = C.c_float()
    by = C.c_double()
    npairs = C.c_int64()
    _check(ctx, lib().dtsph_probe_iterate(ctx, int(launches), C.byref(ms), C.byref(by), C.byref(npairs)))
    return float(ms.value), float(by.value), int(npairs.value)


def dtsph_loop_times(ctx, first: int, count: int):
    """Device ms of the pseudo-time loop of steps first .. first+count-1."""
    ms = (C.c_float * max(count, 1))()
    _check(ctx, lib().dtsph_loop_times(ctx, first, count, ms))
    return [float(ms[i]) for i in range(count)]


def dtsph_tuning_candidates(ctx):
    """(staging depth in use, [(lanes, stages, ms per launch), ...] timed by the
    autotuner, in the order timed)."""
    cnt, s_use = C.c_int32(), C.c_int32()
    _check(ctx, lib().dtsph_tuning_candidates(ctx, 0, None, None, None, C.byref(cnt), C.byref(s_use)))
    n = cnt.value
    la, st, ms = (C.c_int32 * max(n, 1))(), (C.c_int32 * max(n, 1))(), (C.c_float * max(n, 1))()
    _check(ctx, lib().dtsph_tuning_candidates(ctx, n, la, st, ms, C.byref(cnt), C.byref(s_use)))
    return s_use.value, [(int(la[i]), int(st[i]), float(ms[i])) for i in range(n)]


def dtsph_form_stats(ctx):
    """{"kstar", "ms": [cache pass, cached iteration, uncached iteration],
    "steps_cache", "steps_nocache", "steps_switched"} of the pair-term form
    (dtsph_params.form)."""
    k = C.c_double()
    ms = (C.c_float * 3)()
    a, b, sw = C.c_int64(), C.c_int64(), C.c_int64()
    _check(ctx, lib().dtsph_form_stats(ctx, C.byref(k), ms, C.byref(a), C.byref(b), C.byref(sw)))
    return {"kstar": k.value, "ms": [float(m) for m in ms], "steps_cache": a.value, "steps_nocache": b.value,
            "steps_switched": sw.value}


def dtsph_tuning(ctx):
    """(lanes per particle in use, {lanes: ms per launch} measured by the autotuner)."""
    lanes = C.c_int32()
    ms = (C.c_float * 4)()
    _check(ctx, lib().dtsph_tuning(ctx, C.byref(lanes), ms))
    return lanes.value, {L: float(m) for L, m in zip((1, 2, 4, 8), ms) if m >= 0}


def dtsph_kernel_launches(ctx) -> int:
    return lib().dtsph_kernel_launches(ctx)


def dtsph_eval_rates_noalloc(params: dtsph_params, nf, x, v, p, ap, F, nw=0, xw=None, vw=None, status=None,
                             stream=None) -> None:
    """Allocation-free rate evaluation: every array is a device tensor or a
    device address (status: an optional device int32 that receives the call's
    device-side status); only enqueues work on `stream`."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    rc = lib().dtsph_eval_rates_noalloc(C.byref(params), int(nf), _ptr(x), _ptr(v), _ptr(p), int(nw), _ptr(xw),
                                        _ptr(vw), _ptr(ap), _ptr(F), _ptr(status), stream)
    if rc != DTSPH_OK:
        raise DtsphError(rc, "dtsph_eval_rates_noalloc")


def dtsph_fma_peak(precision: int) -> float:
    """Measured vector FMA throughput of the current device in FLOP/s (FP64 for
    DTSPH_FP64, FP32 for DTSPH_FP32C)."""
    out = C.c_double()
    rc = lib().dtsph_fma_peak(int(precision), C.byref(out))
    if rc != DTSPH_OK:
        raise DtsphError(rc, "dtsph_fma_peak")
    return out.value


def dtsph_last_error(ctx) -> str:
    return lib().dtsph_last_error(ctx).decode()


# ------------------------------------------------------------ convenience

class Batch:
    """Owns one batch context: ``Batch([cfg0, cfg1, ...], precision=...)``, then
    ``set_state(list_of_instance_dicts)`` (each with x, v, p, v_prev, nf and
    optional vw walls appended after the fluid in x) and ``step(n)``."""

    def __init__(self, cfgs, precision: int = DTSPH_FP64, stream=None, graph: int = 2, **over):
        self.cfgs = [dict(c) for c in cfgs]
        self.dim = int(cfgs[0]["dim"])
        self.params = [make_params(c, precision=precision, graph=graph, **over) for c in cfgs]
        self.ctx = dtsph_batch_create(self.params, stream)
        self.nfs = []

    def close(self):
        if self.ctx:
            dtsph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, insts):
        for i, d in enumerate(insts):
            nf = d["nf"]
            if len(d["x"]) > nf:
                dtsph_batch_set_boundary(self.ctx, i, d["x"][nf:], d.get("vw"))
        self.nfs = [d["nf"] for d in insts]
        cat = lambda k: np.concatenate([np.asarray(d[k], np.float64)[: d["nf"]] for d in insts])
        vp = None if any(d.get("v_prev") is None for d in insts) else cat("v_prev")
        dtsph_batch_set_particles(self.ctx, self.nfs, cat("x"), cat("v"), cat("p"), vp)

    def step(self, nsteps: int = 1):
        dtsph_step(self.ctx, nsteps)

    def sync(self):
        dtsph_sync(self.ctx)

    def stats(self, inst: int, first=0, count=None):
        n = dtsph_step_count(self.ctx)
        count = n - first if count is None else count
        return dtsph_batch_read_stats(self.ctx, inst, first, count)

    def form_stats(self):
        return dtsph_form_stats(self.ctx)

    def field(self, which: int):
        """One array per instance."""
        comps = 1 if which == FIELD_P else self.dim
        allv = dtsph_read_field(self.ctx, which, sum(self.nfs), comps)
        return np.split(allv, np.cumsum(self.nfs)[:-1])


class Simulation:
    """Owns one context. ``Simulation(cfg, precision=DTSPH_FP32C)`` then
    ``set_state(x, v, p, v_prev, walls=(xw, vw))`` and ``step(n)``."""

    def __init__(self, cfg: dict, precision: int = DTSPH_FP64, stream=None, graph: int = 2, **over):
        self.cfg = dict(cfg)
        self.dim = int(cfg["dim"])
        self.params = make_params(cfg, precision=precision, graph=graph, **over)
        self.ctx = dtsph_create(self.params, stream)
        self.nf = 0

    def close(self):
        if self.ctx:
            dtsph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, x, v, p, v_prev=None, walls=None, nf=None):
        nf = len(v) if nf is None else nf
        x = np.asarray(x, np.float64)
        if walls is None and x.shape[0] > nf:
            walls = (x[nf:], None)
        if walls is not None:
            dtsph_set_boundary(self.ctx, walls[0], walls[1])
        dtsph_set_particles(self.ctx, x[:nf], v, p, v_prev)
        self.nf = nf

    def step(self, nsteps: int = 1):
        dtsph_step(self.ctx, nsteps)

    def sync(self):
        dtsph_sync(self.ctx)

    def stats(self, first=0, count=None):
        n = dtsph_step_count(self.ctx)
        count = n - first if count is None else count
        return dtsph_read_stats(self.ctx, first, count)

    def form_stats(self):
        return dtsph_form_stats(self.ctx)

    def field(self, which: int) -> np.ndarray:
        comps = 1 if which == FIELD_P else self.dim
        return dtsph_read_field(self.ctx, which, self.nf, comps)

    @property
    def x(self):
        return self.field(FIELD_POS)

    @property
    def v(self):
        return self.field(FIELD_VEL)

    @property
    def p(self):
        return self.field(FIELD_P)

    @property
    def v_prev(self):
        return self.field(FIELD_VEL_PREV)

    def rates(self):
        return dtsph_eval_rates(self.ctx, self.nf, self.dim)
