"""FP64 CPU oracle for the frozen-particle dual-time EDAC-SPH scheme.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The CUDA library never
imports this package, and this package never imports the library.

The arithmetic lives in ``dtsph_oracle.c`` (plain C, IEEE double, no FMA
contraction). This module compiles it with gcc on first use and marshals numpy
arrays through ctypes. Each wrapper names the part of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dtsph_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int32),
        ("periodic", C.c_int32 * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
        ("h", C.c_double),
        ("m", C.c_double),
        ("rho0", C.c_double),
        ("beta", C.c_double),
        ("v_ref", C.c_double),
        ("nu", C.c_double),
        ("dt", C.c_double),
        ("eta", C.c_double),
        ("alpha", C.c_double),
        ("g", C.c_double * 3),
        ("eps", C.c_double),
        ("stag_tol", C.c_double),
        ("stag_window", C.c_int32),
        ("max_iter", C.c_int32),
        ("edac", C.c_int32),
        ("edac_h2_literal", C.c_int32),
        ("fixed_iters", C.c_int32),
        ("use_bruteforce", C.c_int32),
        ("shifting", C.c_int32),
        ("steady", C.c_int32),
        ("free_surface", C.c_int32),
        ("moving", C.c_int32),
    ]


class OrcStats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("reason", C.c_int32), ("rp", C.c_double), ("rv", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available). Returns the .so path."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.run(base[:6] + ["-fopenmp"] + base[6:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def compile_source(src: str, out_path: str) -> str:
    """Compiles oracle C source text with the flags of build() into out_path."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src)
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", c_path, "-o",
            out_path, "-lm"]
    try:
        subprocess.run(base[:6] + ["-fopenmp"] + base[6:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    return out_path


def source() -> str:
    """The oracle's C source text."""
    with open(_SRC) as f:
        return f.read()


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = bind(_LIB_PATH)
    return _lib


def bind(path: str):
    """Loads a compiled copy of the oracle and declares its entry points."""
    L = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    i64p = C.POINTER(C.c_int64)
    P = C.POINTER(OrcParams)
    L.orc_w.restype = C.c_double
    L.orc_w.argtypes = [C.c_double, C.c_double, C.c_int]
    L.orc_dwdr.restype = C.c_double
    L.orc_dwdr.argtypes = [C.c_double, C.c_double, C.c_int]
    L.orc_neighbors.restype = C.c_int64
    L.orc_neighbors.argtypes = [P, C.c_int64, dp, i64p, i64p, C.c_int64]
    L.orc_rates.restype = C.c_int
    L.orc_rates.argtypes = [P, C.c_int64, C.c_int64, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_rates_vt.restype = C.c_int
    L.orc_rates_vt.argtypes = [P, C.c_int64, C.c_int64, dp, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_stop_reason.restype = C.c_int
    L.orc_stop_reason.argtypes = [P, C.c_int32, dp, dp]
    L.orc_step.restype = C.c_int
    L.orc_step.argtypes = [P, C.c_int64, C.c_int64, dp, dp, dp, dp, dp, C.POINTER(OrcStats), dp, dp, dp]
    L.orc_run.restype = C.c_int
    L.orc_run.argtypes = [P, C.c_int64, C.c_int64, dp, dp, dp, dp, dp, C.c_int32, C.POINTER(OrcStats)]
    L.orc_prepare_positions.restype = C.c_int
    L.orc_prepare_positions.argtypes = [P, C.c_int64, dp]
    L.orc_shift.restype = C.c_int
    L.orc_shift.argtypes = [P, C.c_int64, C.c_int64, dp, dp, dp]
    L.orc_num_threads.restype = C.c_int
    L.orc_set_num_threads.argtypes = [C.c_int]
    return L


# ---------------------------------------------------------------- marshalling

_DEFAULTS = dict(
    periodic=(0, 0, 0), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), rho0=1.0, beta=10.0, v_ref=1.0,
    eta=0.01, alpha=0.0, g=(0.0, 0.0, 0.0), eps=1e-3, stag_tol=0.05, stag_window=4, max_iter=1000,
    edac=1, edac_h2_literal=0, fixed_iters=0, use_bruteforce=0, shifting=0, steady=0, free_surface=0,
    moving=0,
)


def make_params(cfg: dict, **over) -> OrcParams:
    """Fill the oracle's parameter struct from a plain dict (see ``synth``)."""
    keys = set(_DEFAULTS) | {"dim", "h", "m", "nu", "dt"}
    d = dict(_DEFAULTS)
    d.update({k: v for k, v in cfg.items() if k in keys})
    d.update({k: v for k, v in over.items() if k in keys})
    P = OrcParams()
    P.dim = int(d["dim"])
    for a in range(3):
        P.periodic[a] = int(d["periodic"][a]) if a < len(d["periodic"]) else 0
        P.lo[a] = float(d["lo"][a]) if a < len(d["lo"]) else 0.0
        P.hi[a] = float(d["hi"][a]) if a < len(d["hi"]) else 1.0
        P.g[a] = float(d["g"][a]) if a < len(d["g"]) else 0.0
    for k in ("h", "m", "rho0", "beta", "v_ref", "nu", "dt", "eta", "alpha", "eps", "stag_tol"):
        setattr(P, k, float(d[k]))
    for k in ("stag_window", "max_iter", "edac", "edac_h2_literal", "fixed_iters", "use_bruteforce", "shifting",
              "steady", "free_surface", "moving"):
        setattr(P, k, int(d[k]))
    return P


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def w(r, h, dim):
    """Quintic spline W(r, h)."""
    return lib().orc_w(float(r), float(h), int(dim))


def dwdr(r, h, dim):
    """dW/dr of the quintic spline."""
    return lib().orc_dwdr(float(r), float(h), int(dim))


def neighbors(cfg: dict, x, **over):
    """Neighbour lists N(i) = {j != i : |r_ij| < 3h}, ascending j.

    Returns (start[n+1], idx) as int64 arrays (CSR)."""
    P = make_params(cfg, **over)
    x = _f64(x)
    n = x.shape[0]
    start = np.zeros(n + 1, np.int64)
    cap = max(1, n * 64 if P.dim == 2 else n * 160)
    idx = np.zeros(cap, np.int64)
    tot = lib().orc_neighbors(C.byref(P), n, _dp(x), start.ctypes.data_as(C.POINTER(C.c_int64)),
                              idx.ctypes.data_as(C.POINTER(C.c_int64)), cap)
    if tot < 0:
        raise MemoryError("oracle neighbour search failed")
    if tot > cap:
        idx = np.zeros(tot, np.int64)
        lib().orc_neighbors(C.byref(P), n, _dp(x), start.ctypes.data_as(C.POINTER(C.c_int64)),
                            idx.ctypes.data_as(C.POINTER(C.c_int64)), tot)
    return start, idx[:tot].copy()


def rates(cfg: dict, x, v, p, vw=None, nf=None, vt=None, **over):
    """dp/dtau and F (the momentum right-hand side) at a given state, with the
    advective terms of a pseudo-velocity vt (fluid only) if given.

    x holds fluid then wall positions; v, p are fluid only. Returns (ap, F, pw, vghost)."""
    P = make_params(cfg, **over)
    x = _f64(x)
    dim = P.dim
    nf = v.shape[0] if nf is None else nf
    nw = x.shape[0] - nf
    v = _f64(v)
    p = _f64(p)
    vw = _f64(np.zeros((max(nw, 1), dim)) if vw is None or nw == 0 else vw)
    ap = np.zeros(max(nf, 1))
    F = np.zeros((max(nf, 1), dim))
    pw = np.zeros(max(nw, 1))
    vg = np.zeros((max(nw, 1), dim))
    vt = None if vt is None else _f64(vt)
    if lib().orc_rates_vt(C.byref(P), nf, nw, _dp(x), _dp(v), _dp(p), _dp(vw), _dp(vt) if vt is not None else None,
                          _dp(ap), _dp(F), _dp(pw), _dp(vg)):
        raise MemoryError("oracle rates failed")
    return ap[:nf], F[:nf], pw[:nw], vg[:nw]


def shift(cfg: dict, x, v, p, nf=None, **over):
    """Particle shifting alone (Sec. 3.5, Eqs. shift-deltar and shift-correct)
    at a given state: neighbour lists at x (fluid then walls), the shift of every
    fluid particle and the Taylor correction of V and p. Returns the shifted
    fluid positions and the corrected (V, p); the inputs are not changed."""
    P = make_params(cfg, **over)
    x = _f64(x).copy()
    v = _f64(v).copy()
    p = _f64(p).copy()
    nf = v.shape[0] if nf is None else nf
    nw = x.shape[0] - nf
    if lib().orc_shift(C.byref(P), nf, nw, _dp(x), _dp(v), _dp(p)):
        raise MemoryError("oracle shift failed")
    return x[:nf], v, p


def stop_reason(cfg: dict, hist_p, hist_v, **over):
    P = make_params(cfg, **over)
    hp = _f64(hist_p)
    hv = _f64(hist_v)
    return lib().orc_stop_reason(C.byref(P), len(hp), _dp(hp), _dp(hv))


class State:
    """Oracle simulation state (fluid then walls in x)."""

    def __init__(self, cfg: dict, x, v, p, v_prev=None, vw=None, nf=None, **over):
        self.cfg = dict(cfg)
        self.over = dict(over)
        self.P = make_params(cfg, **over)
        dim = self.P.dim
        self.x = _f64(x).copy()
        if lib().orc_prepare_positions(C.byref(self.P), self.x.shape[0], _dp(self.x)):
            raise ValueError("a particle position is not finite")
        self.v = _f64(v).copy()
        self.nf = self.v.shape[0] if nf is None else nf
        self.nw = self.x.shape[0] - self.nf
        self.p = _f64(p).copy()
        self.v_prev = (self.v if v_prev is None else _f64(v_prev)).copy()
        self.vw = _f64(np.zeros((max(self.nw, 1), dim)) if vw is None or self.nw == 0 else vw).copy()
        self.t = 0.0
        self.stats = []

    def step(self, nsteps: int = 1, hist: bool = False, keep_x0: bool = False):
        """Advance nsteps real steps (Algorithm 2, or Algorithm 1 with moving =
        1 or 2). Returns the per-step stats (with the residual history, the
        positions r^0 after the predictor and the pseudo-time positions r^K at
        the end of the loop if asked)."""
        out = []
        cap = max(1, self.P.fixed_iters if self.P.fixed_iters > 0 else self.P.max_iter)
        for _ in range(nsteps):
            st = OrcStats()
            hbuf = np.zeros(2 * cap) if hist else None
            x0 = np.zeros_like(self.x) if keep_x0 else None
            xk = np.zeros_like(self.x) if keep_x0 else None
            rc = lib().orc_step(C.byref(self.P), self.nf, self.nw, _dp(self.x), _dp(self.v), _dp(self.v_prev),
                                _dp(self.p), _dp(self.vw), C.byref(st), _dp(hbuf) if hist else None,
                                _dp(x0) if keep_x0 else None, _dp(xk) if keep_x0 else None)
            if rc:
                raise MemoryError("oracle step failed")
            rec = dict(iters=st.iters, reason=st.reason, rp=st.rp, rv=st.rv)
            if hist:
                rec["hist_p"] = hbuf[: st.iters].copy()
                rec["hist_v"] = hbuf[cap: cap + st.iters].copy()
            if keep_x0:
                rec["x0"] = x0
                rec["xk"] = xk
            out.append(rec)
            self.t += self.P.dt
        self.stats.extend(out)
        return out


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(int(t))
