"""Seeded synthetic inputs for the DTSPH workloads.

This module holds the input generators that both the oracle and the CUDA
library are fed from: particle lattices, seeded jitter, initial fields and
parameter sets. It holds none of the method's arithmetic (no kernel, no rate,
no integrator); the random numbers are a splitmix64 stream written from its
published definition (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), so the same seed gives the same inputs on every
machine.

Workloads (shapes and parameters follow the paper's test cases, Sec. 4):
  tgv2d    2D Taylor-Green vortex, periodic unit square, jittered lattice,
           exact initial field of Eq. (tgv_sol) (Sec. 4.1).
  cavity2d 2D lid-driven cavity, regular lattice, three layers of wall
           particles, lid moving at U (Sec. 4.2).
  tgv3d    3D periodic Taylor-Green vortex on [0, 2 pi]^3 (textbook initial
           field; not one of the paper's cases).
  batch    many independent tgv2d instances of uneven sizes and Reynolds
           numbers.

Default parameters: rho0 = 1, m = rho0 dx^d, h = dx, V_ref = U, beta = 10
(c = 10 U), dt = 0.25 h / U (Sec. 3.4), eps = 1e-3, eta = 0.01, alpha = 0.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """The first `count` outputs (after `offset`) of splitmix64 seeded with `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def base_params(dim: int, dx: float, U: float, nu: float, *, beta: float = 10.0, cfl: float = 0.25,
                h_over_dx: float = 1.0, rho0: float = 1.0, eps: float = 1e-3) -> dict:
    h = h_over_dx * dx
    return dict(
        dim=dim, h=h, dx=dx, m=rho0 * dx ** dim, rho0=rho0, beta=beta, v_ref=U, nu=nu,
        dt=cfl * h / U, eta=0.01, alpha=0.0, g=(0.0, 0.0, 0.0), eps=eps, stag_tol=0.05,
        stag_window=4, max_iter=1000, edac=1, edac_h2_literal=0, fixed_iters=0,
    )


def _wrap(x: np.ndarray, lo: float, hi: float) -> np.ndarray:
    L = hi - lo
    x = np.where(x >= hi, x - L, x)
    return np.where(x < lo, x + L, x)


def tgv_exact(x: np.ndarray, y: np.ndarray, t: float, U: float = 1.0, re: float = 100.0):
    """Taylor-Green solution of Eq. (tgv_sol) on the unit square (L = 1)."""
    b = -8.0 * math.pi ** 2 / re
    e = U * math.exp(b * t)
    u = -e * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    v = e * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    p = -(U ** 2) * math.exp(2 * b * t) * (np.cos(4 * np.pi * x) + np.cos(4 * np.pi * y)) / 4.0
    return u, v, p


def tgv2d(n: int = 50, re: float = 100.0, U: float = 1.0, jitter: float = 0.1, seed: int = 1904, **kw) -> dict:
    """2D Taylor-Green vortex with n*n particles on [0, 1)^2.

    Lattice points ((i + 1/2) dx, (j + 1/2) dx), particle index j*n + i; each
    coordinate displaced by jitter*dx*U[-1, 1) from splitmix64(seed) (x offsets
    are draws 0..N-1, y offsets draws N..2N-1); fields from Eq. (tgv_sol) at the
    displaced positions; V^{n-1} is the exact field at t = -dt."""
    dx = 1.0 / n
    cfg = base_params(2, dx, U, U * 1.0 / re, **kw)
    cfg.update(periodic=(1, 1, 0), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), workload="tgv2d", n_side=n, re=re)
    N = n * n
    i = np.arange(N) % n
    j = np.arange(N) // n
    r = uniform01(seed, 2 * N)
    x = (i + 0.5) * dx + jitter * dx * (2.0 * r[:N] - 1.0)
    y = (j + 0.5) * dx + jitter * dx * (2.0 * r[N:] - 1.0)
    x = _wrap(x, 0.0, 1.0)
    y = _wrap(y, 0.0, 1.0)
    u, v, p = tgv_exact(x, y, 0.0, U, re)
    um, vm, _ = tgv_exact(x, y, -cfg["dt"], U, re)
    return dict(cfg=cfg, x=np.stack([x, y], 1), v=np.stack([u, v], 1), p=p,
                v_prev=np.stack([um, vm], 1), vw=None, nf=N)


def cavity2d(n: int = 200, re: float = 100.0, U: float = 1.0, layers: int = 3, eps: float = 1e-4, **kw) -> dict:
    """Lid-driven cavity: n*n fluid particles on the regular lattice of [0, 1]^2
    at rest, plus `layers` rings of wall particles on the same lattice outside
    it; the wall particles above y = 1 move at (U, 0), the rest are still. The
    pseudo-time tolerance is the paper's for its cavity runs (Sec. 4, the
    lid-driven-cavity problem: beta = 10, eps = 1e-4); with 1e-3 the loosely
    converged pressure lets a particle at the lid's downstream corner enter the
    side wall at Re = 100 within a few hundred steps."""
    dx = 1.0 / n
    cfg = base_params(2, dx, U, U * 1.0 / re, eps=eps, **kw)
    lo = -layers * dx
    hi = 1.0 + layers * dx
    cfg.update(periodic=(0, 0, 0), lo=(lo, lo, 0.0), hi=(hi, hi, 1.0), workload="cavity2d", n_side=n, re=re)
    i = np.arange(n * n) % n
    j = np.arange(n * n) // n
    xf = np.stack([(i + 0.5) * dx, (j + 0.5) * dx], 1)
    m = n + 2 * layers
    ii = np.arange(m * m) % m - layers
    jj = np.arange(m * m) // m - layers
    wall = (ii < 0) | (ii >= n) | (jj < 0) | (jj >= n)
    xw = np.stack([(ii[wall] + 0.5) * dx, (jj[wall] + 0.5) * dx], 1)
    vw = np.zeros_like(xw)
    vw[xw[:, 1] > 1.0, 0] = U
    N = n * n
    return dict(cfg=cfg, x=np.concatenate([xf, xw]), v=np.zeros((N, 2)), p=np.zeros(N),
                v_prev=np.zeros((N, 2)), vw=vw, nf=N)


def couette2d(n: int = 30, re: float = 10.0, U: float = 1.0, layers: int = 3, **kw) -> dict:
    """Plane Couette channel: periodic in x on [0, 1), n*n fluid particles on the
    regular lattice of [0, 1]^2, `layers` rows of wall particles below y = 0
    (still) and above y = 1 (moving at (U, 0)); the fluid starts at u = U y,
    v = 0, p = 0 (the steady solution)."""
    dx = 1.0 / n
    cfg = base_params(2, dx, U, U * 1.0 / re, **kw)
    cfg.update(periodic=(1, 0, 0), lo=(0.0, -layers * dx, 0.0), hi=(1.0, 1.0 + layers * dx, 1.0),
               workload="couette2d", n_side=n, re=re)
    i = np.arange(n * n) % n
    j = np.arange(n * n) // n
    xf = np.stack([(i + 0.5) * dx, (j + 0.5) * dx], 1)
    iw = np.arange(n * 2 * layers) % n
    jw = np.arange(n * 2 * layers) // n
    jw = np.where(jw < layers, jw - layers, jw - layers + n)
    xw = np.stack([(iw + 0.5) * dx, (jw + 0.5) * dx], 1)
    vw = np.zeros_like(xw)
    vw[xw[:, 1] > 1.0, 0] = U
    N = n * n
    v = np.zeros((N, 2))
    v[:, 0] = U * xf[:, 1]
    return dict(cfg=cfg, x=np.concatenate([xf, xw]), v=v, p=np.zeros(N), v_prev=v.copy(), vw=vw, nf=N)


def dambreak2d(n: int = 20, width: float = 1.0, height: float = 2.0, tank_w: float = 4.0, tank_h: float = 2.5,
               layers: int = 3, g: float = 9.81, jitter: float = 0.0, seed: int = 1904, **kw) -> dict:
    """A water column at rest in a tank (a dam-break-like block with a free
    surface): n x (n height/width) fluid particles on the lattice of
    [0, width] x [0, height], spacing dx = width / n, optional jitter of each
    coordinate by jitter*dx*U[-1, 1); `layers` rows of still wall particles
    under the floor (y < 0) and outside both side walls (x < 0, x > tank_w) up to
    tank_h; gravity (0, -g); v_ref = sqrt(2 g height); V = 0, p = 0."""
    dx = width / n
    U = math.sqrt(2.0 * g * height)
    cfg = base_params(2, dx, U, 0.0, **kw)
    cfg.update(periodic=(0, 0, 0), lo=(-layers * dx, -layers * dx, 0.0), hi=(tank_w + layers * dx, tank_h, 1.0),
               g=(0.0, -g, 0.0), workload="dambreak2d", n_side=n)
    ny = int(round(height / dx))
    N = n * ny
    i = np.arange(N) % n
    j = np.arange(N) // n
    r = uniform01(seed, 2 * N)
    xf = np.stack([(i + 0.5) * dx + jitter * dx * (2.0 * r[:N] - 1.0),
                   (j + 0.5) * dx + jitter * dx * (2.0 * r[N:] - 1.0)], 1)
    nxw = int(round(tank_w / dx))
    nyw = int(round(tank_h / dx))
    ii = np.arange(-layers, nxw + layers)
    jj = np.arange(-layers, nyw)
    II, JJ = np.meshgrid(ii, jj)
    wall = (II < 0) | (II >= nxw) | (JJ < 0)
    xw = np.stack([(II[wall] + 0.5) * dx, (JJ[wall] + 0.5) * dx], 1)
    return dict(cfg=cfg, x=np.concatenate([xf, xw]), v=np.zeros((N, 2)), p=np.zeros(N),
                v_prev=np.zeros((N, 2)), vw=np.zeros_like(xw), nf=N)


def tgv3d(n: int = 128, re: float = 1600.0, U: float = 1.0, jitter: float = 0.05, seed: int = 1904, **kw) -> dict:
    """3D Taylor-Green vortex on [0, 2 pi)^3 with n^3 particles: u = U sin x cos y
    cos z, v = -U cos x sin y cos z, w = 0, p = rho0 U^2/16 (cos 2x + cos 2y)(cos 2z
    + 2); nu = U / Re (unit length scale); V^{n-1} = V^0."""
    L = 2.0 * math.pi
    dx = L / n
    cfg = base_params(3, dx, U, U / re, **kw)
    cfg.update(periodic=(1, 1, 1), lo=(0.0, 0.0, 0.0), hi=(L, L, L), workload="tgv3d", n_side=n, re=re)
    N = n ** 3
    i = np.arange(N) % n
    j = (np.arange(N) // n) % n
    k = np.arange(N) // (n * n)
    r = uniform01(seed, 3 * N)
    pos = [(a + 0.5) * dx + jitter * dx * (2.0 * r[s * N:(s + 1) * N] - 1.0) for s, a in enumerate((i, j, k))]
    x, y, z = (_wrap(c, 0.0, L) for c in pos)
    u = U * np.sin(x) * np.cos(y) * np.cos(z)
    v = -U * np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros(N)
    p = cfg["rho0"] * U ** 2 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    V = np.stack([u, v, w], 1)
    return dict(cfg=cfg, x=np.stack([x, y, z], 1), v=V, p=p, v_prev=V.copy(), vw=None, nf=N)


def batch_draws(count: int = 64, seed: int = 861, n_lo: int = 32, n_hi: int = 256):
    """Side counts n_s ~ U{n_lo..n_hi} and Reynolds numbers Re_s = 10^U[2, 3)."""
    r = uniform01(seed, 2 * count)
    sides = n_lo + np.floor(r[:count] * (n_hi - n_lo + 1)).astype(np.int64)
    res = 10.0 ** (2.0 + r[count:])
    return sides, res


def batch(count: int = 64, seed: int = 861, n_lo: int = 32, n_hi: int = 256, jitter_seed: int = 1904, **kw):
    """`count` independent tgv2d instances (list of the tgv2d dicts)."""
    sides, res = batch_draws(count, seed, n_lo, n_hi)
    return [tgv2d(int(n), float(re), seed=jitter_seed + s, **kw) for s, (n, re) in enumerate(zip(sides, res))]
