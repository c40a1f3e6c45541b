"""Benchmark: particle-pseudo-iterations per second of the frozen EDAC-DTSPH
hot path on one GB300 (or N independent replicas, one per GPU).

Workload (default): the batched ensemble the metric is quoted on, 64
independent 2D periodic Taylor-Green instances with side counts drawn uniformly
from 32..256 (seed 861; 1,499,340 particles in all), Re log-uniform in
[100, 1000], lattices jittered by +-0.1 dx, quintic kernel h = dx, beta = 10,
dt = 0.25 h, eps = 1e-3, FP32-compensated, all instances in one persistent
loop launch per real step inside a CUDA graph, lanes and staging depth
autotuned. One "step" is one real time step of every instance: neighbour
rebuild, state-n rates and predictor, the pseudo-time loop until the
convergence test of the paper holds, and the position update. The metric
counts fluid particles times pseudo-iterations actually taken.

The FP32-compensated path gives `value`; the plain FP64 GPU path is timed in the
same run on the same steps ("fp64" key). The FP64 oracle runs the same warm-up
plus timed steps on the host cores; the L-inf relative velocity error of both
GPU paths against it (`linf_vs_oracle`) and the oracle's own rate
(`cpu_baseline`) come from that run. `e2e` times the same steps through the C
ABI with host arrays (state copied in, step, state copied out).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batch|tgv2d|tgv3d|cavity|dambreak]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "particle-pseudo-iterations/sec (FP32-comp batched vs plain FP64, same GPU) at stated L∞ err"
UNIT = "particle-iterations/s"


# DRAM traffic of the loop kernel from the Nsight Compute captures summarised
# under profiles/: (workload, dim, lanes, stages, pair-term form) -> (DRAM bytes
# of the captured launch, dram__bytes_read.sum + dram__bytes_write.sum;
# algorithmic bytes of that launch; source). A launch's bytes depend on the
# iterations of its step, so the line reports, launch by launch, the captured
# bytes per algorithmic byte of the form it ran times its own algorithmic bytes.
# A variant not listed (a step that switched forms included), or one whose
# kernel changed after its capture, reports null.
NCU_TRAFFIC = {
    ("batch-64x-tgv2d", 2, 1, 2, 1): (6.357158e9 + 0.056701e9, 6.667369e9, "profiles/k_loop_async_batch64_tgv2d.md"),
    ("batch-64x-tgv2d", 2, 1, 2, 2): (0.682724e9 + 0.142967e9, 2.441234e9, "profiles/k_loop_async_batch64_tgv2d.md"),
}

# FP32 flops of the loop without the pair cache, from the FP32 operation counters
# of an Nsight Compute capture (fadd + fmul + 2 ffma, thread instructions):
# dim -> (flops per pair-iteration, workload, source). The form is bound by
# neither HBM nor the FP32 pipe; this places its launches against the FP32 peak.
NCU_FLOPS_NO_CACHE = {
    2: (62.51, "batch-64x-tgv2d", "profiles/k_loop_async_batch64_tgv2d.md"),
    3: (75.46, "tgv3d 80^3", "profiles/k_loop_no_cache_tgv3d_80.md"),
}


def make_workload(name: str, n_side: int, re: float):
    """Synthetic input and its config record. batch (default: 64 Taylor-Green
    instances of 32^2..256^2 particles, Re 100..1000) is the workload the metric
    is quoted on; tgv2d (200 x 200), tgv3d (128^3) and cavity (200 x 200 +
    walls, Re 100 or 1000) are the other single-GPU configurations; dambreak (a 200 x 400 water column
    in a tank, free surface, artificial viscosity 0.1, shifting, eps 1e-4, as
    in the 2D dam break of Sec. 4) measures the free-surface runs."""
    if name == "tgv2d":
        n = n_side or 200
        d = synth.tgv2d(n, re=re or 100.0)
        cfg = dict(workload=f"tgv2d-{n}x{n}", particles=n * n, re=re or 100.0, dims=2)
    elif name == "tgv3d":
        n = n_side or 128
        d = synth.tgv3d(n, re=re or 1600.0)
        cfg = dict(workload=f"tgv3d-{n}^3", particles=n ** 3, re=re or 1600.0, dims=3)
    elif name == "cavity":
        # particle shifting on, as in the paper's test cases: without it the
        # particles the lid drags into the corner pass through the side wall
        n = n_side or 200
        d = synth.cavity2d(n, re=re or 100.0)
        d["cfg"].update(shifting=1)
        cfg = dict(workload=f"cavity2d-{n}x{n}", particles=n * n, wall_particles=len(d["x"]) - d["nf"],
                   re=re or 100.0, dims=2, shifting="on (Eqs. shift-deltar, shift-correct, after every real step)")
    elif name == "batch":
        count = n_side or 64
        d = synth.batch(count)
        cfg = dict(workload=f"batch-{count}x-tgv2d", instances=count, particles=int(sum(x["nf"] for x in d)),
                   sides="U{32..256} seed 861", re="10^U[2,3)", dims=2)
    elif name == "dambreak":
        n = n_side or 200
        d = synth.dambreak2d(n, eps=1e-4)
        d["cfg"].update(alpha=0.1, free_surface=1, shifting=1)
        cfg = dict(workload=f"dambreak2d-{n}x{2 * n}", particles=d["nf"], wall_particles=len(d["x"]) - d["nf"],
                   column="1 m x 2 m at rest, p = 0, gravity 9.81", tank="4 m x 2.5 m, 3 wall layers", dims=2,
                   alpha=0.1, free_surface="on", shifting="on")
    else:
        raise ValueError(name)
    first = d[0] if isinstance(d, list) else d
    cfg.update(dt="0.25h", beta=first["cfg"]["beta"], eps=first["cfg"]["eps"], real_steps_per_bench_step=1)
    if name == "dambreak":
        cfg.update(dt="0.25h/sqrt(2 g H)")
    return d, cfg


def with_shifting(d, wcfg):
    """Particle shifting after every real step (Sec. 3.5) in every instance's
    parameters, for both arms."""
    for x in (d if isinstance(d, list) else [d]):
        x["cfg"] = dict(x["cfg"], shifting=1)
    wcfg["shifting"] = "on (Eqs. shift-deltar, shift-correct, after every real step)"


def with_steady(d, wcfg, iters):
    """Steady-state mode (Sec. 2.3, Eq. mom-steady) with a fixed number of
    pseudo-iterations per solve, in every instance, for both arms."""
    for x in (d if isinstance(d, list) else [d]):
        # the particles stay where they are, so there is nothing to shift
        x["cfg"] = dict(x["cfg"], steady=1, fixed_iters=iters, shifting=0)
    wcfg["steady"] = f"on: one pseudo-time solve of {iters} iterations per step, particles fixed"
    wcfg.pop("shifting", None)


def with_moving(d, wcfg, moving):
    """Particles moved in pseudo-time (Algorithm 1) in every instance, for both
    arms: 1 over the lists of r^0, 2 with neighbours updated every pass (the two
    advected variants that Sec. 4.1 times against the frozen scheme)."""
    for x in (d if isinstance(d, list) else [d]):
        x["cfg"] = dict(x["cfg"], moving=moving)
    wcfg["moving"] = {1: "advected in pseudo-time, lists of r^0 (Algorithm 1)",
                      2: "advected in pseudo-time, neighbours updated every pass (Algorithm 1)"}[moving]


class Job:
    """One context running a workload: a single instance or a batch."""

    def __init__(self, dt, work, precision, stream=None, graph=2, kern=None):
        kern = dict(kern or {})
        # list skin in smoothing lengths -> each instance's own length
        skin_h = kern.pop("list_skin_h", 0.0)
        cfg_of = lambda d: dict(d["cfg"], list_skin=skin_h * d["cfg"]["h"]) if skin_h > 0 else d["cfg"]
        self.dt = dt
        self.batch = isinstance(work, list)
        if self.batch:
            self.sim = dt.Batch([cfg_of(d) for d in work], precision=precision, stream=stream, graph=graph, **kern)
            self.sim.set_state(work)
            self.nfs = [d["nf"] for d in work]
        else:
            self.sim = dt.Simulation(cfg_of(work), precision=precision, stream=stream, graph=graph, **kern)
            nf = work["nf"]
            walls = None if work["vw"] is None else (work["x"][nf:], work["vw"])
            self.sim.set_state(work["x"][:nf], work["v"], work["p"], work["v_prev"], walls=walls)
            self.nfs = [nf]
        self.ctx = self.sim.ctx

    def step(self, n=1):
        self.sim.step(n)

    def sync(self):
        self.sim.sync()

    def particle_iterations(self, first, count):
        """Per real step: sum over instances of fluid particles x iterations."""
        tot = np.zeros(count)
        for i, nf in enumerate(self.nfs):
            st = self.sim.stats(i, first, count) if self.batch else self.sim.stats(first, count)
            tot += nf * np.array([s["iters"] for s in st], dtype=float)
        return tot

    def forms(self, first, count):
        """Per real step: the pair-term form its loop ran (1 cache, 2 recomputed)."""
        st = self.sim.stats(0, first, count) if self.batch else self.sim.stats(first, count)
        return [s["form"] for s in st]

    def iterations(self, first, count):
        its = []
        for i in range(len(self.nfs)):
            st = self.sim.stats(i, first, count) if self.batch else self.sim.stats(first, count)
            its.append([s["iters"] for s in st])
        return its

    def velocities(self):
        if self.batch:
            return np.concatenate(self.sim.field(self.dt.FIELD_VEL))
        return self.sim.v

    def close(self):
        self.sim.close()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch", choices=["batch", "tgv2d", "tgv3d", "cavity", "dambreak"])
    ap.add_argument("--n-side", type=int, default=0,
                    help="particles per side, or instances for batch (0: the workload's default)")
    ap.add_argument("--re", type=float, default=0.0, help="Reynolds number (0: the workload's default)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison leg")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle run (no cpu_baseline and no L-inf against the oracle)")
    ap.add_argument("--trace", type=int, default=0,
                    help="after the timed run, rerun the same steps untimed and record the kinetic energy every "
                         "TRACE steps and the iterations of every step (FP32C)")
    ap.add_argument("--peaks", action="store_true", help="only measure the FP32 and FP64 FMA peaks and print them")
    ap.add_argument("--graph", type=int, default=2, help="2: step graph with the persistent loop kernel; "
                    "1: step graph with a while node; 0: plain launches (per-kernel profiling)")
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="lanes per particle of the iterate kernel (0: autotuned)")
    ap.add_argument("--stages", type=int, default=0, help="staging depth with --lanes 1 (0: autotuned or 3)")
    ap.add_argument("--form", type=int, default=0, choices=[0, 1, 2],
                    help="pair terms of the loop: 1 from the pair-coefficient cache, 2 recomputed every "
                         "pseudo-iteration from the lists (no cache), 0 chosen by the library")
    ap.add_argument("--list-skin", type=float, default=0.05,
                    help="> 0: the r^0 lists, built with this skin (in smoothing lengths), also serve the next "
                         "step's pass at r^n (one list build per step where the motion allows, on the device); "
                         "0: two builds per step. Applies where the library allows it (graph 2, no walls, no "
                         "shifting, no steady mode, frozen particles)")
    ap.add_argument("--cell-scale", type=float, default=0.0,
                    help="binning cell side in list cutoffs (0: the smallest cells the stencil allows)")
    ap.add_argument("--shifting", action="store_true", help="particle shifting after every real step (both arms)")
    ap.add_argument("--moving", type=int, default=0, choices=[0, 1, 2],
                    help="particles moved in pseudo-time (Algorithm 1; both arms): 1 lists of r^0, "
                         "2 neighbours updated every pass; 0 frozen")
    ap.add_argument("--steady", type=int, default=0,
                    help="steady-state mode with this many pseudo-iterations per solve (both arms; 0: off)")
    return ap.parse_args()


def whole_job_rate(work_rank: float, t_rank: float, world: int, device=None):
    """Whole-job throughput of replicas, one per rank: the work of all ranks
    (summed) over the slowest rank's time (max over ranks). Returns (rate,
    slowest time). Needs an initialised process group when world > 1."""
    if world == 1:
        return work_rank / t_rank, t_rank
    import torch
    import torch.distributed as tdist
    w = torch.tensor([work_rank], dtype=torch.float64, device=device)
    t = torch.tensor([t_rank], dtype=torch.float64, device=device)
    tdist.all_reduce(w, op=tdist.ReduceOp.SUM)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(w.item()) / float(t.item()), float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region,
    written to a temporary file that is removed afterwards."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.idx = gpu_index
        self.period = period_ms
        self.proc = None
        self.path = None
        self.rows = []

    def __enter__(self):
        import tempfile
        try:
            fd, self.path = tempfile.mkstemp(prefix="dtsph_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    self.rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        if self.path:
            try:
                os.remove(self.path)
            except OSError:
                pass

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "period_ms": self.period}


# ----------------------------------------------------------------- our arm

def run_gpu_path(dt, torch, d, precision, steps, warmup, flush, graph=2, kern=None):
    """Times `steps` real steps after `warmup`; L2 flushed before each step.
    Returns (particle-iterations/s, ms per step, iterations, launches, job,
    (per-step particle-iterations, per-step pseudo-time loop ms, per-step
    pair-term form, per-instance iterations of those steps) of the last timed
    steps, at most 256)."""
    stream = torch.cuda.Stream()
    job = Job(dt, d, precision, stream=stream, graph=graph, kern=kern)
    job.step(warmup)
    job.sync()
    l0 = dt.dtsph_kernel_launches(job.ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()                 # > L2: every step starts from a cold L2
            ev[k][0].record(stream)
            job.step(1)
            ev[k][1].record(stream)
    stream.synchronize()
    job.sync()
    ms = [a.elapsed_time(b) for a, b in ev]
    work = job.particle_iterations(warmup, steps)
    iters = job.iterations(warmup, steps)
    launches = dt.dtsph_kernel_launches(job.ctx) - l0
    rate = float(work.sum()) / (sum(ms) * 1e-3)
    nl = min(steps, 256)
    loop_ms = dt.dtsph_loop_times(job.ctx, dt.dtsph_step_count(job.ctx) - nl, nl)
    forms = job.forms(dt.dtsph_step_count(job.ctx) - nl, nl)
    its_last = job.iterations(dt.dtsph_step_count(job.ctx) - nl, nl)
    return rate, sum(ms) / steps, iters, launches, job, (work[steps - nl:], loop_ms, forms, its_last)


def run_e2e(dt, torch, d, precision, steps, graph=2, kern=None):
    """End to end through the C ABI with host arrays: per step the state goes
    host -> device, one real step runs, the state comes back device -> host."""
    job = Job(dt, d, precision, graph=graph, kern=kern)   # allocation and graph build outside the timed region
    job.step(1)
    job.sync()
    ctx, dim = job.ctx, (d[0] if job.batch else d)["cfg"]["dim"]
    NF = int(sum(job.nfs))
    # the state lives in pinned host buffers, read into and sent from in place
    pinned = lambda *shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    x, v, p, vp = pinned(NF, dim), pinned(NF, dim), pinned(NF), pinned(NF, dim)
    x, v, p, vp = dt.dtsph_read_state(ctx, NF, dim, out=(x, v, p, vp))
    work = 0.0
    t = 0.0
    torch.cuda.synchronize()
    for _ in range(steps):
        t0 = time.perf_counter()
        if job.batch:
            dt.dtsph_batch_set_particles(ctx, job.nfs, x, v, p, vp)
        else:
            dt.dtsph_set_particles(ctx, x, v, p, vp)
        dt.dtsph_step(ctx, 1)
        x, v, p, vp = dt.dtsph_read_state(ctx, NF, dim, out=(x, v, p, vp))
        t += time.perf_counter() - t0
        # (the step's iteration counts, read outside the timed span: bookkeeping
        # of this measurement, not part of a step)
        work += float(job.particle_iterations(0, 1).sum())
    h2d = NF * (3 * dim + 1) * 8
    d2h = NF * (3 * dim + 1) * 8
    job.close()
    return {"value": work / t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": 1e3 * t / steps, "host_buffers": "pinned, sent and read in place",
            "timing": "host clock around set_particles + step + read_state of each step (the read of the "
                      "step's statistics for the metric's count stays outside)"}


def run_trace(dt, d, steps, every, graph=2, kern=None):
    """The same steps again, untimed (FP32C): the kinetic energy (1/2) sum m |V|^2
    of all fluid particles every `every` steps (t = step x dt of the first
    instance), the mean pseudo-iterations per step over each such block of
    steps, and the stop reasons of all steps."""
    job = Job(dt, d, dt.DTSPH_FP32C, graph=graph, kern=kern)
    insts = d if isinstance(d, list) else [d]
    m = np.concatenate([np.full(x["nf"], x["cfg"]["m"]) for x in insts])
    dt0 = insts[0]["cfg"]["dt"]
    ke = []
    done = 0
    while done < steps:
        k = min(every, steps - done)
        job.step(k)
        done += k
        v = job.velocities()
        ke.append([round(done * dt0, 6), float(0.5 * np.sum(m[:, None] * v * v))])
    job.sync()
    its = np.array(job.iterations(0, steps)).max(0)
    reasons = []
    for i in range(len(insts)):
        st = job.sim.stats(i, 0, steps) if job.batch else job.sim.stats(0, steps)
        reasons += [s["reason"] for s in st]
    job.close()
    blocks = [float(np.mean(its[b:b + every])) for b in range(0, steps, every)]
    names = {0: "converged", 1: "stagnated", 2: "iteration cap", 3: "non-finite", 4: "fixed count"}
    return {"steps": steps, "every": every, "kinetic_energy": ke, "iters_per_step_mean_by_block": blocks,
            "iters_total": int(its.sum()),
            "stop_reasons": {names[r]: int(c) for r, c in zip(*np.unique(reasons, return_counts=True))}}


def oracle_states(d, **over):
    import oracle
    insts = d if isinstance(d, list) else [d]
    return [oracle.State(x["cfg"], x["x"], x["v"], x["p"], x["v_prev"], vw=x["vw"], nf=x["nf"], **over) for x in insts]


def oracle_run(d, nsteps, label):
    """The FP64 oracle as it stands on the host cores: `nsteps` real steps of
    every instance of the workload (instance by instance), timed. Returns the
    final velocities (instances concatenated), the iterations of every step of
    every instance, and the cpu_baseline record of the run."""
    import oracle
    oracle.build()
    states = oracle_states(d)
    t0 = time.perf_counter()
    work = 0.0
    iters = []
    for st in states:
        recs = st.step(nsteps)
        iters.append([r["iters"] for r in recs])
        work += st.nf * sum(r["iters"] for r in recs)
    t = time.perf_counter() - t0
    v = np.concatenate([st.v for st in states])
    tot_it = int(sum(map(sum, iters)))
    rec = {"value": work / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"the first {nsteps} real steps of every instance of the same {label} run ({tot_it} "
                     f"pseudo-iterations, {t:.1f} s wall): the run the L-inf errors compare against"}
    return v, iters, rec


def linf_rel(v, ref):
    return float(np.max(np.abs(v - ref)) / np.max(np.abs(ref)))


# Algorithmic bytes of one pseudo-iteration in the pair-cache form: per fluid
# particle its own state (V and p read and written, the BDF2 source read), per
# cached pair the neighbour index, gradW and F_ij, by path and dimension.
STATE_BYTES = {(2, True): 52.0, (3, True): 72.0, (2, False): 88.0, (3, False): 120.0}
PAIR_BYTES = {(2, True): 16.0, (3, True): 20.0, (2, False): 28.0, (3, False): 36.0}
# Without the cache: the same state bytes plus the particle's position at r^0
# (a 16-byte cell offset on the compensated path, dim doubles in FP64), and per
# listed pair its 4-byte list entry.
POS_BYTES = {(2, True): 16.0, (3, True): 16.0, (2, False): 16.0, (3, False): 24.0}
LIST_BYTES = 4.0


def loop_bytes_per_particle_iteration(dims, fp32c, form, pairs_per_particle):
    """Algorithmic bytes of one particle-iteration of the loop in either form."""
    if form == 2:
        return STATE_BYTES[(dims, fp32c)] + POS_BYTES[(dims, fp32c)] + LIST_BYTES * pairs_per_particle
    return STATE_BYTES[(dims, fp32c)] + PAIR_BYTES[(dims, fp32c)] * pairs_per_particle


def loop_launch_bytes_split(dims, fp32c, form, pairs_per_particle, nfs, iters, kstar):
    """Algorithmic bytes of one step's loop, (iterations with the cache,
    iterations without it): every instance's iterations in the form the step
    ran; a step that switched (form 3) ran its first floor(kstar) iterations
    without the cache and the rest with it."""
    a = loop_bytes_per_particle_iteration(dims, fp32c, 2, pairs_per_particle)
    b = loop_bytes_per_particle_iteration(dims, fp32c, 1, pairs_per_particle)
    m = int(kstar) if 1.0 <= kstar < 1e6 else 0
    cached = uncached = 0.0
    for nf, k in zip(nfs, iters):
        if form == 1:
            cached += nf * k * b
        elif form == 2:
            uncached += nf * k * a
        else:
            uncached += nf * min(k, m) * a
            cached += nf * max(k - m, 0) * b
    return cached, uncached


def loop_launch_bytes(dims, fp32c, form, pairs_per_particle, nfs, iters, kstar):
    """Algorithmic bytes of one step's loop (both parts)."""
    return sum(loop_launch_bytes_split(dims, fp32c, form, pairs_per_particle, nfs, iters, kstar))


def fp64_flops(dim):
    """FP64 flops (FMA = 2) of the FP64 pseudo-iteration, counted from the pair
    terms (EDAC on, no artificial viscosity): per cached pair the divergence
    and EDAC terms of dp/dtau and the pressure and viscous terms of F,
    8 dim + 9; per fluid particle the BDF2 pseudo-acceleration, the update and
    the residual terms, 8 dim + 3."""
    return 8.0 * dim + 3.0, 8.0 * dim + 9.0


def measure_peaks(dt):
    return {"fp32_fma_tflops": dt.dtsph_fma_peak(dt.DTSPH_FP32C) / 1e12,
            "fp64_fma_tflops": dt.dtsph_fma_peak(dt.DTSPH_FP64) / 1e12,
            "how": "dtsph_fma_peak: 8 blocks of 256 threads per SM, 8 independent FMA chains per thread, "
                   "best of 3 launches of ~50 ms, CUDA events"}


def main_ours(args):
    import torch
    import torch.distributed as tdist

    import paper_1904_00861_gb300 as dt
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_1904_00861_gb300 import build as b
    b.build()
    if args.peaks:
        print(json.dumps(measure_peaks(dt)))
        return
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    d, wcfg = make_workload(args.workload, args.n_side, args.re)
    if args.shifting:
        with_shifting(d, wcfg)
    if args.steady:
        with_steady(d, wcfg, args.steady)
    if args.moving:
        with_moving(d, wcfg, args.moving)
    # list reuse where the library supports it
    reuse_ok = (args.graph == 2 and not args.moving and not args.steady and not args.shifting and
                all(x["vw"] is None for x in (d if isinstance(d, list) else [d])))
    kern = dict(lanes=args.lanes, stages=args.stages, form=args.form, cell_scale=args.cell_scale,
                list_skin_h=args.list_skin if reuse_ok else 0.0)
    # batches without walls run the decoupled loop kernel (the library's rule)
    decoupled = (args.graph == 2 and isinstance(d, list) and 1 < len(d) <= 1024 and not args.moving
                 and all(x["vw"] is None for x in d) and os.environ.get("DTSPH_LOCKSTEP_LOOP", "0") in ("", "0"))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        rate32, ms32, it32, launches, sim32, loop32 = run_gpu_path(dt, torch, d, dt.DTSPH_FP32C, args.steps,
                                                                   args.warmup, flush, args.graph, kern)
    torch.cuda.synchronize()
    # whole-job throughput: every rank ran its replica of the workload
    t_rank = ms32 * args.steps * 1e-3
    value, _ = whole_job_rate(rate32 * t_rank, t_rank, world, device="cuda")
    lanes32, tune32 = dt.dtsph_tuning(sim32.ctx)
    stages32, cand32 = dt.dtsph_tuning_candidates(sim32.ctx)
    ms_it, bytes_it, npairs = dt.dtsph_probe_iterate(sim32.ctx, 50)
    v32 = sim32.velocities()
    dims = wcfg["dims"]
    nf_tot = float(sum(sim32.nfs))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (burst copy)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    fma = measure_peaks(dt)

    fp64 = None
    v64 = None
    if not args.no_fp64:
        rate64, ms64, it64, _, sim64, loop64 = run_gpu_path(dt, torch, d, dt.DTSPH_FP64, args.steps, args.warmup,
                                                            flush, args.graph, kern)
        v64 = sim64.velocities()
        ms_it64, bytes_it64, npairs64 = dt.dtsph_probe_iterate(sim64.ctx, 20)
        lanes64, _ = dt.dtsph_tuning(sim64.ctx)
        # the FP64 loop is bound by the FP64 pipe: algorithmic FP64 flops of the
        # timed loops over their device time, against the measured FP64 FMA peak
        f_part, f_pair = fp64_flops(dims)
        w64, lms64, _, _ = loop64
        flops64 = float(np.sum(w64)) * (f_part + f_pair * npairs64 / nf_tot)
        ach64 = flops64 / (sum(lms64) * 1e-3) / 1e12
        fp64 = {"value": rate64 * world, "ms_per_step": ms64, "iters_per_step_mean": float(np.mean(it64)),
                "iterate_kernel_ms": ms_it64, "speedup_fp32c_over_fp64": value / (rate64 * world),
                "roofline": {"bound": "alu", "pipe": "fp64", "achieved": ach64, "peak": fma["fp64_fma_tflops"],
                             "unit": "TFLOP/s", "frac": ach64 / fma["fp64_fma_tflops"],
                             "kernel": f"{'k_loop_async' if decoupled else 'k_loop'}<{dims},FP64,lanes={lanes64}>",
                             "flops_per_launch": flops64 / len(lms64), "launch_ms": sum(lms64) / len(lms64),
                             "flops_counted": f"{f_part:.0f} per particle-iteration + {f_pair:.0f} per pair-iteration "
                                              f"(FMA = 2; the pair terms as the cached form evaluates them, "
                                              f"whichever form ran), {npairs64 / nf_tot:.2f} pairs per particle",
                             "peak_source": "dtsph_fma_peak(FP64), measured in this run"}}
        sim64.close()
    # the dominant kernel of the timed steps is the pseudo-time loop: its
    # algorithmic bytes per step are the state and cache-entry bytes of one
    # pair pass per particle-iteration of the step
    loop_work, loop_ms, loop_forms, loop_its = loop32
    ppp = npairs / nf_tot
    form_rec = dt.dtsph_form_stats(sim32.ctx)
    split_by_launch = [loop_launch_bytes_split(dims, True, f, ppp, sim32.nfs, [its[k] for its in loop_its],
                                               form_rec["kstar"]) for k, f in enumerate(loop_forms)]
    bytes_by_launch = [c + u for c, u in split_by_launch]
    loop_bytes = float(sum(bytes_by_launch))
    achieved = loop_bytes / (sum(loop_ms) * 1e-3) / 1e9
    probe_bytes = STATE_BYTES[(dims, True)] * nf_tot + PAIR_BYTES[(dims, True)] * npairs
    achieved_probe = probe_bytes / (ms_it * 1e-3) / 1e9
    loop_kernel = {2: f"k_loop<{dims},FP32C,lanes={lanes32}> (persistent loop, one launch per step)",
                   1: f"k_iterate<{dims},FP32C,lanes={lanes32}> in the while node (one launch per iteration)",
                   0: f"k_iterate<{dims},FP32C,lanes={lanes32}> (plain launches)"}[args.graph]
    if decoupled:
        loop_kernel = (f"k_loop_async<{dims},FP32C,lanes={lanes32}> (decoupled batch loop, persistent, "
                       f"one launch per step)")
    probe_kernel = f"k_iterate<{dims},FP32C,lanes={lanes32}>"
    if args.moving:
        probe_kernel = f"k_move_walls + k_move_iter<{dims},FP32C> (one lane per particle)"
        loop_kernel = probe_kernel + (" (plain launches)" if args.graph == 0 else
                                      " in the while node (one launch each per iteration)")
    traffic, traffic_src, traffic_cap = None, None, None
    # a switched step (form 3) counts its iterations with and without the cache
    # at the two forms' captured ratios
    used = sorted({g for f in loop_forms for g in ((1, 2) if f == 3 else (f,))})
    keys = [(wcfg["workload"], dims, lanes32, stages32 if lanes32 == 1 else 0, f) for f in used]
    if (args.graph == 2 and not args.moving and not args.steady and not args.shifting
            and all(k in NCU_TRAFFIC for k in keys)):
        ratio = {k[-1]: NCU_TRAFFIC[k][0] / NCU_TRAFFIC[k][1] for k in keys}
        traffic = sum(ratio.get(1, 0.0) * c + ratio.get(2, 0.0) * u for c, u in split_by_launch) / len(split_by_launch)
        traffic_src = "; ".join(f"{NCU_TRAFFIC[k][2]} (form {k[-1]}): the captured launch moved {ratio[k[-1]]:.3f} "
                                f"DRAM bytes per algorithmic byte" for k in sorted(set(keys)))
        traffic_src += ("; each of this line's launches times its own algorithmic bytes in each form "
                        "(a switched step: its iterations without and with the cache), averaged")
        traffic_cap = {f"form{k[-1]}": {"dram_bytes": NCU_TRAFFIC[k][0], "algorithmic_bytes": NCU_TRAFFIC[k][1],
                                        "ratio": ratio[k[-1]]} for k in sorted(set(keys))}
    # the launches that ran without the cache, against the FP32 pipe
    no_cache = None
    nc_idx = [k for k, f in enumerate(loop_forms) if f == 2]
    if nc_idx and dims in NCU_FLOPS_NO_CACHE and not args.moving:
        fpp, fwl, fsrc = NCU_FLOPS_NO_CACHE[dims]
        pit = sum(float(loop_work[k]) for k in nc_idx)
        secs = sum(loop_ms[k] for k in nc_idx) * 1e-3
        tf = fpp * ppp * pit / secs / 1e12
        no_cache = {"bound": "alu", "pipe": "fp32", "achieved": tf, "peak": fma["fp32_fma_tflops"],
                    "unit": "TFLOP/s", "frac": tf / fma["fp32_fma_tflops"], "launches": len(nc_idx),
                    "flops_counted": f"{fpp:.1f} FP32 flops per pair-iteration (fadd + fmul + 2 ffma per thread, "
                                     f"measured on {fwl}: {fsrc}), {ppp:.2f} pairs per particle",
                    "peak_source": "dtsph_fma_peak(FP32), measured in this run"}
    e2e = run_e2e(dt, torch, d, dt.DTSPH_FP32C, max(3, min(args.steps, 30)), args.graph, kern)
    trace = run_trace(dt, d, args.warmup + args.steps, args.trace, args.graph, kern) if args.trace else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+kahan/f64", "data": "synthetic (seeded lattice, closed-form initial field)",
        "config": dict(wcfg, precision="FP32C", parallelism=f"replicas{world}",
                       l2="flushed before every step (256 MB write)"),
        "linf_vs_oracle": None,
        "linf_fp32c_vs_fp64_gpu": None if v64 is None else linf_rel(v32, v64),
        "iters_per_step_mean": float(np.mean(it32)),
        "fp64": fp64,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic, "traffic_source": traffic_src, "traffic_captured_launch": traffic_cap,
                     "kernel": loop_kernel,
                     "bytes_per_launch": loop_bytes / len(loop_ms), "launch_ms": sum(loop_ms) / len(loop_ms),
                     "bytes_by_launch": bytes_by_launch,
                     "bytes_counted": f"cached form: {STATE_BYTES[(dims, True)]:.0f} B per particle-iteration + "
                                      f"{PAIR_BYTES[(dims, True)]:.0f} B per pair-iteration; uncached form: "
                                      f"{STATE_BYTES[(dims, True)] + POS_BYTES[(dims, True)]:.0f} B per "
                                      f"particle-iteration + {LIST_BYTES:.0f} B per pair-iteration; "
                                      f"{npairs / nf_tot:.2f} pairs per particle; each launch counted in the form "
                                      f"it ran (form 3: the first floor(kstar) iterations uncached, the rest cached)",
                     "forms_by_launch": loop_forms,
                     "timing": f"CUDA events around the loop of each of the last {len(loop_ms)} timed steps",
                     "peak_source": hbm_src},
        "roofline_no_cache": no_cache,
        "iterate_probe": {"kernel": probe_kernel, "achieved": achieved_probe,
                          "frac": achieved_probe / hbm, "bytes_per_launch": probe_bytes, "launch_ms": ms_it,
                          "pairs": npairs, "timing": "50 launches after the timed region, every instance active, "
                                                     "CUDA events"},
        "fma_peaks": fma,
        "form": dict(form_rec, requested=args.form,
                     note="kstar = cache pass / (uncached - cached iteration); with form 0 a step starts "
                          "uncached when the previous step took at most kstar iterations and switches to the "
                          "cache after floor(kstar) iterations (form 3)"),
        "autotune": {"lanes_per_particle": lanes32, "stages": stages32, "ms_by_lanes": tune32,
                     "cell_scale": args.cell_scale or 1.0,
                     "list_skin_h": kern["list_skin_h"],
                     "candidates": [{"lanes": L, "stages": S, "ms": m} for L, S, m in cand32]},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if trace is not None:
        out["trace"] = trace
    sim32.close()
    if rank == 0 and not args.no_cpu_baseline:
        vo, it_o, rec = oracle_run(d, args.warmup + args.steps, wcfg["workload"])
        out["cpu_baseline"] = rec
        # the GPU paths' iterations of the timed steps against the oracle's
        it_o_timed = [its[args.warmup:] for its in it_o]
        out["linf_vs_oracle"] = {"fp32c": linf_rel(v32, vo), "fp64": None if v64 is None else linf_rel(v64, vo),
                                 "after_real_steps": args.warmup + args.steps,
                                 "fp32c_same_iterations_as_oracle": bool(np.array_equal(np.array(it32),
                                                                                         np.array(it_o_timed))),
                                 "fp64_same_iterations_as_oracle": None if args.no_fp64 else
                                 bool(np.array_equal(np.array(it64), np.array(it_o_timed))),
                                 "measure": "max |V_gpu - V_oracle| / max |V_oracle| over every fluid particle"}
    if world > 1:
        tdist.barrier()
        tdist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# ------------------------------------------------------------ reference arm

def main_reference(args):
    """The FP64 oracle timed on the host cores, on this arm's workload and
    metric; every step is one real step of the same run."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    d, wcfg = make_workload(args.workload, args.n_side, args.re)
    if args.shifting:
        with_shifting(d, wcfg)
    if args.steady:
        with_steady(d, wcfg, args.steady)
    if args.moving:
        with_moving(d, wcfg, args.moving)
    states = oracle_states(d)
    for st in states:
        st.step(args.warmup)
    t0 = time.perf_counter()
    work = 0.0
    iters = 0
    for _ in range(args.steps):
        for st in states:
            it = st.step(1)[0]["iters"]
            iters += it
            work += st.nf * it
    t = time.perf_counter() - t0
    value = work / t
    cores = oracle.num_threads()
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded lattice, closed-form initial field)",
        "config": dict(wcfg, precision="FP64 CPU oracle", parallelism=f"openmp{cores}"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} real steps after {args.warmup} warm-up steps ({iters} "
                                   f"pseudo-iterations)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
