"""Benchmark: particle-pseudo-iterations per second of the frozen EDAC-DTSPH
hot path on one GB300 (or N independent replicas, one per GPU).

Workload (default): 2D Taylor-Green vortex, periodic unit square, 200 x 200 =
40,000 particles on a lattice jittered by +-0.1 dx (seed 1904), Re = 100, quintic
kernel h = dx, beta = 10, dt = 0.25 h, eps = 1e-3. One "step" is one real time
step: neighbour rebuild, state-n rates and predictor, the pseudo-time loop until
the convergence test of the paper holds, and the position update. The metric
counts fluid particles times pseudo-iterations actually taken.

The FP32-compensated path gives `value`; the plain FP64 GPU path is timed in the
same run on the same steps ("fp64" key), and the L-inf relative velocity error of
FP32C against it is reported. `e2e` times the same steps through the C ABI with
host arrays (state copied in, step, state copied out). `cpu_baseline` times the
FP64 C oracle on the host cores on a bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
WORKLOAD = dict(workload="tgv2d-200x200", particles=40000, re=100, dims=2, dt="0.25h", beta=10, eps=1e-3,
                real_steps_per_bench_step=1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-side", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--graph", type=int, default=1, help="0: plain kernel launches instead of the step graph "
                    "(used for per-kernel profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- our arm

def run_gpu_path(dt, torch, d, precision, steps, warmup, flush, graph=1):
    """Times `steps` real steps after `warmup`; L2 flushed before each step.
    Returns (particle-iterations/s, ms per step, iterations, launches, sim)."""
    stream = torch.cuda.Stream()
    sim = dt.Simulation(d["cfg"], precision=precision, stream=stream, graph=graph)
    sim.set_state(d["x"], d["v"], d["p"], d["v_prev"])
    sim.step(warmup)
    sim.sync()
    l0 = dt.dtsph_kernel_launches(sim.ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()                 # > L2: every step starts from a cold L2
            ev[k][0].record(stream)
            sim.step(1)
            ev[k][1].record(stream)
    stream.synchronize()
    sim.sync()
    ms = [a.elapsed_time(b) for a, b in ev]
    st = sim.stats(warmup, steps)
    iters = [s["iters"] for s in st]
    launches = dt.dtsph_kernel_launches(sim.ctx) - l0
    rate = sim.nf * sum(iters) / (sum(ms) * 1e-3)
    return rate, sum(ms) / steps, iters, launches, sim


def run_e2e(dt, torch, d, precision, steps):
    """End to end through the C ABI with host arrays: per step the state goes
    host -> device, one real step runs, the state comes back device -> host."""
    sim = dt.Simulation(d["cfg"], precision=precision)
    x, v, p, vp = (np.ascontiguousarray(a) for a in (d["x"], d["v"], d["p"], d["v_prev"]))
    sim.set_state(x, v, p, vp)           # allocation and graph build outside the timed region
    sim.step(1)
    sim.sync()
    x, v, p, vp = sim.x, sim.v, sim.p, sim.v_prev
    nf, dim = sim.nf, sim.dim
    iters = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        dt.dtsph_set_particles(sim.ctx, x, v, p, vp)
        dt.dtsph_step(sim.ctx, 1)
        x, v, p, vp = sim.x, sim.v, sim.p, sim.v_prev
        iters += sim.stats(0, 1)[0]["iters"]
    t = time.perf_counter() - t0
    h2d = nf * (3 * dim + 1) * 8
    d2h = nf * (3 * dim + 1) * 8
    sim.close()
    return {"value": nf * iters / t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": 1e3 * t / steps}


def cpu_baseline(d, seconds):
    """The FP64 oracle as it stands on the host cores: real steps of the same
    workload until `seconds` of wall time have passed (at least one)."""
    import oracle
    oracle.build()
    st = oracle.State(d["cfg"], d["x"], d["v"], d["p"], d["v_prev"])
    t0 = time.perf_counter()
    iters = 0
    nsteps = 0
    while True:
        iters += st.step(1)[0]["iters"]
        nsteps += 1
        if time.perf_counter() - t0 > seconds:
            break
    t = time.perf_counter() - t0
    return {"value": st.nf * iters / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {nsteps} real steps of the same 200x200 Taylor-Green run ({iters} pseudo-iterations, "
                      f"{t:.1f} s wall)"}


def main_ours(args):
    import torch
    import torch.distributed as tdist

    import paper_1904_00861_gb300 as dt
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1904_00861_gb300 import build as b
    b.build()
    d = synth.tgv2d(args.n_side)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        rate32, ms32, it32, launches, sim32 = run_gpu_path(dt, torch, d, dt.DTSPH_FP32C, args.steps, args.warmup,
                                                           flush, args.graph)
    torch.cuda.synchronize()
    # whole-job throughput: every rank ran the same workload independently
    t_rank = ms32 * args.steps
    if world > 1:
        tt = torch.tensor([t_rank], device="cuda", dtype=torch.float64)
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        t_max = float(tt.item())
    else:
        t_max = t_rank
    value = world * sim32.nf * sum(it32) / (t_max * 1e-3)
    rate64, ms64, it64, _, sim64 = run_gpu_path(dt, torch, d, dt.DTSPH_FP64, args.steps, args.warmup, flush,
                                                args.graph)
    v32, v64 = sim32.v, sim64.v
    linf = float(np.max(np.abs(v32 - v64)) / np.max(np.abs(v64)))
    lanes32, tune32 = dt.dtsph_tuning(sim32.ctx)
    ms_it, bytes_it, npairs = dt.dtsph_probe_iterate(sim32.ctx, 50)
    ms_it64, bytes_it64, _ = dt.dtsph_probe_iterate(sim64.ctx, 20)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bytes_it / (ms_it * 1e-3) / 1e9
    e2e = run_e2e(dt, torch, d, dt.DTSPH_FP32C, max(3, min(args.steps, 30)))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+kahan/f64", "data": "synthetic (seeded jittered lattice, exact TGV field)",
        "config": dict(WORKLOAD, precision="FP32C", parallelism=f"replicas{world}",
                       l2="flushed before every step (256 MB write)"),
        "linf_rel_vel_err_vs_fp64": linf,
        "iters_per_step_mean": float(np.mean(it32)),
        "fp64": {"value": rate64 * world, "ms_per_step": ms64, "iters_per_step_mean": float(np.mean(it64)),
                 "iterate_kernel_ms": ms_it64, "speedup_fp32c_over_fp64": value / (rate64 * world)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "kernel": "k_iterate<2,FP32C>", "bytes_per_launch": bytes_it,
                     "launch_ms": ms_it, "pairs": npairs, "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)"},
        "autotune": {"lanes_per_particle": lanes32, "ms_by_lanes": tune32},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    sim32.close()
    sim64.close()
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(d, args.cpu_seconds)
    if world > 1:
        tdist.barrier()
        tdist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# ------------------------------------------------------------ reference arm

def main_reference(args):
    """The FP64 oracle timed on the host cores, on this arm's workload and
    metric; every step is one real step of the 200 x 200 Taylor-Green run."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    d = synth.tgv2d(args.n_side)
    st = oracle.State(d["cfg"], d["x"], d["v"], d["p"], d["v_prev"])
    st.step(args.warmup)
    t0 = time.perf_counter()
    iters = sum(r["iters"] for r in st.step(args.steps))
    t = time.perf_counter() - t0
    value = st.nf * iters / t
    cores = oracle.num_threads()
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded jittered lattice, exact TGV field)",
        "config": dict(WORKLOAD, precision="FP64 CPU oracle", parallelism=f"openmp{cores}"),
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
