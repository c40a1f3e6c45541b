"""The multi-GPU contract of bench.py on the host: N replicas, one per rank,
whole-job throughput = work of all ranks / slowest rank's time; the reference
arm under torchrun prints one line from rank 0 and the other ranks exit 0.
World size 2 over gloo on 127.0.0.1, no GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as tdist
    sys.path.insert(0, ROOT)
    import bench
    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    # rank r did 100 (r + 1) units of work in 1 + r seconds
    rate, t_max = bench.whole_job_rate(100.0 * (rank + 1), 1.0 + rank, world)
    out[rank] = (rate, t_max)
    tdist.barrier()
    tdist.destroy_process_group()


def test_whole_job_rate_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [mp.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    # (100 + 200) units over the slowest rank's 2 s, the same on both ranks
    assert res[0] == res[1] == (150.0, 2.0)


def test_single_rank_rate_is_its_own():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(300.0, 2.0, 1) == (150.0, 2.0)


def test_reference_arm_under_torchrun_two_ranks():
    """bench.py --impl reference launched as the driver launches N > 1: exit 0,
    one JSON line (rank 0), n_gpus = 2."""
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--n-side", "16", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="2"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
