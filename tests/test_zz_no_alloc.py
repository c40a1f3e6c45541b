"""The allocation-free rate evaluation (dtsph_eval_rates_noalloc) against the
context entry point dtsph_eval_rates and against the FP64 oracle.

The entry exists for callers that cannot allocate device memory when they need
the rates (inside a stream capture they do not own, under a fixed device-memory
budget, or where an allocation could stall the host thread). It must give the
same rates as the regular entry, with the same reading of every parameter
(steady mode, free-surface wall pressure, artificial viscosity, walls), call
after call, even though every call reuses one fixed scratch array that keeps the
previous call's contents; it must take no device memory; and a neighbour list
cut at its capacity must show in the status word. This file is collected last
so that a run stopping at the first failure has run every other test first; it
also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
import paper_1904_00861_gb300 as dt
import synth

pytestmark = pytest.mark.gpu

CASES = {
    "tgv2d": lambda: synth.tgv2d(50, seed=1904),
    "cavity": lambda: synth.cavity2d(23),
    "tgv3d": lambda: synth.tgv3d(12, jitter=0.1, seed=5),
    "dambreak": lambda: synth.dambreak2d(14, jitter=0.1, seed=3),
}

# parameter variants on top of each case's own (the modes that change the rates)
MODES = {
    "plain": {},
    "steady": dict(steady=1),
    "free_surface_av": dict(free_surface=1, alpha=0.1),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_00861_gb300 import build
    build.build()


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def state(case, mode="plain"):
    d = CASES[case]()
    rng = np.random.default_rng(2)
    v = d["v"] + 0.1 * rng.normal(size=d["v"].shape)
    p = d["p"] + 0.1 * rng.normal(size=d["p"].shape)
    return dict(d, v=v, p=p, cfg=dict(d["cfg"], **MODES[mode]))


def context_rates(d, prec):
    sim = dt.Simulation(d["cfg"], precision=prec, lanes=4)
    nf = d["nf"]
    walls = None if d["vw"] is None else (d["x"][nf:], d["vw"])
    sim.set_state(d["x"][:nf], d["v"], d["p"], walls=walls)
    ap, F = sim.rates()
    sim.close()
    return ap, F


class Device:
    """The device copies of one state and the output buffers, made once."""

    def __init__(self, d):
        import torch
        self.d = d
        nf = d["nf"]
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")
        self.x, self.v, self.p = dev(d["x"][:nf]), dev(d["v"]), dev(d["p"])
        self.nw = len(d["x"]) - nf
        self.xw = dev(d["x"][nf:]) if self.nw else None
        self.vw = dev(d["vw"]) if self.nw else None
        self.ap = torch.empty(nf, dtype=torch.float64, device="cuda")
        self.F = torch.empty((nf, d["cfg"]["dim"]), dtype=torch.float64, device="cuda")
        self.status = torch.empty(1, dtype=torch.int32, device="cuda")

    def call(self, prec, **over):
        params = dt.make_params(self.d["cfg"], precision=prec, **over)
        self.ap.fill_(float("nan"))
        self.F.fill_(float("nan"))
        self.status.fill_(12345)
        dt.dtsph_eval_rates_noalloc(params, self.d["nf"], self.x, self.v, self.p, self.ap, self.F, nw=self.nw,
                                    xw=self.xw, vw=self.vw, status=self.status)

    def result(self):
        import torch
        torch.cuda.synchronize()
        return self.ap.cpu().numpy(), self.F.cpu().numpy(), int(self.status.item())


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_context_entry_and_oracle_twice(case, mode, prec):
    """Two calls in a row, with another problem in between (which leaves other
    contents in the shared scratch): both equal dtsph_eval_rates (1e-12; the
    same kernels run) and the oracle (1e-12 in FP64, 1e-4 in FP32C)."""
    d = state(case, mode)
    ap_ref, F_ref = context_rates(d, prec)
    ap_orc, F_orc, _, _ = oracle.rates(d["cfg"], d["x"], d["v"], d["p"], vw=d["vw"], nf=d["nf"])
    tol = 1e-12 if prec == dt.DTSPH_FP64 else 1e-4
    mine = Device(d)
    other = Device(state("cavity" if case != "cavity" else "tgv2d"))
    for call in range(2):
        mine.call(prec)
        ap, F, status = mine.result()
        assert status == dt.DTSPH_OK, (case, mode, call)
        assert rel(ap, ap_ref) < 1e-12, (case, mode, call)
        assert rel(F, F_ref) < 1e-12, (case, mode, call)
        assert rel(ap, ap_orc) < tol, (case, mode, call)
        assert rel(F, F_orc) < tol, (case, mode, call)
        other.call(prec)


def test_noalloc_takes_no_device_memory():
    """After a first call (which looks up the scratch address and loads the
    kernels), further calls change neither torch's allocations nor the device's
    free memory."""
    import torch
    dev = Device(state("cavity", "free_surface_av"))
    dev.call(dt.DTSPH_FP32C)
    dev.result()
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    for _ in range(3):
        dev.call(dt.DTSPH_FP32C)
    dev.result()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_reports_a_cut_list_in_its_status():
    """A neighbour capacity below the real counts: the lists are cut and the
    status word says DTSPH_E_CAPACITY; the next call with room says DTSPH_OK."""
    dev = Device(state("tgv2d"))
    dev.call(dt.DTSPH_FP64, max_neighbors=8)
    assert dev.result()[2] == dt.DTSPH_E_CAPACITY
    dev.call(dt.DTSPH_FP64)
    assert dev.result()[2] == dt.DTSPH_OK


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    d = synth.tgv2d(129)                       # 16,641 particles > 16,384
    nf = d["nf"]
    z = torch.zeros((nf, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(dt.DtsphError) as e:
        dt.dtsph_eval_rates_noalloc(dt.make_params(d["cfg"]), nf, z, z, z[:, 0].contiguous(),
                                    torch.zeros(nf, dtype=torch.float64, device="cuda"), z)
    assert e.value.code == dt.DTSPH_E_CAPACITY
