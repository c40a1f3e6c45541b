"""The allocation-free rate evaluation (dtsph_eval_rates_noalloc) against the
context entry point dtsph_eval_rates.

It exists for callers that cannot allocate device memory when they need the
rates (inside a stream capture they do not own, under a fixed device-memory
budget, or where an allocation could stall the host thread). It must give the
same rates as the regular entry, call after call, even though every call reuses
one fixed scratch array that keeps the previous call's contents. This file is
collected last so that a run stopping at the first failure has run every other
test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import paper_1904_00861_gb300 as dt
import synth

pytestmark = pytest.mark.gpu

CASES = {
    "tgv2d": lambda: synth.tgv2d(50, seed=1904),
    "cavity": lambda: synth.cavity2d(23),
    "tgv3d": lambda: synth.tgv3d(12, jitter=0.1, seed=5),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_00861_gb300 import build
    build.build()


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def state(case):
    d = CASES[case]()
    rng = np.random.default_rng(2)
    v = d["v"] + 0.1 * rng.normal(size=d["v"].shape)
    p = d["p"] + 0.1 * rng.normal(size=d["p"].shape)
    return dict(d, v=v, p=p)


def reference_rates(d, prec):
    sim = dt.Simulation(d["cfg"], precision=prec, lanes=4)
    nf = d["nf"]
    walls = None if d["vw"] is None else (d["x"][nf:], d["vw"])
    sim.set_state(d["x"][:nf], d["v"], d["p"], walls=walls)
    ap, F = sim.rates()
    sim.close()
    return ap, F


def noalloc_rates(d, prec, out_ap, out_F):
    import torch
    nf = d["nf"]
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float64), device="cuda")
    x, v, p = dev(d["x"][:nf]), dev(d["v"]), dev(d["p"])
    nw = len(d["x"]) - nf
    xw = dev(d["x"][nf:]) if nw else None
    vw = dev(d["vw"]) if nw else None
    params = dt.make_params(d["cfg"], precision=prec)
    out_ap.fill_(float("nan"))
    out_F.fill_(float("nan"))
    dt.dtsph_eval_rates_noalloc(params, nf, x, v, p, out_ap, out_F, nw=nw, xw=xw, vw=vw)
    torch.cuda.synchronize()
    return out_ap.cpu().numpy(), out_F.cpu().numpy()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_context_entry_twice(case, prec):
    import torch
    d = state(case)
    ap_ref, F_ref = reference_rates(d, prec)
    nf, dim = d["nf"], d["cfg"]["dim"]
    ap = torch.empty(nf, dtype=torch.float64, device="cuda")
    F = torch.empty((nf, dim), dtype=torch.float64, device="cuda")
    other = state("cavity" if case != "cavity" else "tgv2d")
    ap_o = torch.empty(other["nf"], dtype=torch.float64, device="cuda")
    F_o = torch.empty((other["nf"], other["cfg"]["dim"]), dtype=torch.float64, device="cuda")
    for call in range(2):
        got_ap, got_F = noalloc_rates(d, prec, ap, F)
        assert rel(got_ap, ap_ref) < 1e-12, (case, call)
        assert rel(got_F, F_ref) < 1e-12, (case, call)
        # a different problem in between leaves other contents in the shared scratch
        noalloc_rates(other, prec, ap_o, F_o)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    d = synth.tgv2d(129)                       # 16,641 particles > 16,384
    nf = d["nf"]
    z = torch.zeros((nf, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(dt.DtsphError) as e:
        dt.dtsph_eval_rates_noalloc(dt.make_params(d["cfg"]), nf, z, z, z[:, 0].contiguous(),
                                    torch.zeros(nf, dtype=torch.float64, device="cuda"), z)
    assert e.value.code == -5
