"""Failure detection and input checks on the GPU, without faulting it: each
failure is made on the host (bad input, an allocation cap, a barrier give-up
time of zero) and must come back as a status code, with the context still
usable afterwards.

- Positions outside [lo, hi) on a periodic axis are brought in by whole box
  lengths, as the oracle does; a non-finite position is refused.
- A non-finite pressure stops the first pseudo-time loop with reason 3
  (non-finite residual), as in the oracle.
- DTSPH_TEST_ALLOC_LIMIT below the context's needs gives DTSPH_E_OOM.
- DTSPH_TEST_BARRIER_WAIT_NS = 0 makes the persistent loop's grid barrier give
  up at once: the step ends and dtsph_sync reports DTSPH_E_TIMEOUT.
"""
import numpy as np
import pytest

import oracle
import paper_1904_00861_gb300 as dt
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_00861_gb300 import build
    build.build()
    oracle.build()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


def sim_of(d, precision=dt.DTSPH_FP64, **over):
    sim = dt.Simulation(d["cfg"], precision=precision, **over)
    nf = d["nf"]
    walls = None if d["vw"] is None else (d["x"][nf:], d["vw"])
    sim.set_state(d["x"][:nf], d["v"], d["p"], d["v_prev"], walls=walls)
    return sim


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_periodic_inputs_outside_the_box_are_brought_in(prec):
    """Every other particle given one box length to the right, every third
    three box lengths below: the GPU and the oracle bring them in the same way
    (FP64 within 1e-10, FP32C within 1e-4 of the oracle after two steps), and
    the run equals the one from the unshifted input up to the rounding of the
    shift."""
    d = synth.tgv2d(30, jitter=0.1, seed=21)
    x = d["x"].copy()
    x[::2, 0] += 1.0
    x[::3, 1] -= 3.0
    shifted = dict(d, x=x)
    orc = oracle.State(d["cfg"], x, d["v"], d["p"], d["v_prev"])
    orc.step(2)
    sim = sim_of(shifted, prec)
    sim.step(2)
    sim.sync()
    tol = 1e-10 if prec == dt.DTSPH_FP64 else 1e-4
    assert rel(sim.v, orc.v) < tol and rel(sim.p, orc.p) < tol
    assert np.all(sim.x >= 0.0) and np.all(sim.x < 1.0)
    ref = sim_of(d, prec)
    ref.step(2)
    assert rel(sim.v, ref.v) < (1e-9 if prec == dt.DTSPH_FP64 else 1e-5)
    sim.close()
    ref.close()


def test_non_finite_position_is_refused_and_the_context_stays_usable():
    import torch
    d = synth.tgv2d(20, seed=3)
    sim = dt.Simulation(d["cfg"], precision=dt.DTSPH_FP32C, lanes=4)   # no tuning run on set
    bad = d["x"].copy()
    bad[5, 1] = np.nan
    with pytest.raises(dt.DtsphError) as e:
        sim.set_state(bad, d["v"], d["p"], d["v_prev"])
    assert e.value.code == dt.DTSPH_E_ARG
    # the device-pointer path reports it at the next sync
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    bx, v, p, vp = dev(bad), dev(d["v"]), dev(d["p"]), dev(d["v_prev"])
    dt.dtsph_set_particles_device(sim.ctx, d["nf"], bx, v, p, vp)
    with pytest.raises(dt.DtsphError) as e:
        dt.dtsph_sync(sim.ctx)
    assert e.value.code == dt.DTSPH_E_ARG
    torch.cuda.synchronize()
    sim.set_state(d["x"], d["v"], d["p"], d["v_prev"])
    sim.step(1)
    sim.sync()
    assert sim.stats()[0]["reason"] in (0, 1)
    sim.close()


@pytest.mark.parametrize("graph", [0, 1, 2])
@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_nan_pressure_stops_with_reason_3_like_the_oracle(prec, graph):
    d = synth.tgv2d(24, seed=5)
    p = d["p"].copy()
    p[7] = np.nan
    bad = dict(d, p=p)
    orc = oracle.State(d["cfg"], d["x"], d["v"], p, d["v_prev"])
    rec = orc.step(1)[0]
    sim = sim_of(bad, prec, graph=graph)
    sim.step(1)
    sim.sync()
    st = sim.stats()[0]
    assert rec["reason"] == 3 and st["reason"] == 3
    assert st["iters"] == rec["iters"] == 1
    sim.close()


def test_allocation_cap_gives_oom(monkeypatch):
    d = synth.tgv2d(40, seed=2)
    sim = dt.Simulation(d["cfg"], precision=dt.DTSPH_FP32C)
    monkeypatch.setenv("DTSPH_TEST_ALLOC_LIMIT", "65536")
    with pytest.raises(dt.DtsphError) as e:
        sim.set_state(d["x"], d["v"], d["p"], d["v_prev"])
    assert e.value.code == dt.DTSPH_E_OOM
    monkeypatch.delenv("DTSPH_TEST_ALLOC_LIMIT")
    sim.set_state(d["x"], d["v"], d["p"], d["v_prev"])
    sim.step(1)
    sim.sync()
    sim.close()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_grid_barrier_give_up_is_reported(monkeypatch, prec):
    """A give-up time of zero: the first block to reach a grid barrier stops
    waiting at once, so the step's persistent loop ends early; dtsph_sync says
    DTSPH_E_TIMEOUT, and a new context without the setting runs normally.
    (form = 1: the automatic form would time the loop at dtsph_set_particles,
    where the give-up would already be reported.)"""
    d = synth.tgv2d(100, seed=4)
    monkeypatch.setenv("DTSPH_TEST_BARRIER_WAIT_NS", "0")
    sim = sim_of(d, prec, graph=2, lanes=1, form=1)
    sim.step(1)
    with pytest.raises(dt.DtsphError) as e:
        sim.sync()
    assert e.value.code == dt.DTSPH_E_TIMEOUT
    sim.close()
    monkeypatch.delenv("DTSPH_TEST_BARRIER_WAIT_NS")
    ok = sim_of(d, prec, graph=2, lanes=1)
    ok.step(1)
    ok.sync()
    assert ok.stats()[0]["reason"] in (0, 1)
    ok.close()
