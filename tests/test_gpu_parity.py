"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.

Bars: neighbour sets bit-exact; FP64 rates and steps within 1e-10 normwise
relative (max_i |x_i - y_i| / max_i |y_i|); FP32C velocities within 1e-4 L-inf
relative (the reduced-precision bar), with the error printed.
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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def wrap_diff(a, b, box):
    d = np.asarray(a) - np.asarray(b)
    if box is not None:
        d -= box * np.round(d / box)
    return d


def make_sim(d, precision=dt.DTSPH_FP64, graph=1, **over):
    sim = dt.Simulation(d["cfg"], precision=precision, graph=graph, **over)
    nf = d["nf"]
    walls = None if d["vw"] is None else (d["x"][nf:], d["vw"])
    sim.set_state(d["x"][:nf], d["v"], d["p"], d["v_prev"], walls=walls)
    return sim


def make_oracle(d, **over):
    return oracle.State(d["cfg"], d["x"], d["v"], d["p"], d["v_prev"], vw=d["vw"], nf=d["nf"], **over)


def box_of(d):
    cfg = d["cfg"]
    dim = cfg["dim"]
    if all(cfg["periodic"][:dim]):
        return np.array(cfg["hi"][:dim]) - np.array(cfg["lo"][:dim])
    return None


# ------------------------------------------------------------- neighbours

CASES = {
    "tgv2d_jitter": lambda: synth.tgv2d(50, seed=1904),
    "tgv2d_lattice": lambda: synth.tgv2d(37, jitter=0.0),          # exact 3h ties, ragged n
    "cavity": lambda: synth.cavity2d(23),
    "tgv3d": lambda: synth.tgv3d(12, jitter=0.1, seed=5),
}


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("case", sorted(CASES))
def test_neighbour_sets_bit_exact(case, prec):
    d = CASES[case]()
    sim = make_sim(d, precision=prec)
    dt.dtsph_build_neighbors(sim.ctx)
    start, idx = oracle.neighbors(d["cfg"], d["x"])
    n = len(d["x"])
    for i in range(n):
        got = dt.dtsph_get_neighbors(sim.ctx, i)
        assert np.array_equal(got, idx[start[i]:start[i + 1]]), (case, i)
    sim.close()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("case", ["tgv2d_jitter", "cavity", "tgv3d"])
def test_wider_cells_give_the_same_sets_and_iterations(case, prec):
    """cell_scale = 1.3 bins into cells 1.3 cutoffs wide: the same neighbour sets
    as the oracle's, and over three steps the same iteration counts and, up to
    the summation order of the lists, the same velocities as the smallest cells."""
    d = CASES[case]()
    wide = make_sim(d, precision=prec, graph=2, lanes=1, cell_scale=1.3)
    dt.dtsph_build_neighbors(wide.ctx)
    start, idx = oracle.neighbors(d["cfg"], d["x"])
    for i in range(0, len(d["x"]), 7):
        assert np.array_equal(dt.dtsph_get_neighbors(wide.ctx, i), idx[start[i]:start[i + 1]]), i
    base = make_sim(d, precision=prec, graph=2, lanes=1)
    for s in (base, wide):
        s.step(3)
        s.sync()
    assert [r["iters"] for r in base.stats()] == [r["iters"] for r in wide.stats()]
    tol = 1e-12 if prec == dt.DTSPH_FP64 else 1e-5
    assert rel(wide.v, base.v) < tol
    base.close()
    wide.close()


def test_neighbour_sets_of_the_row_segment_builder():
    """At 700^2 (18,174 row segments of three 3h cells) the FP32C lists come from
    the builder that takes a row segment per warp: the sets equal the oracle's
    for sampled particles, those next to the periodic edges included."""
    d = synth.tgv2d(700, seed=7)
    sim = make_sim(d, precision=dt.DTSPH_FP32C)
    dt.dtsph_build_neighbors(sim.ctx)
    start, idx = oracle.neighbors(d["cfg"], d["x"])
    x = d["x"]
    rng = np.random.default_rng(3)
    edge = np.concatenate([np.argsort(x[:, 0])[:20], np.argsort(x[:, 0])[-20:],
                           np.argsort(x[:, 1])[:20], np.argsort(x[:, 1])[-20:]])
    for i in np.concatenate([rng.choice(len(x), 160, replace=False), edge]):
        got = dt.dtsph_get_neighbors(sim.ctx, int(i))
        assert np.array_equal(got, idx[start[i]:start[i + 1]]), i
    sim.close()


# ------------------------------------------------------------------ rates

@pytest.mark.parametrize("case", sorted(CASES))
def test_rates_fp64(case):
    d = CASES[case]()
    rng = np.random.default_rng(0)
    v = d["v"] + 0.1 * rng.normal(size=d["v"].shape)
    p = d["p"] + 0.1 * rng.normal(size=d["p"].shape)
    d = dict(d, v=v, p=p)
    sim = make_sim(d)
    ap, F = sim.rates()
    ap0, F0, _, _ = oracle.rates(d["cfg"], d["x"], v, p, vw=d["vw"], nf=d["nf"])
    assert rel(ap, ap0) < 1e-12
    assert rel(F, F0) < 1e-12
    sim.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_rates_fp32c(case):
    """FP32C rates against the FP64 oracle, normwise relative. The state is
    randomised so that no rate is zero by symmetry (a zero reference would make
    any FP32 rounding look infinitely large)."""
    d = CASES[case]()
    rng = np.random.default_rng(1)
    v = d["v"] + 0.1 * rng.normal(size=d["v"].shape)
    p = d["p"] + 0.1 * rng.normal(size=d["p"].shape)
    d = dict(d, v=v, p=p)
    sim = make_sim(d, precision=dt.DTSPH_FP32C)
    ap, F = sim.rates()
    ap0, F0, _, _ = oracle.rates(d["cfg"], d["x"], v, p, vw=d["vw"], nf=d["nf"])
    e_ap, e_F = rel(ap, ap0), rel(F, F0)
    print(f"{case}: FP32C rates L-inf rel err ap {e_ap:.2e} F {e_F:.2e}")
    assert e_ap < 1e-4 and e_F < 1e-4
    sim.close()


# ------------------------------------------------------------------ steps

def run_pair(d, nsteps, precision=dt.DTSPH_FP64, graph=1, **over):
    sim = make_sim(d, precision=precision, graph=graph, **over)
    orc = make_oracle(d, **over)
    out = []
    for _ in range(nsteps):
        sim.step(1)
        rec = orc.step(1)[0]
        sim.sync()
        st = sim.stats(dt.dtsph_step_count(sim.ctx) - 1, 1)[0]
        out.append((st, rec, sim.x, sim.v, sim.p))
    return sim, orc, out


@pytest.mark.parametrize("case,nsteps", [("tgv2d_jitter", 10), ("cavity", 6), ("tgv3d", 3)])
def test_steps_fp64_match_oracle(case, nsteps):
    """Every real step: same iteration count and stop reason, and r, V, p within
    1e-10 normwise relative of the oracle."""
    d = CASES[case]()
    box = box_of(d)
    sim, orc, out = run_pair(d, nsteps)
    for k, (st, rec, x, v, p) in enumerate(out):
        assert (st["iters"], st["reason"]) == (rec["iters"], rec["reason"]), (k, st, rec)
        assert abs(st["rp"] - rec["rp"]) <= 1e-10 * rec["rp"] and abs(st["rv"] - rec["rv"]) <= 1e-10 * rec["rv"]
    st, rec, x, v, p = out[-1]
    assert np.max(np.abs(wrap_diff(x, orc.x[:d["nf"]], box))) < 1e-10 * np.max(np.abs(orc.x))
    assert rel(v, orc.v) < 1e-10
    assert rel(p, orc.p) < 1e-10
    assert rel(sim.v_prev, orc.v_prev) < 1e-10
    sim.close()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("case,nsteps", [("tgv2d_jitter", 4), ("cavity", 3), ("tgv3d", 2)])
def test_shifting_matches_oracle(case, nsteps, prec):
    """Particle shifting with the Taylor correction (Sec. 3.5) after every real
    step against the oracle's shifting: FP64 within 1e-10 with the same
    iteration counts, FP32C velocities within 1e-4; and the shift really moves
    the particles (an unshifted oracle run ends elsewhere)."""
    d = CASES[case]()
    box = box_of(d)
    nf = d["nf"]
    sim, orc, out = run_pair(d, nsteps, precision=prec, shifting=1)
    st, rec, x, v, p = out[-1]
    tol = 1e-10 if prec == dt.DTSPH_FP64 else 1e-4
    if prec == dt.DTSPH_FP64:
        assert [o[0]["iters"] for o in out] == [o[1]["iters"] for o in out]
        assert rel(p, orc.p) < tol
    assert np.max(np.abs(wrap_diff(x, orc.x[:nf], box))) < tol * np.max(np.abs(orc.x))
    assert rel(v, orc.v) < tol
    plain = make_oracle(d)
    plain.step(nsteps)
    moved = np.max(np.abs(wrap_diff(plain.x[:nf], orc.x[:nf], box)))
    assert moved > 1e-6 * np.max(np.abs(orc.x)), moved
    sim.close()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("case", ["tgv2d_jitter", "cavity"])
def test_artificial_viscosity_matches_oracle(case, prec):
    """Monaghan's artificial viscosity (Eqs. mom-av, av-phiij) on: FP64 within
    1e-10 of the oracle with the same iteration counts, FP32C within 1e-4."""
    d = CASES[case]()
    sim, orc, out = run_pair(d, 3, precision=prec, alpha=0.1)
    st, rec, x, v, p = out[-1]
    if prec == dt.DTSPH_FP64:
        assert [o[0]["iters"] for o in out] == [o[1]["iters"] for o in out]
        assert rel(v, orc.v) < 1e-10 and rel(p, orc.p) < 1e-10
    else:
        assert rel(v, orc.v) < 1e-4
    sim.close()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("shift", [0, 1])
def test_dambreak_free_surface_matches_oracle(shift, prec):
    """A water column in a tank under gravity with a free surface: artificial
    viscosity, wall pressure kept >= 0, and (shift = 1) shifting that leaves
    free-surface particles in place. FP64 within 1e-10 of the oracle with the
    same iteration counts, FP32C within 1e-4."""
    d = synth.dambreak2d(12, jitter=0.1, seed=2)
    nf = d["nf"]
    sim, orc, out = run_pair(d, 3, precision=prec, alpha=0.1, free_surface=1, shifting=shift)
    st, rec, x, v, p = out[-1]
    tol = 1e-10 if prec == dt.DTSPH_FP64 else 1e-4
    if prec == dt.DTSPH_FP64:
        assert [o[0]["iters"] for o in out] == [o[1]["iters"] for o in out]
        assert rel(p, orc.p) < tol
    assert np.max(np.abs(x - orc.x[:nf])) < tol * np.max(np.abs(orc.x))
    assert rel(v, orc.v) < tol
    sim.close()


STEADY_CASES = {
    "couette": lambda: synth.couette2d(14, re=5.0),
    "cavity": lambda: synth.cavity2d(18, re=100.0),
    # a viscous vortex (cell Reynolds number U h / nu ~ 0.2): the steady iteration's
    # explicit central convection is unstable at cell Reynolds numbers well above 2
    "tgv2d_viscous": lambda: synth.tgv2d(30, re=5.0, seed=3),
}


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("case", sorted(STEADY_CASES))
@pytest.mark.parametrize("fixed", [300, 0])
def test_steady_mode_matches_oracle(case, prec, fixed):
    """Steady-state mode (Sec. 2.3, Eq. mom-steady): each step is one
    pseudo-time solve at fixed positions, no BDF2 and no EDAC term, with the
    convection term. FP64 within 1e-10 of the oracle's steady mode with the
    same iteration counts (fixed count, and the stop rules), FP32C velocities
    within 1e-4; the particles never move."""
    d = STEADY_CASES[case]()
    nf = d["nf"]
    over = dict(steady=1, fixed_iters=fixed) if fixed else dict(steady=1, max_iter=400)
    sim, orc, out = run_pair(d, 2, precision=prec, **over)
    st, rec, x, v, p = out[-1]
    assert np.array_equal(x, d["x"][:nf])
    tol = 1e-10 if prec == dt.DTSPH_FP64 else 1e-4
    if prec == dt.DTSPH_FP64:
        assert [o[0]["iters"] for o in out] == [o[1]["iters"] for o in out]
        assert rel(p, orc.p) < tol or np.max(np.abs(orc.p)) < 1e-12
    assert rel(v, orc.v) < tol
    sim.close()


def test_steady_couette_from_rest_on_gpu():
    """The steady iteration drives plane Couette flow from rest to u = U y."""
    d = synth.couette2d(16, re=5.0)
    d["v"][:] = 0.0
    d["v_prev"][:] = 0.0
    sim = make_sim(d, precision=dt.DTSPH_FP32C, graph=2, steady=1, fixed_iters=4000)
    sim.step(1)
    nf = d["nf"]
    assert np.max(np.abs(sim.v[:, 0] - d["x"][:nf, 1])) < 2e-3
    assert np.max(np.abs(sim.v[:, 1])) < 1e-5
    sim.close()


def test_steady_same_bits_in_every_graph_mode():
    d = STEADY_CASES["cavity"]()
    runs = []
    for graph in (0, 1, 2):
        sim = make_sim(d, precision=dt.DTSPH_FP32C, graph=graph, lanes=1, steady=1, fixed_iters=50)
        sim.step(2)
        runs.append((sim.v, sim.p, sim.stats()))
        sim.close()
    for r in runs[1:]:
        assert np.array_equal(r[0], runs[0][0]) and np.array_equal(r[1], runs[0][1]) and r[2] == runs[0][2]


def test_steady_with_shifting_is_rejected():
    d = STEADY_CASES["couette"]()
    with pytest.raises(dt.DtsphError):
        make_sim(d, steady=1, shifting=1)


def test_shifting_same_bits_in_every_graph_mode():
    d = CASES["tgv2d_jitter"]()
    runs = []
    for graph in (0, 1, 2):
        sim = make_sim(d, precision=dt.DTSPH_FP32C, graph=graph, lanes=1, shifting=1)
        sim.step(3)
        runs.append((sim.x, sim.v, sim.p))
        sim.close()
    for r in runs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(r, runs[0]))


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_every_lane_split_matches_oracle(lanes, prec):
    """Each lanes-per-particle variant of the iterate kernel (the autotuner's
    candidates) on 2D walls and 3D periodic cases."""
    for case, nsteps in (("cavity", 3), ("tgv3d", 2)):
        d = CASES[case]()
        sim, orc, out = run_pair(d, nsteps, precision=prec, lanes=lanes)
        tol = 1e-10 if prec == dt.DTSPH_FP64 else 1e-4
        assert rel(out[-1][3], orc.v) < tol, (case, lanes)
        if prec == dt.DTSPH_FP64:
            assert [o[0]["iters"] for o in out] == [o[1]["iters"] for o in out]
        sim.close()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_staging_depth_does_not_change_the_bits(prec):
    """The one-lane kernel's shared-memory ring depth only changes how many
    pair-cache chunks are in flight, never the arithmetic."""
    d = CASES["tgv3d"]()
    ref = None
    for stages in (2, 3, 5, 8):
        sim = make_sim(d, precision=prec, graph=2, lanes=1, stages=stages)
        sim.step(2)
        got = (sim.v, sim.p, sim.x, [{k: v for k, v in r.items() if k != "form"} for r in sim.stats()])
        sim.close()
        if ref is None:
            ref = got
        else:
            assert all(np.array_equal(a, b) for a, b in zip(got[:3], ref[:3])) and got[3] == ref[3], stages


def test_autotuner_picks_a_candidate_and_caches_it():
    d = synth.tgv2d(64)
    a = make_sim(d, precision=dt.DTSPH_FP32C, lanes=0)
    lanes, ms = dt.dtsph_tuning(a.ctx)
    assert lanes in (1, 2, 4, 8) and set(ms) == {1, 2, 4, 8} and ms[lanes] == min(ms.values())
    s_use, cand = dt.dtsph_tuning_candidates(a.ctx)
    assert [(c[0], c[1]) for c in cand] == [(1, 2), (1, 3), (1, 4), (1, 6), (2, 0), (4, 0), (8, 0)]
    best = min(cand, key=lambda c: c[2])
    assert (lanes, s_use) == (best[0], best[1])
    b = make_sim(d, precision=dt.DTSPH_FP32C, lanes=0)     # same shape: taken from the cache
    assert dt.dtsph_tuning(b.ctx) == (lanes, {})
    assert dt.dtsph_tuning_candidates(b.ctx) == (s_use, [])
    a.close()
    b.close()


def test_autotuner_choice_persists_across_processes(tmp_path):
    """With DTSPH_TUNE_CACHE set, the first process tunes a shape and appends its
    choice to the file; a fresh process takes the same choice from the file and
    times nothing."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import json, synth, paper_1904_00861_gb300 as dt\n"
            "d = synth.tgv2d(72, seed=2)\n"
            "s = dt.Simulation(d['cfg'], precision=dt.DTSPH_FP32C, lanes=0, graph=2)\n"
            "s.set_state(d['x'], d['v'], d['p'], d['v_prev'])\n"
            "print(json.dumps([dt.dtsph_tuning(s.ctx)[0], *dt.dtsph_tuning_candidates(s.ctx)]))\n")
    env = dict(os.environ, DTSPH_TUNE_CACHE=str(tmp_path / "tune.txt"))
    run = lambda: json.loads(subprocess.run([sys.executable, "-c", code], cwd=root, env=env, check=True,
                                            capture_output=True, text=True).stdout.strip().splitlines()[-1])
    lanes1, stages1, cand1 = run()
    assert len(cand1) == 7
    lines = (tmp_path / "tune.txt").read_text().split("\n")
    assert lines[0].startswith("dtsph-tune-v1 ") and lines[0].split()[-2:] == [str(lanes1), str(stages1 or 3)]
    lanes2, stages2, cand2 = run()
    assert (lanes2, stages2, cand2) == (lanes1, stages1, [])


@pytest.mark.parametrize("graph", [0, 1, 2])
def test_loop_times_cover_each_step(graph):
    """Events around the pseudo-time loop of every step (graph event nodes, or
    events on the stream with plain launches)."""
    d = CASES["tgv2d_jitter"]()
    sim = make_sim(d, precision=dt.DTSPH_FP32C, graph=graph)
    sim.step(3)
    sim.sync()
    ms = dt.dtsph_loop_times(sim.ctx, 0, 3)
    assert len(ms) == 3 and all(0.0 < m < 1e4 for m in ms)
    with pytest.raises(dt.DtsphError):
        dt.dtsph_loop_times(sim.ctx, 2, 2)        # step 3 has not been taken
    sim.close()


def test_graph_and_plain_launches_are_bit_identical():
    d = CASES["tgv2d_jitter"]()
    a = make_sim(d, graph=1, lanes=4)
    b = make_sim(d, graph=0, lanes=4)
    a.step(4)
    b.step(4)
    assert np.array_equal(a.v, b.v) and np.array_equal(a.p, b.p) and np.array_equal(a.x, b.x)
    assert a.stats() == b.stats()
    a.close()
    b.close()


@pytest.mark.parametrize("lanes", [1, 2])
@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("case,nsteps", [("tgv2d_jitter", 4), ("cavity", 3), ("tgv3d", 2)])
def test_persistent_loop_is_bit_identical(case, nsteps, prec, lanes):
    """graph = 2 (the whole pseudo-time loop in one cooperative kernel with a
    grid barrier per iteration) gives the same bits as graph = 1 (one launch
    per iteration in a conditional while node), residuals included. lanes = 1
    streams the pair cache through the bulk-copy ring, which the persistent
    kernel keeps across tiles and iterations."""
    d = CASES[case]()
    a = make_sim(d, precision=prec, graph=1, lanes=lanes)
    b = make_sim(d, precision=prec, graph=2, lanes=lanes)
    a.step(nsteps)
    b.step(nsteps)
    b.sync()
    assert np.array_equal(a.v, b.v) and np.array_equal(a.p, b.p) and np.array_equal(a.x, b.x)
    # the persistent loop picks the pair-term form per step (same bits)
    drop = lambda st: [{k: v for k, v in r.items() if k != "form"} for r in st]
    assert drop(a.stats()) == drop(b.stats())
    a.close()
    b.close()


def test_persistent_loop_matches_oracle_and_caps():
    d = CASES["tgv2d_jitter"]()
    sim, orc, out = run_pair(d, 3, graph=2)
    for st, rec, *_ in out:
        assert (st["iters"], st["reason"]) == (rec["iters"], rec["reason"])
    assert rel(out[-1][3], orc.v) < 1e-10
    sim.close()
    sim = make_sim(d, graph=2, eps=1e-14, stag_window=0, max_iter=7)
    sim.step(2)
    assert [s["iters"] for s in sim.stats()] == [7, 7] and all(s["reason"] == 2 for s in sim.stats())
    sim.close()


def test_fixed_iteration_mode_matches_oracle():
    d = CASES["tgv2d_jitter"]()
    sim, orc, out = run_pair(d, 3, fixed_iters=5)
    for st, rec, *_ in out:
        assert st["iters"] == rec["iters"] == 5 and st["reason"] == rec["reason"] == 4
    assert rel(out[-1][3], orc.v) < 1e-10
    sim.close()


@pytest.mark.parametrize("case,nsteps", [("tgv2d_jitter", 10), ("cavity", 6), ("tgv3d", 3)])
def test_steps_fp32c_linf(case, nsteps):
    """FP32-compensated path: L-inf relative velocity error against the FP64
    oracle after the run (the bar is 1e-4); iteration counts reported."""
    d = CASES[case]()
    sim, orc, out = run_pair(d, nsteps, precision=dt.DTSPH_FP32C)
    its = [(st["iters"], rec["iters"]) for st, rec, *_ in out]
    err = rel(out[-1][3], orc.v)
    perr = rel(out[-1][4], orc.p)
    print(f"{case}: FP32C L-inf rel velocity err {err:.2e}, pressure {perr:.2e}, iters (gpu, oracle) {its}")
    assert err < 1e-4
    sim.close()


def test_full_size_taylor_green_200sq():
    """The 200^2 Taylor-Green workload in the benchmark's launch configuration
    (graph = 2: one persistent loop kernel per step, autotuned lanes): FP64
    against the oracle at 1e-10 and FP32C at 1e-4, over 3 real steps."""
    d = synth.tgv2d(200)
    sim, orc, out = run_pair(d, 3, graph=2)
    for st, rec, *_ in out:
        assert st["iters"] == rec["iters"]
    assert rel(out[-1][3], orc.v) < 1e-10 and rel(out[-1][4], orc.p) < 1e-10
    sim.close()
    sim32 = make_sim(d, precision=dt.DTSPH_FP32C, graph=2)
    sim32.step(3)
    err = rel(sim32.v, orc.v)
    print(f"200^2 FP32C L-inf rel velocity err after 3 steps: {err:.2e}")
    assert err < 1e-4
    sim32.close()


def test_full_size_taylor_green_3d_128():
    """The 128^3 3D Taylor-Green workload (2,097,152 particles) in the
    benchmark's launch configuration, one real step against the oracle's full
    step: FP64 with the same iteration count within 1e-10, FP32C within 1e-4."""
    d = synth.tgv3d(128)
    orc = make_oracle(d)
    rec = orc.step(1)[0]
    for prec, tol in ((dt.DTSPH_FP64, 1e-10), (dt.DTSPH_FP32C, 1e-4)):
        sim = make_sim(d, precision=prec, graph=2)
        sim.step(1)
        sim.sync()
        st = sim.stats(0, 1)[0]
        if prec == dt.DTSPH_FP64:
            assert st["iters"] == rec["iters"]
        err = rel(sim.v, orc.v)
        print(f"128^3 precision {prec}: L-inf rel velocity err after 1 step {err:.2e}")
        assert err < tol
        sim.close()


# -------------------------------------------------------------- invariants

def test_uniform_flow_exact_on_gpu():
    d = synth.tgv2d(33, jitter=0.1, seed=9)
    v = np.tile([0.5, -0.25], (d["nf"], 1))
    d = dict(d, v=v, p=np.zeros(d["nf"]), v_prev=v)
    for prec in (dt.DTSPH_FP64, dt.DTSPH_FP32C):
        sim = make_sim(d, precision=prec)
        sim.step(3)
        assert np.array_equal(sim.v, v) and np.array_equal(sim.p, np.zeros(d["nf"]))
        assert all(s["iters"] == 1 and s["reason"] == 0 for s in sim.stats())
        sim.close()


def test_momentum_conserved_fp64():
    d = synth.tgv2d(40, seed=3)
    rng = np.random.default_rng(4)
    v = d["v"] + 0.05 * rng.normal(size=d["v"].shape)
    d = dict(d, v=v, v_prev=v)
    sim = make_sim(d)
    P0 = v.sum(0)
    sim.step(5)
    assert np.max(np.abs(sim.v.sum(0) - P0)) < 1e-12 * np.abs(v).sum()
    sim.close()


def test_deterministic_and_resume_bit_identical():
    d = CASES["tgv2d_jitter"]()
    a = make_sim(d, lanes=2)
    a.step(4)
    b = make_sim(d, lanes=2)
    b.step(2)
    b.sync()
    x, v, p, vp = b.x, b.v, b.p, b.v_prev
    c = make_sim(dict(d, x=x, v=v, p=p, v_prev=vp), lanes=2)
    c.step(2)
    assert np.array_equal(a.v, c.v) and np.array_equal(a.p, c.p) and np.array_equal(a.x, c.x)
    a2 = make_sim(d, lanes=2)
    a2.step(4)
    assert np.array_equal(a.v, a2.v)
    for s in (a, b, c, a2):
        s.close()


# -------------------------------------------------------------- edge cases

@pytest.mark.parametrize("n", [10, 11, 33])
def test_small_and_ragged_sizes(n):
    """Particle counts that leave partial warps and blocks (10^2 particles is
    the smallest periodic box with three cells wider than 3h per axis)."""
    d = synth.tgv2d(n, seed=n)
    sim, orc, out = run_pair(d, 2)
    assert rel(out[-1][3], orc.v) < 1e-10
    sim.close()


@pytest.mark.parametrize("lanes", [0, 4])
def test_capacity_overflow_reported(lanes):
    """Too small a neighbour capacity is reported (at set-up when the autotuner
    builds a cache there, else at the first sync), never silently truncated."""
    d = synth.tgv2d(30)
    with pytest.raises(dt.DtsphError) as e:
        sim = make_sim(d, max_neighbors=8, lanes=lanes)
        sim.step(1)
        sim.sync()
    assert e.value.code == -5


@pytest.mark.parametrize("lanes", [0, 4])
def test_domain_error_reported(lanes):
    d = synth.cavity2d(12)
    nf = d["nf"]
    x = d["x"].copy()
    x[0] = [-1.0, 0.5]            # outside the closed box
    sim = dt.Simulation(d["cfg"], lanes=lanes)
    with pytest.raises(dt.DtsphError) as e:
        sim.set_state(x[:nf], d["v"], d["p"], walls=(x[nf:], d["vw"]))
        sim.step(1)
        sim.sync()
    assert e.value.code == -6
    sim.close()


def test_call_order_and_argument_errors():
    d = synth.tgv2d(12)
    sim = dt.Simulation(d["cfg"])
    with pytest.raises(dt.DtsphError) as e:
        sim.step(1)
    assert e.value.code == -2
    with pytest.raises(dt.DtsphError):
        dt.dtsph_read_field(sim.ctx, 7, 1, 1)
    sim.set_state(d["x"], d["v"], d["p"])
    with pytest.raises(dt.DtsphError):
        dt.dtsph_read_stats(sim.ctx, 0, 1)      # no step taken yet
    sim.close()


# ------------------------------------------- moving particles (Algorithm 1)

MOVING_CASES = {
    "tgv2d_jitter": (lambda: synth.tgv2d(50, seed=1904), 4),
    "cavity": (lambda: synth.cavity2d(23), 3),
    "tgv3d": (lambda: synth.tgv3d(12, jitter=0.1, seed=5), 2),
    "dambreak": (lambda: synth.dambreak2d(12, jitter=0.1, seed=2), 3),
}


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("moving", [1, 2])
@pytest.mark.parametrize("case", sorted(MOVING_CASES))
def test_moving_matches_oracle(case, moving, prec):
    """Particles moving in pseudo-time (Algorithm 1) against the oracle's
    moving loop, with the lists of r^0 (moving = 1) or neighbours updated at
    every pass (moving = 2: the GPU's lists with a skin against the oracle's
    rebuild): FP64 within 1e-10 with the same iteration counts, FP32C within
    1e-4."""
    make, nsteps = MOVING_CASES[case]
    d = make()
    over = dict(moving=moving)
    if case == "dambreak":
        over.update(alpha=0.1, free_surface=1, shifting=1)
    box = box_of(d)
    nf = d["nf"]
    sim, orc, out = run_pair(d, nsteps, precision=prec, **over)
    st, rec, x, v, p = out[-1]
    if prec == dt.DTSPH_FP64:
        assert [(o[0]["iters"], o[0]["reason"]) for o in out] == [(o[1]["iters"], o[1]["reason"]) for o in out]
        assert rel(v, orc.v) < 1e-10 and rel(p, orc.p) < 1e-10
        assert np.max(np.abs(wrap_diff(x, orc.x[:nf], box))) < 1e-10 * np.max(np.abs(orc.x))
    else:
        e = rel(v, orc.v)
        print(f"{case} moving={moving}: FP32C L-inf rel err {e:.2e}")
        assert e < 1e-4
    sim.close()


def test_moving_one_iteration_equals_frozen_on_gpu():
    """With one pseudo-iteration the moving pass runs at r^0 with V~ = 0 and adds
    nothing, so the FP64 moving step gives the bits of the frozen step with one
    lane per particle (the same summation order)."""
    d = CASES["tgv2d_jitter"]()
    a = make_sim(d, fixed_iters=1, lanes=1)
    b = make_sim(d, fixed_iters=1, moving=1, lanes=1)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v) and np.array_equal(a.p, b.p)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_moving_lanes_agree(prec):
    """1, 2, 4 or 8 lanes per particle in the moving pass only reorder the pair
    sums: the same iteration counts, and velocities within rounding of each
    other (1e-12 in FP64, 1e-5 in FP32C)."""
    d = CASES["cavity"]()
    runs = []
    for L in (1, 2, 4, 8):
        sim = make_sim(d, precision=prec, moving=2, lanes=L)
        sim.step(3)
        sim.sync()
        runs.append((sim.v, [s["iters"] for s in sim.stats(0, 3)]))
        sim.close()
    tol = 1e-12 if prec == dt.DTSPH_FP64 else 1e-5
    for v, its in runs[1:]:
        assert its == runs[0][1] and rel(v, runs[0][0]) < tol


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_moving_same_bits_in_every_graph_mode(prec):
    """Plain launches, the while-node graph and graph = 2 (which runs the moving
    loop as graph = 1) give the same bits."""
    d = CASES["cavity"]()
    res = []
    for g in (0, 1, 2):
        sim = make_sim(d, precision=prec, graph=g, moving=2)
        sim.step(3)
        sim.sync()
        res.append((sim.x, sim.v, sim.p, [s["iters"] for s in sim.stats(0, 3)]))
        sim.close()
    for r in res[1:]:
        assert all(np.array_equal(u, w) for u, w in zip(r[:3], res[0][:3])) and r[3] == res[0][3]


def test_moving_skin_exceeded_is_reported():
    """moving = 2 with a skin far below the pseudo-time displacement ends the
    step with DTSPH_E_SKIN on the host (no device fault); the probe of a moving
    context times the moving pass and leaves the state alone."""
    d = CASES["tgv2d_jitter"]()
    sim = make_sim(d, moving=2, skin=1e-9 * d["cfg"]["h"])
    sim.step(1)
    with pytest.raises(dt.DtsphError) as e:
        sim.sync()
    assert e.value.code == -9
    sim.close()
    sim = make_sim(d, moving=1)
    sim.step(1)
    sim.sync()
    x, v = sim.x, sim.v
    ms, by, npairs = dt.dtsph_probe_iterate(sim.ctx, 2)
    assert ms > 0 and by > 0 and npairs > 0
    assert np.array_equal(sim.x, x) and np.array_equal(sim.v, v)
    sim.close()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("case", ["cavity", "tgv3d"])
def test_probe_after_shifting_leaves_the_run_unchanged(case, prec):
    """With shifting on, the shifting pass after the loop replaces the step's
    neighbour lists by its own; the probe then times the iterate kernel on a
    cache built for the current positions (walls and 3D included). It runs,
    leaves r, V, p alone, and the next step is bit-identical to that of an
    unprobed run. With particles moving in pseudo-time and shifting on, it
    refuses (DTSPH_E_STATE)."""
    d = CASES[case]()
    d["cfg"] = dict(d["cfg"], shifting=1)
    ref = make_sim(d, precision=prec, graph=2)
    ref.step(3)
    ref.sync()
    want = (ref.x, ref.v, ref.p)
    ref.close()
    sim = make_sim(d, precision=prec, graph=2)
    sim.step(2)
    sim.sync()
    x, v, p = sim.x, sim.v, sim.p
    ms, by, npairs = dt.dtsph_probe_iterate(sim.ctx, 3)
    assert ms > 0 and by > 0 and npairs > 0
    assert np.array_equal(sim.x, x) and np.array_equal(sim.v, v) and np.array_equal(sim.p, p)
    sim.step(1)
    sim.sync()
    assert all(np.array_equal(a, b) for a, b in zip((sim.x, sim.v, sim.p), want))
    sim.close()
    if case == "cavity":
        sim = make_sim(d, precision=prec, moving=1)
        sim.step(1)
        sim.sync()
        with pytest.raises(dt.DtsphError) as e:
            dt.dtsph_probe_iterate(sim.ctx, 2)
        assert e.value.code == -2
        sim.close()


def test_host_and_device_transfers_agree():
    """dtsph_set_particles / dtsph_read_field with host arrays (read and written
    in place by kernels where the device accesses pageable memory, through
    cudaMemcpyAsync elsewhere), pageable or pinned, give the same state as the
    device-pointer entry points."""
    torch = pytest.importorskip("torch")
    d = CASES["cavity"]()
    nf = d["nf"]
    a = make_sim(d)
    a.step(2)
    a.sync()
    x = dt.dtsph_read_field(a.ctx, dt.FIELD_POS, nf, 2)
    v = dt.dtsph_read_field(a.ctx, dt.FIELD_VEL, nf, 2)
    p = dt.dtsph_read_field(a.ctx, dt.FIELD_P, nf, 1)
    vp = dt.dtsph_read_field(a.ctx, dt.FIELD_VEL_PREV, nf, 2)
    xd = torch.empty((nf, 2), dtype=torch.float64, device="cuda")
    dt.dtsph_read_field_device(a.ctx, dt.FIELD_POS, xd)
    torch.cuda.synchronize()
    assert np.array_equal(x, xd.cpu().numpy())
    pin = torch.empty((nf, 2), dtype=torch.float64, pin_memory=True).numpy()
    dt.dtsph_read_field(a.ctx, dt.FIELD_VEL, nf, 2, out=pin)
    assert np.array_equal(pin, v)
    # the whole state in one call, field by field the same
    xs, vs, ps, vps = dt.dtsph_read_state(a.ctx, nf, 2)
    assert all(np.array_equal(u, w) for u, w in ((xs, x), (vs, v), (ps, p), (vps, vp)))
    # the same state sent from host arrays and from device arrays steps to the same bits
    b = make_sim(d)
    dt.dtsph_set_particles(b.ctx, x, v, p, vp)
    c = make_sim(d)
    t = [torch.from_numpy(np.ascontiguousarray(u)).cuda() for u in (x, v, p, vp)]
    torch.cuda.synchronize()
    dt.dtsph_set_particles_device(c.ctx, nf, *t)
    b.step(1)
    c.step(1)
    b.sync()
    c.sync()
    for f, comps in ((dt.FIELD_POS, 2), (dt.FIELD_VEL, 2), (dt.FIELD_P, 1)):
        assert np.array_equal(dt.dtsph_read_field(b.ctx, f, nf, comps), dt.dtsph_read_field(c.ctx, f, nf, comps))
    for s in (a, b, c):
        s.close()


@pytest.mark.parametrize("graph", [0, 1, 2])
def test_step_stats_report_max_velocity(graph):
    """dtsph_step_stats.vmax is max |V^{n+1}| over the fluid particles: the
    maximum over the velocities read back after the step (to an ulp or two), and within 1e-10
    of the oracle's on the FP64 path (the Taylor-Green decay diagnostic)."""
    d = CASES["tgv2d_jitter"]()
    sim = make_sim(d, graph=graph)
    orc = make_oracle(d)
    for k in range(3):
        sim.step(1)
        orc.step(1)
        st = sim.stats(k, 1)[0]
        v = sim.v
        vmax = np.max(np.sqrt(np.sum(v * v, axis=1)))
        assert abs(st["vmax"] - vmax) <= 4e-16 * vmax       # the GPU sums the squares with FMA
        vo = np.max(np.sqrt(np.sum(orc.v * orc.v, axis=1)))
        assert abs(st["vmax"] - vo) < 1e-10 * vo
    sim.close()


@pytest.mark.parametrize("graph", [0, 1, 2])
@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("case", ["tgv2d_jitter", "tgv3d"])
def test_form_without_cache_gives_the_bits_of_the_cache(case, prec, graph):
    """form = 2 recomputes every pair's geometry in every pseudo-iteration from
    the lists at r^0, with the operations of the pair-cache pass: the same
    positions, velocities, pressures and iteration counts, bit for bit, as
    form = 1 (the cache), for one and four lanes per particle."""
    d = CASES[case]()
    nsteps = 4 if case == "tgv2d_jitter" else 2
    for lanes in (1, 4):
        out = []
        for form in (1, 2):
            sim = make_sim(d, precision=prec, graph=graph, lanes=lanes, form=form)
            sim.step(nsteps)
            sim.sync()
            out.append((sim.x, sim.v, sim.p, [s["iters"] for s in sim.stats()]))
            sim.close()
        assert all(np.array_equal(a, b) for a, b in zip(out[0][:3], out[1][:3])), lanes
        assert out[0][3] == out[1][3], lanes


def test_form_without_cache_in_a_batch_and_its_limits():
    """A batch without walls (the decoupled loop) gives the same bits in both
    forms; form = 2 is refused with walls (their values come from the cache)
    and with particles moving in pseudo-time."""
    work = [synth.tgv2d(37, re=100.0, seed=11), synth.tgv2d(20, re=630.0, seed=12),
            synth.tgv2d(45, re=250.0, seed=13)]
    res = []
    for form in (1, 2):
        b = dt.Batch([dict(w["cfg"], form=form) for w in work], precision=dt.DTSPH_FP32C, graph=2, lanes=1)
        b.set_state(work)
        b.step(3)
        b.sync()
        res.append((b.field(dt.FIELD_VEL), [[s["iters"] for s in b.stats(i)] for i in range(len(work))]))
        b.close()
    assert all(np.array_equal(a, c) for a, c in zip(res[0][0], res[1][0])) and res[0][1] == res[1][1]
    cav = CASES["cavity"]()
    with pytest.raises(dt.DtsphError) as e:
        make_sim(cav, precision=dt.DTSPH_FP32C, graph=2, form=2)
    assert e.value.code == dt.DTSPH_E_UNSUPPORTED
    with pytest.raises(dt.DtsphError) as e:
        dt.Simulation(CASES["tgv2d_jitter"]()["cfg"], precision=dt.DTSPH_FP32C, moving=1, form=2)
    assert e.value.code == dt.DTSPH_E_UNSUPPORTED


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_form_without_cache_at_200sq_every_lane_count(prec):
    """The persistent loop without the cache at 200^2, where there are more
    tiles than SMs and several blocks share an SM: the bits of the cached form
    over three steps at 1, 2, 4 and 8 lanes per particle."""
    d = synth.tgv2d(200)
    for lanes in (1, 2, 4, 8):
        out = []
        for form in (1, 2):
            sim = make_sim(d, precision=prec, graph=2, lanes=lanes, form=form)
            sim.step(3)
            sim.sync()
            out.append((sim.v, sim.p, [s["iters"] for s in sim.stats()]))
            sim.close()
        assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1]), lanes
        assert out[0][2] == out[1][2], lanes


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_automatic_form_gives_the_bits_and_reports_its_choice(prec):
    """form = 0 on the persistent loop measures the cache pass and one
    pseudo-iteration in each form at dtsph_set_particles, then picks the form
    of each step on the device from the previous step's iteration count: the bits of
    form = 1 whatever it picks, k* = cache / (uncached - cached), and every step
    counted in one of the two forms."""
    d = CASES["tgv2d_jitter"]()
    out = []
    for form in (1, 0):
        sim = make_sim(d, precision=prec, graph=2, lanes=1, form=form)
        sim.step(5)
        sim.sync()
        st = sim.stats()
        out.append((sim.x, sim.v, sim.p, [s["iters"] for s in st], sim.form_stats(), [s["form"] for s in st]))
        sim.close()
    assert all(np.array_equal(a, b) for a, b in zip(out[0][:3], out[1][:3]))
    assert out[0][3] == out[1][3] and out[0][5] == [1] * 5
    fixed, auto = out[0][4], out[1][4]
    assert fixed["kstar"] < 0 and fixed["steps_cache"] == 5 and fixed["steps_nocache"] == 0
    ms = auto["ms"]
    assert ms[0] >= 0 and ms[1] > 0 and ms[2] > 0
    want = ms[0] / (ms[2] - ms[1]) if ms[2] > ms[1] else 1e9
    assert auto["kstar"] == pytest.approx(want, rel=1e-5)
    assert auto["steps_cache"] + auto["steps_nocache"] + auto["steps_switched"] == 5
    assert out[1][5].count(2) == auto["steps_nocache"] and out[1][5].count(3) == auto["steps_switched"]
    # a form = 2 context reports every step uncached
    sim = make_sim(d, precision=prec, graph=2, lanes=1, form=2)
    sim.step(2)
    assert [s["form"] for s in sim.stats()] == [2, 2] and sim.form_stats()["steps_nocache"] == 2
    sim.close()


def form_rule(iters, nfs, kstar):
    """The form each step of a form = 0 run takes: without the cache when the
    previous step's iterations, averaged over the instances with their fluid
    counts as weights, are at most kstar (an instance with no step yet counts
    one iteration), else with it (1). Without the cache the loop pauses after
    m = floor(kstar) iterations (1 <= kstar < 1e6), so a step in which some
    instance takes more than m iterations switches to the cache (3); otherwise
    it stays without it (2)."""
    m = int(kstar) if 1.0 <= kstar < 1e6 else 0
    prev = [1] * len(nfs)
    forms = []
    for k in range(len(iters[0])):
        kw = float(sum(nf * p for nf, p in zip(nfs, prev)))
        its = [i[k] for i in iters]
        if kw > kstar * float(sum(nfs)):
            forms.append(1)
        else:
            forms.append(3 if m > 0 and max(its) > m else 2)
        prev = its
    return forms


def test_automatic_form_follows_the_iteration_count(tmp_path):
    """The per-step choice follows the rule exactly, in a solo context and in a
    batch, for thresholds below, between and above the iteration counts: the
    measured costs persist in DTSPH_TUNE_CACHE, a fresh process reads the
    threshold from there, so the test sets kstar by editing the file. A loop
    without the cache that pauses and goes on with it (form 3) takes the same
    iterations; the bits do not depend on the choice."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import json, numpy as np, synth, paper_1904_00861_gb300 as dt\n"
            "out = {}\n"
            "d = synth.tgv2d(41, seed=5)\n"
            "s = dt.Simulation(d['cfg'], precision=dt.DTSPH_FP32C, graph=2, lanes=1, stages=2)\n"
            "s.set_state(d['x'], d['v'], d['p'], d['v_prev'])\n"
            "s.step(6)\n"
            "st = s.stats()\n"
            "out['solo'] = dict(iters=[[r['iters'] for r in st]], forms=[r['form'] for r in st], nfs=[d['nf']],\n"
            "                   fs=s.form_stats(), v=float(np.sum(np.abs(s.v))))\n"
            "w = [synth.tgv2d(29, re=100.0, seed=21), synth.tgv2d(17, re=630.0, seed=22),\n"
            "     synth.tgv2d(33, re=250.0, seed=23)]\n"
            "b = dt.Batch([x['cfg'] for x in w], precision=dt.DTSPH_FP32C, graph=2, lanes=1, stages=2)\n"
            "b.set_state(w)\n"
            "b.step(6)\n"
            "out['batch'] = dict(iters=[[r['iters'] for r in b.stats(i)] for i in range(3)],\n"
            "                    forms=[r['form'] for r in b.stats(0)], nfs=[x['nf'] for x in w], fs=b.form_stats(),\n"
            "                    v=float(sum(np.sum(np.abs(v)) for v in b.field(dt.FIELD_VEL))))\n"
            "d = synth.tgv3d(16, jitter=0.1, seed=9)\n"
            "s = dt.Simulation(d['cfg'], precision=dt.DTSPH_FP32C, graph=2, lanes=1, stages=2)\n"
            "s.set_state(d['x'], d['v'], d['p'], d['v_prev'])\n"
            "s.step(6)\n"
            "st = s.stats()\n"
            "out['solo3'] = dict(iters=[[r['iters'] for r in st]], forms=[r['form'] for r in st], nfs=[d['nf']],\n"
            "                    fs=s.form_stats(), v=float(np.sum(np.abs(s.v))))\n"
            "print(json.dumps(out))\n")
    path = tmp_path / "tune.txt"
    env = dict(os.environ, DTSPH_TUNE_CACHE=str(path))
    run = lambda: json.loads(subprocess.run([sys.executable, "-c", code], cwd=root, env=env, check=True,
                                            capture_output=True, text=True).stdout.strip().splitlines()[-1])
    first = run()
    lines = [ln.split() for ln in path.read_text().splitlines() if ln.startswith("dtsph-form-v1 ")]
    assert len(lines) == 3
    names = ("solo", "batch", "solo3")
    for name in names:
        r = first[name]
        assert r["forms"] == form_rule(r["iters"], r["nfs"], r["fs"]["kstar"]), name
        assert r["fs"]["steps_nocache"] == r["forms"].count(2) and r["fs"]["steps_cache"] == r["forms"].count(1)
        assert r["fs"]["steps_switched"] == r["forms"].count(3)
    # thresholds that put every step in one form, one that switches after one
    # iteration, and one between the counts
    allk = sorted({k for name in names for its in first[name]["iters"] for k in its})
    mid = 0.5 * (allk[0] + allk[-1])
    seen = set()
    # 1.5: every first step starts without the cache and pauses after one iteration
    for kstar in (0.5, 1.5, mid, 1e6):
        path.write_text("".join(" ".join(ln[:9] + [repr(kstar)] + ln[10:]) + "\n" for ln in lines))
        got = run()
        for name in names:
            r = got[name]
            assert r["fs"]["kstar"] == kstar
            assert r["iters"] == first[name]["iters"] and r["v"] == first[name]["v"], (name, kstar)
            assert r["forms"] == form_rule(r["iters"], r["nfs"], kstar), (name, kstar)
            seen.update(r["forms"])
        if kstar == 0.5:
            assert all(got[name]["forms"] == [1] * 6 for name in names)
        if kstar == 1e6:
            assert all(got[name]["forms"] == [2] * 6 for name in names)
    assert seen == {1, 2, 3}


def test_automatic_form_counts_restart_with_the_state():
    """A second set_particles of the same shape keeps k* (no new measurement)
    and restarts the per-form step counts."""
    d = CASES["tgv2d_jitter"]()
    sim = make_sim(d, precision=dt.DTSPH_FP32C, graph=2, lanes=1, form=0)
    sim.step(3)
    fs = sim.form_stats()
    assert fs["steps_cache"] + fs["steps_nocache"] + fs["steps_switched"] == 3 and fs["kstar"] > 0
    sim.set_state(d["x"][:d["nf"]], d["v"], d["p"], d["v_prev"])
    fs2 = sim.form_stats()
    assert fs2["steps_cache"] == 0 and fs2["steps_nocache"] == 0 and fs2["steps_switched"] == 0
    assert fs2["kstar"] == fs["kstar"]
    sim.step(2)
    fs3 = sim.form_stats()
    assert fs3["steps_cache"] + fs3["steps_nocache"] + fs3["steps_switched"] == 2
    sim.close()


# ------------------------------------------------- lists reused at r^n (list_skin)

@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
@pytest.mark.parametrize("case", ["tgv2d_jitter", "tgv3d"])
def test_reused_lists_match_the_oracle(case, prec):
    """list_skin = h/20: the lists built at r^0 to 3h + skin also serve the next
    step's pass at r^n (pairs beyond 3h add exact zeros). Over four steps: the
    oracle's velocities and pressures (1e-10 FP64, 1e-5 FP32C relative) and the
    iteration counts of the two-build pipeline, step by step; an eval_rates call
    between steps (which bins and lists anew) changes nothing."""
    d = CASES[case]()
    h = d["cfg"]["h"]
    reuse = make_sim(d, precision=prec, graph=2, lanes=1, list_skin=0.05 * h)
    base = make_sim(d, precision=prec, graph=2, lanes=1)
    orc = make_oracle(d)
    for k in range(4):
        reuse.step(1)
        base.step(1)
        orc.step(1)
        if k == 1:
            reuse.rates()
    reuse.sync()
    tol = 1e-10 if prec == dt.DTSPH_FP64 else 1e-5
    assert rel(reuse.v, orc.v) < tol and rel(reuse.p, orc.p) < 10 * tol
    assert [r["iters"] for r in reuse.stats()] == [r["iters"] for r in base.stats()]
    assert rel(reuse.v, base.v) < tol
    reuse.close()
    base.close()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_reused_lists_with_particles_crossing_the_periodic_edges(prec):
    """The Taylor-Green field carried by a uniform drift, so that particles
    cross the periodic edges every step (the vortex alone has no flow through
    them): with the r^0 lists reused at r^n, a particle wrapped to the far side
    keeps the FP32 offset its lists' cell shifts assume, and after four steps
    the velocities and pressures match the oracle's as without reuse."""
    d = CASES["tgv2d_jitter"]()
    v = d["v"] + np.array([0.5, -0.25])
    d = dict(d, v=v, v_prev=v)
    h = d["cfg"]["h"]
    reuse = make_sim(d, precision=prec, graph=2, lanes=1, list_skin=0.05 * h)
    orc = make_oracle(d)
    reuse.step(4)
    recs = orc.step(4)
    reuse.sync()
    tol = 1e-10 if prec == dt.DTSPH_FP64 else 1e-5
    assert rel(reuse.v, orc.v) < tol and rel(reuse.p, orc.p) < 10 * tol
    assert [r["iters"] for r in reuse.stats()] == [r["iters"] for r in recs]
    reuse.close()


@pytest.mark.parametrize("prec", [dt.DTSPH_FP64, dt.DTSPH_FP32C])
def test_reused_lists_survive_setting_the_state_again(prec):
    """With reused lists, setting the state read back after a step (same
    particles) writes it into the slots as they are and keeps the lists: the
    run then has the bits of one that never left the device, across periodic
    edges (a drift carries particles through them)."""
    d = CASES["tgv2d_jitter"]()
    v = d["v"] + np.array([0.5, -0.25])
    d = dict(d, v=v, v_prev=v)
    skin = 0.05 * d["cfg"]["h"]
    a = make_sim(d, precision=prec, graph=2, lanes=1, list_skin=skin)
    b = make_sim(d, precision=prec, graph=2, lanes=1, list_skin=skin)
    a.step(4)
    b.step(2)
    x, vb, p, vp = dt.dtsph_read_state(b.ctx, b.nf, 2)
    b.set_state(x, vb, p, vp)
    b.step(2)
    for s in (a, b):
        s.sync()
    assert np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v) and np.array_equal(a.p, b.p)
    assert [r["iters"] for r in a.stats()][2:] == [r["iters"] for r in b.stats()]
    a.close()
    b.close()


def test_reused_lists_in_a_batch_and_their_limits():
    """A batch with each instance's own list skin (h/20) takes the iterations
    of the instances' solo runs with two builds per step and their velocities to
    FP32 rounding; with a skin too small for any step's motion every step bins
    and lists at r^n again, with the same results; walls, shifting and the other
    loop drivers are refused."""
    work = [synth.tgv2d(37, re=100.0, seed=11), synth.tgv2d(20, re=630.0, seed=12),
            synth.tgv2d(45, re=250.0, seed=13)]
    b = dt.Batch([dict(w["cfg"], list_skin=0.05 * w["cfg"]["h"]) for w in work], precision=dt.DTSPH_FP32C,
                 graph=2, lanes=1)
    b.set_state(work)
    b.step(3)
    b.sync()
    vb = b.field(dt.FIELD_VEL)
    for i, w in enumerate(work):
        s = make_sim(w, precision=dt.DTSPH_FP32C, graph=2, lanes=1)
        s.step(3)
        assert [r["iters"] for r in b.stats(i)] == [r["iters"] for r in s.stats()], i
        assert rel(vb[i], s.v) < 1e-5, i
        s.close()
    b.close()
    d = CASES["tgv2d_jitter"]()
    tiny = make_sim(d, precision=dt.DTSPH_FP32C, graph=2, lanes=1, list_skin=1e-12)
    base = make_sim(d, precision=dt.DTSPH_FP32C, graph=2, lanes=1)
    for s in (tiny, base):
        s.step(4)
        s.sync()
    assert [r["iters"] for r in tiny.stats()] == [r["iters"] for r in base.stats()]
    assert rel(tiny.v, base.v) < 1e-5
    tiny.close()
    base.close()
    with pytest.raises(dt.DtsphError) as e:
        make_sim(CASES["cavity"](), precision=dt.DTSPH_FP32C, graph=2, list_skin=1e-3)
    assert e.value.code == dt.DTSPH_E_UNSUPPORTED
    for over in (dict(shifting=1), dict(graph=1)):
        with pytest.raises(dt.DtsphError) as e:
            dt.Simulation(d["cfg"], precision=dt.DTSPH_FP32C, **dict(dict(graph=2, list_skin=1e-3), **over))
        assert e.value.code == dt.DTSPH_E_UNSUPPORTED
