"""Batched sweep (hbf_batch_*): cavities of different sizes and rheologies
advanced together, one persistent launch per stage.  Per cavity the batch runs
the single-context step's arithmetic; only the summation order of norms and
dot products differs.  Checked against separate contexts advanced from the
same states (FP64 and mixed), against the FP64 oracle, across tilings, with
per-cavity tolerances, and for the size rule of the exact bottom solve."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.grid import Grid  # noqa: E402
from oracle.step import Rheology, step  # noqa: E402
from paper_1803_00417_gb300.inputs import cavity, random_state  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_00417_gb300 import build

    build.build()


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# sizes chosen so that the hierarchies differ in depth and bottom shape
# (2 x 2, 3 x 3, 4 x 2 and 2 x 2 x 2 coarsest levels)
CASES_2D = [
    ((32, 32), dict(Re=1.0, Bi=2.0, Pa=1e4, nexp=1.0), 41),
    ((48, 48), dict(Re=1000.0, Bi=5.0, Pa=1e5, nexp=0.5), 42),
    ((64, 32), dict(Re=10.0, Bi=20.0, Pa=1e4, nexp=1.5), 43),
    ((16, 16), dict(Re=100.0, Bi=0.0, Pa=1e4, nexp=1.0), 44),
]
CASES_3D = [
    ((8, 8, 8), dict(Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5), 51),
    ((16, 8, 8), dict(Re=10.0, Bi=2.0, Pa=1e4, nexp=0.7), 52),
]


def make_batch(cases, precision, rtols=None):
    from paper_1803_00417_gb300.hbflow import Batch

    cfgs = [cavity(n, **over) for n, over, _ in cases]
    B = Batch([c["n"] for c in cfgs], [c["h"] for c in cfgs], [c["wall_u"] for c in cfgs], precision=precision)
    states = []
    for i, ((n, _, seed), cfg) in enumerate(zip(cases, cfgs)):
        v = B.cavity(i)
        v.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
        if rtols is not None:
            v.set_solver(rtol=rtols[i])
        u, p = random_state(cfg["n"], seed=seed)
        v.set_velocity(u)
        v.set_pressure(p)
        states.append((u, p))
    B.set_dt([c["dt"] for c in cfgs])
    return B, cfgs, states


def singles(cfgs, states, precision, rtols=None):
    from paper_1803_00417_gb300.hbflow import HBFlow

    out = []
    for i, (cfg, (u, p)) in enumerate(zip(cfgs, states)):
        s = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=precision)
        s.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
        if rtols is not None:
            s.set_solver(rtol=rtols[i])
        s.set_velocity(u)
        s.set_pressure(p)
        out.append(s)
    return out


def compare(B, sims, cfgs, nsteps, tol, cyc_slack=1):
    for k in range(nsteps):
        bst = B.step()
        for i, (s, cfg) in enumerate(zip(sims, cfgs)):
            sst = s.step(cfg["dt"])
            for key in ("mac", "visc", "nodal"):
                assert bst[i][key]["converged"], (i, key, bst[i][key])
                assert abs(bst[i][key]["cycles"] - sst[key]["cycles"]) <= cyc_slack, (i, key, bst[i], sst)
            v = B.cavity(i)
            eu = rel(v.get_field("U"), s.get_field("U"))
            ep = rel(v.get_field("P"), s.get_field("P"))
            assert eu < tol and ep < tol, (k, i, eu, ep)


def test_batch_2d_fp64_matches_single_contexts():
    from paper_1803_00417_gb300.hbflow import FP64

    B, cfgs, states = make_batch(CASES_2D, FP64)
    sims = singles(cfgs, states, FP64)
    compare(B, sims, cfgs, 3, 1e-10)
    assert B.launch_count() > 0
    B.close()


def test_batch_2d_mixed_matches_single_contexts():
    from paper_1803_00417_gb300.hbflow import MIXED

    B, cfgs, states = make_batch(CASES_2D, MIXED)
    sims = singles(cfgs, states, MIXED)
    compare(B, sims, cfgs, 3, 1e-6, cyc_slack=2)
    B.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_3d_matches_single_contexts(precision):
    B, cfgs, states = make_batch(CASES_3D, precision)
    sims = singles(cfgs, states, precision)
    compare(B, sims, cfgs, 2, 1e-10 if precision == 0 else 1e-6, cyc_slack=1 if precision == 0 else 2)
    B.close()


def test_batch_matches_oracle():
    from paper_1803_00417_gb300.hbflow import FP64

    cases = [CASES_2D[0], CASES_2D[2]]
    B, cfgs, states = make_batch(cases, FP64)
    st = B.step()
    for i, cfg in enumerate(cfgs):
        u, p = states[i]
        g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
        ref = step(g, u, p, cfg["dt"], Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"]))
        v = B.cavity(i)
        for key in ("mac", "visc", "nodal"):
            assert st[i][key]["rnorm"] <= 1e-10 * st[i][key]["bnorm"]
        eu = rel(np.concatenate([c.ravel() for c in v.velocity()]), np.concatenate([c.ravel() for c in ref.u]))
        ep = rel(v.pressure(), ref.p)
        assert eu < 1e-10 and ep < 1e-10, (i, eu, ep)
    B.close()


def test_batch_tilings_agree():
    from paper_1803_00417_gb300.hbflow import FP64

    outs = []
    for tile, bps in ((256, 2), (4096, 16)):
        B, cfgs, states = make_batch(CASES_2D, FP64)
        B.set_tiling(tile, bps)
        B.step()
        B.step()
        assert B.tiling()["tile"] == tile
        outs.append([B.cavity(i).get_field("U") for i in range(len(cfgs))])
        B.close()
    for a, b in zip(*outs):
        assert rel(a, b) < 1e-10


def test_batch_per_cavity_tolerance_and_masking():
    """A cavity with a looser tolerance stops earlier; the others are unaffected."""
    from paper_1803_00417_gb300.hbflow import FP64

    rtols = [1e-10, 1e-5, 1e-10, 1e-10]
    B, cfgs, states = make_batch(CASES_2D, FP64, rtols=rtols)
    sims = singles(cfgs, states, FP64, rtols=rtols)
    compare(B, sims, cfgs, 2, 1e-9)
    st = B.step()
    assert st[1]["nodal"]["cycles"] < st[0]["nodal"]["cycles"] or st[1]["visc"]["cycles"] < st[0]["visc"]["cycles"]
    B.close()


def test_batch_autotune_then_step():
    from paper_1803_00417_gb300.hbflow import MIXED

    B, cfgs, states = make_batch(CASES_2D, MIXED)
    sims = singles(cfgs, states, MIXED)
    best = B.autotune(reps=2)
    assert best["tile"] in (1024, 2048, 4096, 8192) and best["probe_ms"] > 0
    assert B.tiling()["tile"] == best["tile"]
    compare(B, sims, cfgs, 1, 1e-6, cyc_slack=2)
    B.close()


def test_batch_rejects_cavity_without_exact_bottom():
    from paper_1803_00417_gb300.hbflow import FP64, Batch, HBFlowError

    B = Batch([(32, 32), (26, 26)], [1 / 32, 1 / 26], precision=FP64)
    B.set_dt([0.01, 0.01])
    with pytest.raises(HBFlowError, match="exact"):
        B.step()
    B.close()


def test_batch_sweep_full_size_sample():
    """The 64-cavity sweep the bench times (mixed precision): after one batched
    step, one cavity of each size matches a separate context stepped from the
    same state, and every solve of every cavity reached its tolerance."""
    from paper_1803_00417_gb300.hbflow import MIXED, Batch, HBFlow
    from paper_1803_00417_gb300.inputs import batch_sweep

    cfgs = batch_sweep(ncav=64, seed=0)
    B = Batch([c["n"] for c in cfgs], [c["h"] for c in cfgs], [c["wall_u"] for c in cfgs], precision=MIXED)
    states = []
    for i, c in enumerate(cfgs):
        v = B.cavity(i)
        v.set_rheology(c["K"], c["nexp"], c["tau_y"], c["m"])
        u, p = random_state(c["n"], seed=1000 + i, amp=0.5)
        v.set_velocity(u)
        v.set_pressure(p)
        states.append((u, p))
    B.set_dt([c["dt"] for c in cfgs])
    B.autotune(reps=1)
    st = B.step()
    for i in range(len(cfgs)):
        for key in ("mac", "visc", "nodal"):
            assert st[i][key]["converged"], (i, key, st[i][key])
    picked = {}
    for i, c in enumerate(cfgs):
        picked.setdefault(c["n"][0], i)
    assert len(picked) == 4
    for size, i in sorted(picked.items()):
        c = cfgs[i]
        s = HBFlow(c["n"], c["h"], c["wall_u"], precision=MIXED)
        s.set_rheology(c["K"], c["nexp"], c["tau_y"], c["m"])
        s.set_velocity(states[i][0])
        s.set_pressure(states[i][1])
        s.step(c["dt"])
        eu = rel(B.cavity(i).get_field("U"), s.get_field("U"))
        ep = rel(B.cavity(i).get_field("P"), s.get_field("P"))
        s.close()
        assert eu < 1e-6 and ep < 1e-6, (size, i, eu, ep)
    B.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_fused_tail_matches_level_by_level(precision):
    """The fused V-cycle tail (one block per cavity over its small levels)
    performs the level-by-level launches' operations in the same order: the
    steps agree to rounding with the tail off, on, and covering every level."""
    outs = []
    for cells in (0, 300, 1 << 20):
        B, cfgs, states = make_batch(CASES_2D, precision)
        B.set_tail(cells)
        for _ in range(2):
            st = B.step()
            assert all(s[k]["converged"] for s in st for k in ("mac", "visc", "nodal"))
        outs.append([np.concatenate([B.cavity(i).get_field("U"), B.cavity(i).get_field("P")])
                     for i in range(len(cfgs))])
        B.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert rel(b, a) < 1e-12
