"""The start-up / steady-state / cessation study (Sec. III A steady
criterion; Sec. IV) and its diagnostics through the C-ABI, against the
oracle's ``diagnostics`` module on the same seeded inputs.

* checkpoint: a context restored from another's record and fields (in
  memory and through files) continues bit for bit like the original;
* |tau|, the unyielded cells and their zones (stagnant / plug / attached):
  the maximum to 1e-12, the zone partition and kinds exactly (both sides take
  the |tau| <= tau_y decision in FP64; no cell lies within 1e-9 of it here);
* centre lines and the stream function to 1e-13, the vortex centre to 1e-12;
* the drivers: from rest, the steady criterion stops after the oracle's
  number of steps with its change, and cessation after the lid stops ends
  after the oracle's number of steps with its t_c.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import diagnostics as dg  # noqa: E402
from oracle.grid import Grid  # noqa: E402
from oracle.step import Rheology  # noqa: E402
from paper_1803_00417_gb300.inputs import cavity, random_state  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_00417_gb300 import build

    build.build()


def _pair(n, seed, amp, **over):
    from paper_1803_00417_gb300.hbflow import HBFlow

    cfg = cavity(n, **over)
    u, p = random_state(cfg["n"], seed=seed, amp=amp)
    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"])
    sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    sim.set_velocity(u)
    sim.set_pressure(p)
    g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
    rh = Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    return sim, g, rh, cfg, u, p


def test_checkpoint_restores_a_context(tmp_path):
    from paper_1803_00417_gb300.hbflow import HBFlow

    sim, g, rh, cfg, u, p = _pair((24, 16), 71, 0.5, Re=10.0, Bi=3.0, Pa=1e3, nexp=0.8)
    sim.set_density(1.3)
    sim.set_body_force([0.2, -0.1])
    for _ in range(2):
        sim.step(cfg["dt"])
    rec, uf, pf = sim.get_state()
    assert rec["step"] == 2 and rec["t"] == pytest.approx(2 * cfg["dt"], rel=1e-15)
    assert rec["tau_y"] == cfg["tau_y"] and rec["rho"] == 1.3
    other = HBFlow(cfg["n"], cfg["h"])  # resting walls and default rheology until restored
    other.set_state(rec, uf, pf)
    sim.save_checkpoint(str(tmp_path / "ck"))
    third = HBFlow(cfg["n"], cfg["h"])
    rec3 = third.load_checkpoint(str(tmp_path / "ck"))
    assert rec3 == rec
    for s in (sim, other, third):
        s.step(cfg["dt"])
    ref = sim.get_field("U")
    assert np.array_equal(other.get_field("U"), ref)
    assert np.array_equal(third.get_field("U"), ref)
    assert other.get_state(False)[0]["step"] == 3
    # a record of another grid is refused
    small = HBFlow((8, 8), 1.0 / 8)
    from paper_1803_00417_gb300.hbflow import HBFlowError

    with pytest.raises(HBFlowError):
        small.set_state(rec)
    for s in (sim, other, third, small):
        s.close()


def _canonical(labels_oracle, n):
    """Oracle component indices -> the smallest x-fastest cell index of each
    component (the GPU's label); -1 stays."""
    flat = labels_oracle.T.ravel()  # x fastest
    out = -np.ones_like(flat)
    for k in np.unique(flat[flat >= 0]):
        idx = np.nonzero(flat == k)[0]
        out[idx] = idx.min()
    return out.reshape(labels_oracle.T.shape).T


@pytest.mark.parametrize("n,seed,amp", [((40, 24), 72, 4e-3), ((16, 12, 10), 73, 4e-3), ((64, 64), 74, 4e-3)])
def test_yield_zones_match_oracle(n, seed, amp):
    sim, g, rh, cfg, u, p = _pair(n, seed, amp, Re=1.0, Bi=10.0, Pa=400.0, nexp=1.0)
    info = sim.yield_info(labels=True)
    tau = dg.stress_norm(u, g, rh)
    assert info["tau_max"] == pytest.approx(float(np.max(tau)), rel=1e-12)
    assert np.min(np.abs(tau / rh.tau_y - 1.0)) > 1e-9  # no decision at the rounding level
    mask = tau <= rh.tau_y
    labels, comps = dg.zones(mask, g)
    assert 0 < mask.sum() < mask.size  # both kinds of cells occur
    assert sum(1 for c in comps if c["kind"] == "plug") > 0 and len(comps) > 1
    np.testing.assert_array_equal(info["labels"], _canonical(labels, g.n))
    assert info["yielded"] == int((~mask).sum())
    for kind in ("stagnant", "plug", "attached"):
        assert info["zones"][kind] == sum(1 for c in comps if c["kind"] == kind)
        assert info["cells"][kind] == sum(c["size"] for c in comps if c["kind"] == kind)
    sim.close()


@pytest.mark.parametrize("n,seed", [((40, 24), 75), ((12, 10, 14), 76), ((15, 9, 8), 77)])
def test_centrelines_and_vortex_match_oracle(n, seed):
    sim, g, rh, cfg, u, p = _pair(n, seed, 1.0)
    for comp in range(g.d):
        for along in range(g.d):
            ref = dg.centreline(u, g, comp, along)
            np.testing.assert_allclose(sim.centreline(comp, along), ref, rtol=0, atol=1e-14)
    v = sim.vortex(with_psi=True)
    psi = dg.stream_function(u, g)
    np.testing.assert_allclose(v["field"], psi, rtol=0, atol=1e-13 * max(1.0, np.max(np.abs(psi))))
    x0, y0, pc = dg.vortex_centre(psi, g.h)
    assert v["centre"][0] == pytest.approx(x0, abs=1e-12)
    assert v["centre"][1] == pytest.approx(y0, abs=1e-12)
    assert v["psi"] == pytest.approx(pc, rel=1e-12)
    sim.close()


def test_steady_and_cessation_drivers_match_oracle():
    from paper_1803_00417_gb300.hbflow import HBFlow

    n, dt, tol = (16, 16), 5e-4, 0.05
    cfg = cavity(n, Re=1.0, Bi=10.0, Pa=400.0, nexp=1.0)
    g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
    rh = Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    zero = [np.zeros(n), np.zeros(n)]
    p0 = np.zeros((17, 17))
    u1, p1, steps, ok = dg.run_to_steady(g, zero, p0, dt, rh, tol=tol, max_steps=300)
    assert ok
    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"])
    sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    sim.set_velocity(zero)
    sim.set_pressure(p0)
    r = sim.run_steady(dt, tol=tol, max_steps=300)
    assert r["reached"] == 1 and r["steps"] == steps
    assert r["t"] == pytest.approx(steps * dt, rel=1e-13)
    uo = [np.asarray(c) for c in u1]
    assert max(np.max(np.abs(a - b)) for a, b in zip(sim.velocity(), uo)) < 1e-10
    # cessation from that state
    _, _, csteps, tc, tci, hist = dg.run_cessation(g, u1, p1, dt, rh, max_steps=600)
    assert np.isfinite(tc)
    rec, us, ps = sim.get_state()
    c = sim.run_cessation(dt, max_steps=600)
    assert c["reached"] == 1 and c["steps"] == csteps
    assert c["t_c"] == pytest.approx(tc, rel=1e-12)
    assert c["t_c_interp"] == pytest.approx(tci, rel=1e-6)
    info = sim.yield_info()
    assert info["yielded"] == 0
    # the same cessation with two backward-Euler steps after the lid stops
    _, _, dsteps, dtc, _, _ = dg.run_cessation(g, u1, p1, dt, rh, max_steps=600, damp_steps=2)
    sim.set_state(rec, us, ps)
    c2 = sim.run_cessation(dt, max_steps=600, damp_steps=2)
    assert c2["reached"] == 1 and c2["steps"] == dsteps
    assert c2["t_c"] == pytest.approx(dtc, rel=1e-12)
    assert sim.get_state(False)[0]["theta"] == 0.5  # restored after the damped steps
    sim.close()
