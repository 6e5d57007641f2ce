"""Mixed precision (FP32 smoothing and transfers inside FP64 defect
correction, FP64 residuals, bottom solve and viscosity) against the FP64
oracle: every solve reaches the same 1e-10 relative FP64 residual, and the
velocity stays within 1e-6 relative L2 of the oracle per step."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.grid import Grid  # noqa: E402
from oracle.step import Rheology, step  # noqa: E402
from paper_1803_00417_gb300.inputs import cavity, random_state  # noqa: E402

TOL_MIXED = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_00417_gb300 import build

    build.build()


def rel_l2(a, b):
    num = sum(float(np.sum((x - y) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(y ** 2)) for y in b)
    return np.sqrt(num / den)


@pytest.mark.parametrize("n,seed,over", [
    ((64, 64), 31, dict(Re=1.0, Bi=2.0, Pa=1e4, nexp=1.0)),
    ((48, 32), 32, dict(Re=1000.0, Bi=5.0, Pa=1e5, nexp=0.5)),
    ((16, 16, 16), 33, dict(Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)),
    ((24, 20, 12), 34, dict(Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)),
    # ragged for the thread -> cell maps: rows not a multiple of the 16-row
    # groups on the coarse levels, x extents that leave partial warps
    ((64, 32, 40), 35, dict(Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)),
])
def test_mixed_step_matches_fp64_oracle(n, seed, over):
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow

    cfg = cavity(n, **over)
    u, p = random_state(cfg["n"], seed=seed)
    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
    sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
    rh = Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    for _ in range(2):
        sim.set_velocity(u)
        sim.set_pressure(p)
        ref = step(g, u, p, cfg["dt"], rh)
        st = sim.step(cfg["dt"])
        for k in ("mac", "visc", "nodal"):
            assert st[k]["converged"], (k, st[k])
            assert st[k]["rnorm"] <= 1e-10 * st[k]["bnorm"]
        err = rel_l2(sim.velocity(), ref.u)
        assert err < TOL_MIXED, err
        perr = np.linalg.norm(sim.pressure() - ref.p) / np.linalg.norm(ref.p)
        assert perr < 10 * TOL_MIXED, perr
        u, p = ref.u, ref.p
    sim.close()


def test_mixed_from_rest():
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow

    cfg = cavity((32, 32), Re=1.0, Bi=2.0, Pa=1e4, nexp=1.0)
    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
    sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
    rh = Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    u = [np.zeros(cfg["n"]) for _ in range(2)]
    p = np.zeros(tuple(v + 1 for v in cfg["n"]))
    sim.set_velocity(u)
    sim.set_pressure(p)
    for _ in range(3):
        ref = step(g, u, p, cfg["dt"], rh)
        sim.step(cfg["dt"])
        assert rel_l2(sim.velocity(), ref.u) < TOL_MIXED
        u, p = ref.u, ref.p
        sim.set_velocity(u)
        sim.set_pressure(p)
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [(48, 32), (24, 20, 12)])
def test_fused_tail_matches_level_by_level(precision, n):
    """The fused V-cycle tail (one block over the small levels) performs the
    level-by-level launches' operations in the same order: two steps agree
    to rounding with the tail off, from the default level, from a coarser
    level, and over every level."""
    from paper_1803_00417_gb300.hbflow import HBFlow

    cfg = cavity(n, Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)
    u, p = random_state(cfg["n"], seed=36)
    outs = []
    for cells in (0, 64, 512, 1 << 20):
        sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=precision)
        sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
        sim.set_tail(cells)
        sim.set_velocity(u)
        sim.set_pressure(p)
        for _ in range(2):
            st = sim.step(cfg["dt"])
            assert all(st[k]["converged"] for k in ("mac", "visc", "nodal")), st
        outs.append(np.concatenate([sim.get_field("U"), sim.get_field("P")]))
        sim.close()
    for other in outs[1:]:
        assert np.linalg.norm(other - outs[0]) <= 1e-12 * np.linalg.norm(outs[0])


def test_inner_drop_keeps_the_tolerance():
    """The residual drop of each FP32 BiCGStab pass (hbf_set_inner_drop) only
    changes how the FP64 defect correction gets to its tolerance: with drops
    of 1e-2, 1e-3 (default) and 1e-5 every solve converges and the steps
    agree to the solve tolerance; drops outside [1e-7, 1) are rejected."""
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow, HBFlowError

    cfg = cavity((24, 20, 16), Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)
    u, p = random_state(cfg["n"], seed=37)
    outs = []
    for drop in (1e-3, 1e-2, 1e-5):
        sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
        sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
        sim.set_inner_drop(drop)
        sim.set_velocity(u)
        sim.set_pressure(p)
        for _ in range(2):
            st = sim.step(cfg["dt"])
            assert all(st[k]["converged"] for k in ("mac", "visc", "nodal")), st
        outs.append(sim.get_field("U"))
        if drop == 1e-5:
            for bad in (0.0, 1.0, 1e-9, float("nan")):
                with pytest.raises(HBFlowError):
                    sim.set_inner_drop(bad)
        sim.close()
    for other in outs[1:]:
        assert np.max(np.abs(other - outs[0])) <= 1e-8 * np.max(np.abs(outs[0]))
