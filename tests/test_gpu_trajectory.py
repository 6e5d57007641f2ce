"""Trajectories of the configured workloads, not just single steps.

* The 64^2 Bingham cavity (n = 1, Re = 1, Bi = 2, Pa = 1e4, CFL 0.5), 100
  steps from rest: at every step the GPU step taken from the oracle's state
  matches the oracle's step to relative L2 <= 1e-10 (velocity) and relative
  max-norm <= 1e-9, and a GPU trajectory left to run on its own stays within
  1e-9 of the oracle's trajectory over all 100 steps.
* Mixed precision against FP64 over a run of the shear-thinning 2D workload's
  parameters (n = 0.5, Re = 1000, Bi = 5, Pa = 1e5) at 256^2 for 100 steps
  from rest: velocity relative L2 <= 1e-6 at every step.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.grid import Grid  # noqa: E402
from oracle.step import Rheology, step  # noqa: E402
from paper_1803_00417_gb300.inputs import cavity  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_00417_gb300 import build

    build.build()


def rel_l2(a, b):
    num = sum(float(np.sum((np.asarray(x) - np.asarray(y)) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(np.asarray(y) ** 2)) for y in b)
    return np.sqrt(num / den)


def rel_max(a, b):
    num = max(float(np.max(np.abs(np.asarray(x) - np.asarray(y)))) for x, y in zip(a, b))
    den = max(float(np.max(np.abs(np.asarray(y)))) for y in b)
    return num / den


def _ctx(cfg, precision=0):
    from paper_1803_00417_gb300.hbflow import HBFlow

    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=precision)
    sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    d = len(cfg["n"])
    sim.set_velocity([np.zeros(cfg["n"]) for _ in range(d)])
    sim.set_pressure(np.zeros(tuple(v + 1 for v in cfg["n"])))
    return sim


def test_bingham_cavity_100_steps_every_step_against_oracle():
    cfg = cavity("cavity64_bingham")
    g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
    rh = Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    reset = _ctx(cfg)   # restarted from the oracle's state before each step
    free = _ctx(cfg)    # its own trajectory
    u = [np.zeros(cfg["n"]) for _ in range(2)]
    p = np.zeros(tuple(v + 1 for v in cfg["n"]))
    worst = dict(step_l2=0.0, step_max=0.0, p_l2=0.0, free_l2=0.0, free_max=0.0)
    for m in range(100):
        reset.set_velocity(u)
        reset.set_pressure(p)
        ref = step(g, u, p, cfg["dt"], rh)
        s = reset.step(cfg["dt"])
        free.step(cfg["dt"])
        assert all(s[k]["converged"] for k in ("mac", "visc", "nodal"))
        ug = reset.velocity()
        worst["step_l2"] = max(worst["step_l2"], rel_l2(ug, ref.u))
        worst["step_max"] = max(worst["step_max"], rel_max(ug, ref.u))
        worst["p_l2"] = max(worst["p_l2"], rel_l2([reset.pressure()], [ref.p]))
        uf = free.velocity()
        worst["free_l2"] = max(worst["free_l2"], rel_l2(uf, ref.u))
        worst["free_max"] = max(worst["free_max"], rel_max(uf, ref.u))
        u, p = ref.u, ref.p
    print("C1 100 steps, worst over the steps:", worst)
    assert worst["step_l2"] <= 1e-10
    assert worst["step_max"] <= 1e-9
    assert worst["p_l2"] <= 1e-9
    assert worst["free_l2"] <= 1e-9
    assert worst["free_max"] <= 1e-8
    reset.close()
    free.close()


def test_mixed_against_fp64_over_100_steps():
    cfg = cavity((256, 256), nexp=0.5, Re=1000.0, Bi=5.0, Pa=1e5)
    a = _ctx(cfg, precision=0)
    b = _ctx(cfg, precision=1)
    worst = 0.0
    for m in range(100):
        sa = a.step(cfg["dt"])
        sb = b.step(cfg["dt"])
        assert all(sa[k]["converged"] and sb[k]["converged"] for k in ("mac", "visc", "nodal"))
        if m % 10 == 9:
            worst = max(worst, rel_l2(b.velocity(), a.velocity()))
    print("mixed vs FP64, 256^2 HB n=0.5 Re=1000, 100 steps: worst velocity rel-L2", worst)
    assert worst <= 1e-6
    a.close()
    b.close()
