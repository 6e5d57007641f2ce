"""The one-launch red-black sweep of the 3D FP32 finest level
(hbf_set_fused_sweep) against the default two-launch red/black sweeps: the same cavity steps
from the same seeded states agree to the mixed-precision tolerance (the
per-cell updates are the same arithmetic; the sweep order is the same), on
sizes that are not multiples of the tile (32 x 16 x 16) and on a full tile
grid, with the same solver iteration counts; and the fused path matches the
FP64 oracle like the rest of the mixed path."""

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
    num = max(float(np.max(np.abs(np.asarray(x) - np.asarray(y)))) for x, y in zip(a, b))
    return num / max(float(np.max(np.abs(np.asarray(y)))) for y in b)


@pytest.mark.parametrize("n,seed", [((40, 24, 34), 81), ((64, 64, 64), 82), ((18, 50, 12), 83)])
def test_fused_sweep_matches_two_launch_sweeps(n, seed):
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow

    cfg = cavity(n, Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)
    u, p = random_state(cfg["n"], seed=seed)
    sims = []
    for fused in (True, False):
        s = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
        s.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
        s.set_fused_sweep(fused)
        s.set_velocity(u)
        s.set_pressure(p)
        sims.append(s)
    worst = 0.0
    for _ in range(2):
        st = [s.step(cfg["dt"]) for s in sims]
        for k in ("mac", "visc", "nodal"):
            assert st[0][k]["converged"] and st[1][k]["converged"]
        assert abs(st[0]["visc"]["cycles"] - st[1]["visc"]["cycles"]) <= 1
        worst = max(worst, rel(sims[0].velocity(), sims[1].velocity()))
    print(f"fused vs two-launch sweeps {n}: max relative difference {worst:.3e}")
    assert worst < 1e-6
    g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
    rh = Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    ref = step(g, u, p, cfg["dt"], rh)
    sims[0].set_velocity(u)
    sims[0].set_pressure(p)
    sims[0].step(cfg["dt"])
    ug = sims[0].velocity()
    num = sum(float(np.sum((a - b) ** 2)) for a, b in zip(ug, ref.u))
    den = sum(float(np.sum(b ** 2)) for b in ref.u)
    assert np.sqrt(num / den) < 1e-6
    for s in sims:
        s.close()
