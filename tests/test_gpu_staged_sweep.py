"""The TMA-staged red-black sweeps of the 3D FP32 finest level
(hbf_set_staged_sweep) and the TMA-staged viscous operator
(hbf_set_staged_op) against the unstaged kernels: from the same
seeded states, cavity steps give the same velocity and pressure bit for bit
and the same solver iteration counts (every interior update is the same
arithmetic on the same values; the wall cells take the same global path).
Sizes cover partial tiles in x and y, a last z chunk shorter than the others,
chunks of one plane, both tile widths, and a width that is not a multiple of
4 (the staged sweep is then not taken and the results are trivially equal).
The staged path also matches the FP64 oracle like the rest of the mixed
path."""

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


CASES = [
    ((40, 24, 34), 91, 128, 16),
    ((64, 64, 64), 92, 64, 16),
    ((136, 36, 24), 93, 128, 5),
    ((20, 50, 12), 94, 64, 1),
    ((36, 28, 30), 95, 64, 7),
    ((18, 30, 12), 96, 128, 16),  # 18 % 4 != 0: unstaged
]


@pytest.mark.parametrize("n,seed,tx,tz", CASES)
def test_staged_sweep_matches_unstaged(n, seed, tx, tz):
    _check_staged(n, seed, lambda s: s.set_staged_sweep(tx, tz), f"sweep {tx}x8x{tz}")


OP_CASES = [
    ((40, 24, 34), 101, 4, 16),
    ((64, 64, 64), 102, 8, 16),
    ((136, 36, 24), 103, 8, 5),
    ((20, 50, 12), 104, 4, 1),
    ((36, 28, 30), 105, 4, 7),
    ((18, 30, 12), 106, 8, 16),  # 18 % 4 != 0: unstaged
]


@pytest.mark.parametrize("n,seed,rows,tz", OP_CASES)
def test_staged_operator_matches_unstaged(n, seed, rows, tz):
    _check_staged(n, seed, lambda s: s.set_staged_op(rows, tz), f"operator 64x{rows}x{tz}")


def test_staged_sweep_and_operator_together():
    def both(s):
        s.set_staged_sweep(64, 8)
        s.set_staged_op(8, 8)

    _check_staged((48, 40, 32), 107, both, "sweep and operator")


def _check_staged(n, seed, enable, what):
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow

    cfg = cavity(n, Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)
    u, p = random_state(cfg["n"], seed=seed)
    sims = []
    for staged in (True, False):
        s = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
        s.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
        # the staged forms read the natural layout: so does the reference (the
        # colour-split default sums the Krylov dot products in another order)
        s.set_split_layout(0)
        if staged:
            enable(s)
        s.set_velocity(u)
        s.set_pressure(p)
        sims.append(s)
    for _ in range(2):
        st = [s.step(cfg["dt"]) for s in sims]
        for k in ("mac", "visc", "nodal"):
            assert st[0][k]["cycles"] == st[1][k]["cycles"], (k, st[0][k], st[1][k])
            assert st[0][k]["converged"] and st[1][k]["converged"], (k, st[0][k], st[1][k])
        ua, ub = sims[0].get_field("U"), sims[1].get_field("U")
        pa, pb = sims[0].get_field("P"), sims[1].get_field("P")
        print(f"staged {what} vs unstaged {n}: max |du| {np.max(np.abs(ua - ub)):.3e}")
        assert np.array_equal(ua, ub)
        assert np.array_equal(pa, pb)
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


def test_staged_arguments():
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow, HBFlowError

    cfg = cavity((16, 16, 16), Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)
    s = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
    for bad in ((32, 16), (128, 0), (64, 5000)):
        with pytest.raises(HBFlowError):
            s.set_staged_sweep(*bad)
    for bad in ((6, 16), (4, 0), (8, 5000)):
        with pytest.raises(HBFlowError):
            s.set_staged_op(*bad)
    s.set_staged_sweep(0)
    s.set_staged_op(0)
    s.close()
