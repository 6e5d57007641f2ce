"""The colour-split layout of the FP32 finest level of the mixed viscous solve
(the default for 3D walled grids with an even x extent) on the GPU: with and
without it every solve converges to the same FP64 tolerance and the steps
agree to that tolerance (the layouts give the same sweeps and operator bit for
bit; only the summation order of the Krylov dot products differs), with the
previous-increment guess carried across steps and across a change of layout;
the setting rejects values other than 0 and 1."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1803_00417_gb300.inputs import cavity, random_state  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_00417_gb300 import build

    build.build()


def _run(n, seed, layouts, guess=0):
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow

    cfg = cavity(n, Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)
    u, p = random_state(cfg["n"], seed=seed)
    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
    sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    if guess:
        sim.set_visc_guess(guess)
    sim.set_velocity(u)
    sim.set_pressure(p)
    cycles = []
    for on in layouts:
        sim.set_split_layout(on)
        st = sim.step(cfg["dt"])
        for k in ("mac", "visc", "nodal"):
            assert st[k]["converged"], (k, st[k])
            assert st[k]["rnorm"] <= 1e-10 * st[k]["bnorm"]
        cycles.append(st["visc"]["cycles"])
    out = np.concatenate([sim.get_field("U"), sim.get_field("P")])
    sim.close()
    return out, cycles


# even x extents: n0 / 2 even and odd (partial rows of the interior slots),
# ragged y / z, and a grid that coarsens once (30 x 18 x 22 -> 15 x 9 x 11)
@pytest.mark.parametrize("n,seed", [((24, 20, 16), 41), ((30, 18, 22), 42), ((64, 32, 40), 43)])
def test_split_layout_matches_natural(n, seed):
    nat, cn = _run(n, seed, [0, 0, 0])
    spl, cs = _run(n, seed, [1, 1, 1])
    assert np.max(np.abs(spl - nat)) <= 1e-8 * np.max(np.abs(nat)), (cn, cs)


def test_split_layout_with_guess_and_layout_change():
    n, seed = (32, 24, 16), 44
    nat, _ = _run(n, seed, [0, 0, 0, 0], guess=1)
    mixed, _ = _run(n, seed, [1, 1, 0, 1], guess=1)  # the kept increment is dropped at each change
    spl, _ = _run(n, seed, [1, 1, 1, 1], guess=1)
    for other in (mixed, spl):
        assert np.max(np.abs(other - nat)) <= 1e-8 * np.max(np.abs(nat))


def test_split_layout_setting_checked():
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow, HBFlowError

    cfg = cavity((8, 8, 8), Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)
    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
    for bad in (-1, 2, 7):
        with pytest.raises(HBFlowError):
            sim.set_split_layout(bad)
    sim.set_split_layout(0)
    sim.set_split_layout(1)
    sim.close()
