"""Failure paths of the C-ABI, driven from the host without harming the GPU.

* A solve capped at one cycle returns HBF_ERR_NOT_CONVERGED and leaves the
  last iterate and filled statistics; that iterate is the oracle's after the
  same single cycle.
* A NaN in the velocity makes the step return HBF_ERR_NONFINITE (its
  residual norms are not finite), and the time-step rule returns NaN.
* A learned initial guess whose weights are noise cannot spoil a solve: the
  guess is kept only if it lowers the warm-start residual, and the solve
  runs to the same tolerance either way.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.grid import Grid  # noqa: E402
from oracle.multigrid import SolverParams  # noqa: E402
from oracle.step import Rheology, step  # noqa: E402
from paper_1803_00417_gb300.inputs import cavity, random_state  # noqa: E402

HBF_ERR_NOT_CONVERGED = -4
HBF_ERR_NONFINITE = -6


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


def _sim(n, seed, precision=0):
    from paper_1803_00417_gb300.hbflow import HBFlow

    cfg = cavity(n, Re=1.0, Bi=2.0, Pa=1e4, nexp=1.0)
    u, p = random_state(cfg["n"], seed=seed)
    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=precision)
    sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    sim.set_velocity(u)
    sim.set_pressure(p)
    return sim, cfg, u, p


@pytest.mark.parametrize("n", [(32, 32), (16, 12, 8)])
def test_one_cycle_cap_returns_not_converged_with_last_iterate(n):
    from paper_1803_00417_gb300.hbflow import StepStats

    sim, cfg, u, p = _sim(n, 61)
    sim.set_solver(rtol=1e-10, max_cycles=1)
    s = StepStats()
    st = sim.lib.hbf_step(sim.ctx, cfg["dt"], ctypes.byref(s))
    assert st == HBF_ERR_NOT_CONVERGED
    assert b"did not converge" in sim.lib.hbf_last_error(sim.ctx)
    stats = s.as_dict()
    for k in ("mac", "visc", "nodal"):
        assert stats[k]["cycles"] <= 1
        assert stats[k]["r0"] > 0.0 and np.isfinite(stats[k]["rnorm"])
    assert not all(stats[k]["converged"] for k in ("mac", "visc", "nodal"))
    # the last iterate is the oracle's after the same single cycle
    g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
    rh = Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    ref = step(g, u, p, cfg["dt"], rh, params=SolverParams(rtol=1e-10, max_cycles=1))
    for k in ("mac", "visc", "nodal"):
        assert stats[k]["converged"] == ref.stats[k].converged
    ug = sim.velocity()
    assert all(np.all(np.isfinite(c)) for c in ug)
    assert rel_l2(ug, ref.u) < 1e-10
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_velocity_returns_nonfinite(precision):
    from paper_1803_00417_gb300.hbflow import HBFlowError, to_device_layout

    sim, cfg, u, p = _sim((16, 16), 62, precision)
    u[1][5, 7] = np.nan
    sim.set_velocity(u)
    assert np.isnan(sim.cfl_dt(0.5))
    with pytest.raises(HBFlowError) as e:
        sim.step(cfg["dt"])
    assert e.value.code == HBF_ERR_NONFINITE
    # the allocation-free time-step rule reports it through a NaN dt
    flat = torch.tensor(to_device_layout(u), device="cuda")
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = sim.lib.hbf_cfl_dt_noalloc(ctypes.c_void_p(flat.data_ptr()), flat.numel(), cfg["h"], 0.5,
                                    ctypes.c_void_p(dt_dev.data_ptr()), None)
    assert st == 0
    torch.cuda.synchronize()
    assert np.isnan(float(dt_dev.item()))
    sim.close()


@pytest.mark.parametrize("n,level", [((48, 48), 0), ((32, 32, 32), 1)])
def test_noise_guess_still_converges_to_the_plain_result(n, level):
    from paper_1803_00417_gb300.hbflow import UNet, set_guess_model

    plain, cfg, u, p = _sim(n, 63)
    guided, _, _, _ = _sim(n, 63)
    e = [v // (2 ** level) + 1 for v in n]
    box = [((v + 7) // 8) * 8 for v in e]
    net = UNet(box, train=False, seed=5)
    rng = np.random.default_rng(9)
    net.set_params((10.0 * rng.normal(size=net.param_count())).astype(np.float32))
    set_guess_model(guided, net, level)
    for _ in range(2):
        s0 = plain.step(cfg["dt"])
        s1 = guided.step(cfg["dt"])
        for k in ("mac", "visc", "nodal"):
            assert s0[k]["converged"] and s1[k]["converged"]
        assert rel_l2(guided.velocity(), plain.velocity()) < 1e-8
    set_guess_model(guided, None)
    net.close()
    plain.close()
    guided.close()
