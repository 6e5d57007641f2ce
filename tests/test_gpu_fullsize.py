"""The 256^3 3D Herschel-Bulkley cavity at full size, in the launch
configuration bench.py times, from a seeded smooth state.  The CPU oracle
cannot step this grid, so the checks are the ones that hold at any size or
that the oracle computes point by point:

* the viscosity at sampled interior cells against the oracle's rheology on
  the cells' own neighbourhoods (Eqs. 1, 23);
* every solve of the step at its 1e-10 relative residual;
* the MAC-projected face velocity discretely divergence-free to the MAC
  solve's tolerance (the exact projection of reading R13);
* the mixed-precision step within the configured 1e-6 relative L2 of the
  FP64 step (itself pinned to the oracle at small sizes by
  test_gpu_parity.py)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.rheology import viscosity  # noqa: E402
from paper_1803_00417_gb300.inputs import cavity, random_state  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_00417_gb300 import build

    build.build()


@pytest.fixture(scope="module")
def state():
    cfg = cavity("cavity256_3d_hb")
    u, p = random_state(cfg["n"], seed=2024, amp=0.5)
    return cfg, u, p


def _sim(cfg, u, p, precision):
    from paper_1803_00417_gb300.hbflow import HBFlow

    s = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=precision)
    s.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    s.set_solver(rtol=1e-10, max_cycles=200)
    s.set_velocity(u)
    s.set_pressure(p)
    return s


def _mac_divergence(umac, n, h):
    """max |D^MAC u| over the cells, from the axis-major face arrays."""
    n0, n1, n2 = n
    sizes = [(n0 + 1) * n1 * n2, n0 * (n1 + 1) * n2, n0 * n1 * (n2 + 1)]
    fx = umac[:sizes[0]].reshape(n2, n1, n0 + 1)
    fy = umac[sizes[0]:sizes[0] + sizes[1]].reshape(n2, n1 + 1, n0)
    fz = umac[sizes[0] + sizes[1]:].reshape(n2 + 1, n1, n0)
    div = (fx[:, :, 1:] - fx[:, :, :-1]) + (fy[:, 1:, :] - fy[:, :-1, :]) + (fz[1:, :, :] - fz[:-1, :, :])
    return float(np.max(np.abs(div))) / h


def test_full_size_step(state):
    from paper_1803_00417_gb300.hbflow import FP64, MIXED

    cfg, u, p = state
    n, h = cfg["n"], cfg["h"]
    mixed = _sim(cfg, u, p, MIXED)
    st = mixed.step(cfg["dt"])
    for k in ("mac", "visc", "nodal"):
        assert st[k]["converged"] and st[k]["rnorm"] <= 1e-10 * st[k]["bnorm"], (k, st[k])

    # viscosity of u^m at sampled interior cells, point by point
    eta = mixed.get_field("ETA").reshape(n[2], n[1], n[0])
    rng = np.random.default_rng(7)
    idx = rng.integers(1, np.array(n) - 1, size=(400, 3))
    for i, j, k in idx:
        G = np.empty((3, 3))
        for b in range(3):
            for a in range(3):
                lo = [i, j, k]
                hi = [i, j, k]
                lo[a] -= 1
                hi[a] += 1
                G[a, b] = (u[b][tuple(hi)] - u[b][tuple(lo)]) / (2.0 * h)
        Dm = 0.5 * (G + G.T)
        g = np.sqrt(0.5 * np.sum(Dm * Dm))
        ref = float(viscosity(g, cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"]))
        assert abs(eta[k, j, i] - ref) <= 1e-12 * abs(ref), (i, j, k, eta[k, j, i], ref)

    # the MAC projection: D^MAC u^MAC at the MAC solve's tolerance
    umac = mixed.get_field("UMAC")
    uadv = mixed.get_field("UADV")
    d_mac, d_adv = _mac_divergence(umac, n, h), _mac_divergence(uadv, n, h)
    assert d_mac <= 1e-9 * d_adv, (d_mac, d_adv)

    u_mixed = mixed.get_field("U")
    mixed.close()
    ref = _sim(cfg, u, p, FP64)
    st64 = ref.step(cfg["dt"])
    for k in ("mac", "visc", "nodal"):
        assert st64[k]["converged"], (k, st64[k])
    u64 = ref.get_field("U")
    ref.close()
    err = np.linalg.norm(u_mixed - u64) / np.linalg.norm(u64)
    assert err <= 1e-6, err
