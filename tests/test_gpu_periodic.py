"""Periodic axes through the C-ABI (hbf_set_periodic) against the oracle, and
the closed-form fixed points of the method that need them.

* stage by stage and over two steps on cavities periodic along x (2D) and
  along x and y (3D), lid on the last axis: explicit stages <= 1e-12, solves
  and steps <= 1e-10 relative L2 (the nodal field repeats node 0 at node n);
* plane Couette flow (periodic along the walls, top wall moving) is an exact
  steady state of the step: u = z stays to 1e-10 and the pressure stays 0;
* Bingham and Herschel-Bulkley plane Poiseuille flow between walls, driven
  by a body force along the periodic axis: six steps from the closed-form
  profile stay within the oracle's tolerance of it (3% and 4%), flat in the
  plug, and equal to the oracle's own six steps to 1e-10.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.grid import Grid  # noqa: E402
from oracle.multigrid import SolverParams  # noqa: E402
from oracle.step import Rheology, step  # noqa: E402
from paper_1803_00417_gb300.inputs import random_state  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_00417_gb300 import build

    build.build()


def rel_l2(a, b):
    a = [np.asarray(x) for x in (a if isinstance(a, (list, tuple)) else [a])]
    b = [np.asarray(x) for x in (b if isinstance(b, (list, tuple)) else [b])]
    num = sum(float(np.sum((x - y) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(y ** 2)) for y in b)
    return np.sqrt(num / den) if den > 0 else np.sqrt(num)


def _periodic_nodes(p, per):
    """Node n := node 0 along every periodic axis."""
    p = p.copy()
    for a, on in enumerate(per):
        if on:
            idx = [slice(None)] * p.ndim
            src = [slice(None)] * p.ndim
            idx[a] = -1
            src[a] = 0
            p[tuple(idx)] = p[tuple(src)]
    return p


def _sim(n, h, wall, per, rh, u, p, f=None):
    from paper_1803_00417_gb300.hbflow import HBFlow

    sim = HBFlow(n, h, wall)
    sim.set_periodic(per)
    sim.set_rheology(rh.K, rh.n, rh.tau_y, rh.m, rh.reg_power)
    if f is not None:
        sim.set_body_force(f)
    sim.set_velocity(u)
    sim.set_pressure(p)
    return sim


@pytest.mark.parametrize("n,per,seed", [((32, 24), (True, False), 91), ((16, 12, 10), (True, True, False), 92)])
def test_periodic_stages_and_steps_match_oracle(n, per, seed):
    d = len(n)
    h = 1.0 / max(n)
    wall = np.zeros((d, 2, d))
    wall[d - 1, 1, 0] = 1.0
    g = Grid(n, h, periodic=per, wall_u=wall)
    rh = Rheology(K=1.0, n=1.0, tau_y=2.0, m=1e4)
    u, p = random_state(n, seed=seed)
    p = _periodic_nodes(p, per)
    dt = 0.5 * h
    sim = _sim(n, h, wall, per, rh, u, p)
    ref = step(g, u, p, dt, rh, keep=True)
    sim.compute_viscosity()
    assert rel_l2(sim.cell_scalar("ETA"), ref.eta) < 1e-13
    sim.predict(dt)
    assert rel_l2(sim.velocity("GP"), ref.Gp) < 1e-12
    assert rel_l2(sim.velocity("LU"), ref.Lu) < 1e-12
    uL, uR = sim.face_field("UL", d), sim.face_field("UR", d)
    for a in range(d):
        assert rel_l2(uL[a], ref.uL[a]) < 1e-12
        assert rel_l2(uR[a], ref.uR[a]) < 1e-12
    st = sim.mac_project()
    assert st["converged"]
    assert rel_l2(sim.cell_scalar("PHI_MAC"), ref.phi_mac) < 1e-10
    umac = sim.face_field("UMAC", 1)
    assert rel_l2([x[0] for x in umac], ref.umac) < 1e-10
    sim.advect_rhs(dt)
    assert rel_l2(sim.velocity("RHS"), ref.rhs) < 1e-10
    sim.set_velocity(u)
    sim.set_pressure(p)
    for _ in range(2):
        ref = step(g, u, p, dt, rh)
        s = sim.step(dt)
        assert all(s[k]["converged"] for k in ("mac", "visc", "nodal"))
        assert rel_l2(sim.velocity(), ref.u) < 1e-10
        assert rel_l2(sim.pressure(), ref.p) < 1e-9
        u, p = ref.u, ref.p
        sim.set_velocity(u)
        sim.set_pressure(p)
    sim.close()


@pytest.mark.parametrize("d", [2, 3])
def test_plane_couette_is_steady(d):
    n = (8,) * d
    h = 1.0 / 8
    wall = np.zeros((d, 2, d))
    wall[d - 1, 1, 0] = 1.0
    per = tuple(a < d - 1 for a in range(d))
    X = np.meshgrid(*[(np.arange(s) + 0.5) * h for s in n], indexing="ij")
    u = [X[d - 1].copy()] + [np.zeros(n) for _ in range(d - 1)]
    p = np.zeros(tuple(s + 1 for s in n))
    rh = Rheology(K=0.7, n=1.0, tau_y=0.0, m=1e4, reg_power=False)
    sim = _sim(n, h, wall, per, rh, u, p)
    sim.set_solver(rtol=1e-12)
    for _ in range(3):
        sim.step(0.05)
    ug = sim.velocity()
    for c in range(d):
        np.testing.assert_allclose(ug[c], u[c], atol=1e-10)
    assert np.max(np.abs(sim.pressure())) < 1e-10
    sim.close()


def _poiseuille(y, K, n, tau, G, H):
    ay = np.abs(y)
    return (n / (n + 1)) * K ** (-1 / n) / G * ((G * H - tau) ** (1 + 1 / n)
                                                 - np.clip(G * ay - tau, 0, None) ** (1 + 1 / n))


@pytest.mark.parametrize("n_idx,tol", [(1.0, 0.03), (0.5, 0.04)])
def test_poiseuille_closed_form(n_idx, tol):
    K, tau, G, m = 1.0, 0.5, 4.0, 1e3
    Nx, Ny = 8, 32
    per = (True, False)
    g = Grid((Nx, Ny), 1.0 / Ny, periodic=per)
    y = (np.arange(Ny) + 0.5) / Ny - 0.5
    ex = _poiseuille(y, K, n_idx, tau, G, 0.5)
    u = [np.tile(ex, (Nx, 1)), np.zeros((Nx, Ny))]
    p = np.zeros((Nx + 1, Ny + 1))
    rh = Rheology(K=K, n=n_idx, tau_y=tau, m=m)
    sim = _sim((Nx, Ny), 1.0 / Ny, np.zeros((2, 2, 2)), per, rh, u, p, f=[G, 0.0])
    uo, po = u, p
    for _ in range(6):
        r = step(g, uo, po, 0.1, rh, f=[G, 0.0])
        uo, po = r.u, r.p
        s = sim.step(0.1)
        assert all(s[k]["converged"] for k in ("mac", "visc", "nodal"))
    ug = sim.velocity()
    assert rel_l2(ug, uo) < 1e-10
    prof = ug[0][0]
    assert np.max(np.abs(prof - ex)) / np.max(ex) < tol
    assert np.max(np.abs(ug[0] - ug[0][:1])) < 1e-9  # x-invariant
    assert np.max(np.abs(ug[1])) < 1e-9
    plug = np.abs(y) < 0.8 * tau / G
    assert np.ptp(prof[plug]) < 0.05 * np.max(prof)
    sim.close()


def test_periodic_axis_needs_an_even_count():
    from paper_1803_00417_gb300.hbflow import HBFlow, HBFlowError

    sim = HBFlow((10, 7), 0.1)
    with pytest.raises(HBFlowError):
        sim.set_periodic((False, True))
    sim.set_periodic((True, False))
    rec = sim.get_state(False)[0]
    assert list(rec["periodic"]) == [1, 0, 0]
    sim.close()
