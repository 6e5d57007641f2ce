"""Pins for the oracle's full time step (Sec. III A + B).

Fixed points of the method: plane Couette flow (exact steady state of the
discrete scheme), Bingham and Herschel-Bulkley plane Poiseuille flow (textbook
closed forms, derived from Eqs. 9-10 for a parallel shear flow), exact
translation by one cell at Courant number 1, mirror symmetry of the cavity,
rest state, and the discrete divergence-free MAC velocity."""

import numpy as np
import pytest

from oracle.grid import Grid
from oracle.multigrid import SolverParams
from oracle.operators import mac_div
from oracle.step import Rheology, step


def _centres(n, h):
    return np.meshgrid(*[(np.arange(s) + 0.5) * h for s in n], indexing="ij")


@pytest.mark.parametrize("d", [2, 3])
def test_plane_couette_is_steady(d):
    # periodic in the flow-normal-to-wall-free directions, walls on the last
    # axis, top wall moving with speed 1: u_x = z is the exact steady state
    n = (8,) * d
    h = 1.0 / 8
    wall = np.zeros((d, 2, d))
    wall[d - 1, 1, 0] = 1.0
    g = Grid(n, h, periodic=tuple(a < d - 1 for a in range(d)), wall_u=wall)
    X = _centres(n, h)
    u = [X[d - 1].copy()] + [np.zeros(n) for _ in range(d - 1)]
    p = np.zeros(tuple(s + 1 for s in n))
    rh = Rheology(K=0.7, n=1.0, tau_y=0.0, m=1e4, reg_power=False)
    r = step(g, u, p, 0.05, rh, params=SolverParams(rtol=1e-12))
    for c in range(d):
        np.testing.assert_allclose(r.u[c], u[c], atol=1e-10)
    assert np.max(np.abs(r.p)) < 1e-10


def _poiseuille(y, K, n, tau, G, H):
    """u(y) for |tau_xy| = K |u'|^n + tau_y = G |y| (plug for |y| < tau_y/G)."""
    ay = np.abs(y)
    return (n / (n + 1)) * K ** (-1 / n) / G * ((G * H - tau) ** (1 + 1 / n)
                                                 - np.clip(G * ay - tau, 0, None) ** (1 + 1 / n))


@pytest.mark.parametrize("n_idx,tol", [(1.0, 0.03), (0.5, 0.04)])
def test_poiseuille_closed_form(n_idx, tol):
    # Bingham (n=1) and Herschel-Bulkley (n=0.5) channel between walls at
    # y = 0, 1 driven by a body force G along the periodic x axis.  The
    # regularised (m = 1e3), discretised (32 cells) steady profile stays within
    # a few per cent of the exact one and the plug |y - 1/2| < tau_y/G is flat.
    K, tau, G, m = 1.0, 0.5, 4.0, 1e3
    Nx, Ny = 8, 32
    g = Grid((Nx, Ny), 1.0 / Ny, periodic=(True, False))
    y = (np.arange(Ny) + 0.5) / Ny - 0.5
    ex = _poiseuille(y, K, n_idx, tau, G, 0.5)
    u = [np.tile(ex, (Nx, 1)), np.zeros((Nx, Ny))]
    p = np.zeros((Nx + 1, Ny + 1))
    rh = Rheology(K=K, n=n_idx, tau_y=tau, m=m)
    for _ in range(6):
        r = step(g, u, p, 0.1, rh, f=[G, 0.0])
        u, p = r.u, r.p
    assert np.max(np.abs(u[0][0] - ex)) / np.max(ex) < tol
    assert np.max(np.abs(u[0] - u[0][:1])) < 1e-9  # x-invariant
    assert np.max(np.abs(u[1])) < 1e-9
    plug = np.abs(y) < 0.8 * tau / G
    prof = u[0][0]
    assert np.ptp(prof[plug]) < 0.05 * np.max(prof)
    # regularisation: viscosity stays bounded by tau_y m / 2 in the plug
    # (checked through the profile being finite and monotone away from it)
    upper = y > tau / G
    assert np.all(np.diff(prof[upper]) < 0)


def test_translation_at_unit_courant_number_is_exact():
    # u = (1, v(x)) on a doubly periodic box with eta = 0: divergence-free, so
    # both projections are inert and the step is pure advection of v.  At
    # U dt = h the slope factor (1/2 - U dt/(2h)) vanishes, the upwind state is
    # the left cell value and v moves exactly one cell.
    N = 8
    h = 1.0 / N
    g = Grid((N, N), h, periodic=(True, True))
    rng = np.random.default_rng(7)
    v = np.tile(rng.normal(size=(N, 1)), (1, N))
    u = [np.ones((N, N)), v]
    p = np.zeros((N + 1, N + 1))
    rh = Rheology(K=0.0, n=1.0, tau_y=0.0, m=1.0)
    r = step(g, u, p, h, rh)
    np.testing.assert_allclose(r.u[1], np.roll(v, 1, axis=0), atol=1e-13)
    np.testing.assert_allclose(r.u[0], 1.0, atol=1e-13)


def test_cavity_mirror_symmetry():
    # reversing the lid and mirroring x maps solutions onto solutions:
    # u_x(x) -> -u_x(1-x), u_y(x) -> u_y(1-x), p(x) -> p(1-x)
    from paper_1803_00417_gb300.inputs import random_state
    N = 16
    wall = np.zeros((2, 2, 2))
    wall[1, 1, 0] = 1.0
    wall_m = -wall
    u, p = random_state((N, N), seed=3, amp=0.5)
    um = [-u[0][::-1, :], u[1][::-1, :]]
    pm = p[::-1, :]
    rh = Rheology(K=0.05, n=0.7, tau_y=0.2, m=1e3)
    prm = SolverParams(rtol=1e-13)
    r1 = step(Grid((N, N), 1.0 / N, wall_u=wall), u, p, 0.02, rh, params=prm)
    r2 = step(Grid((N, N), 1.0 / N, wall_u=wall_m), um, pm, 0.02, rh, params=prm)
    np.testing.assert_allclose(-r2.u[0][::-1, :], r1.u[0], atol=1e-10)
    np.testing.assert_allclose(r2.u[1][::-1, :], r1.u[1], atol=1e-10)
    np.testing.assert_allclose(r2.p[::-1, :], r1.p, atol=1e-9 * max(1.0, np.max(np.abs(r1.p))))


@pytest.mark.parametrize("d", [2, 3])
def test_rest_state_and_mac_divergence(d):
    n = (8,) * d
    g0 = Grid(n, 1.0 / 8)
    rh = Rheology(K=1.0, n=1.0, tau_y=1.0, m=1e3)
    zero = [np.zeros(n) for _ in range(d)]
    r = step(g0, zero, np.zeros(tuple(s + 1 for s in n)), 0.05, rh)
    assert all(np.all(c == 0.0) for c in r.u) and np.all(r.p == 0.0)
    # a moving state: the MAC velocity is discretely divergence-free
    from paper_1803_00417_gb300.inputs import random_state
    wall = np.zeros((d, 2, d))
    wall[d - 1, 1, 0] = 1.0
    g = Grid(n, 1.0 / 8, wall_u=wall)
    u, p = random_state(n, seed=11)
    r = step(g, u, p, 0.05, rh, keep=True)
    div_adv = np.max(np.abs(mac_div(r.uadv, g)))
    div_mac = np.max(np.abs(mac_div(r.umac, g)))
    assert div_adv > 1e-3 and div_mac <= 1e-9 * div_adv


@pytest.mark.parametrize("theta", [0.5, 0.75, 1.0])
def test_viscous_decay_of_a_shear_wave_has_the_theta_amplification(theta):
    # u = (0, v(x)) with v = sin(2 pi k x) on a doubly periodic box and a
    # constant viscosity: divergence-free, no advection (u_x = 0, v does not
    # vary along y), no pressure.  The step is the viscous solve alone, whose
    # discrete operator acts on the mode by -nu 4 sin^2(pi k h) / h^2, so one
    # step multiplies v by R(z) = (1 - (1 - theta) z) / (1 + theta z),
    # z = dt nu 4 sin^2(pi k h) / h^2 (the theta-scheme's amplification).
    N, k, nu, dt = 16, 3, 0.8, 0.05
    h = 1.0 / N
    g = Grid((N, N), h, periodic=(True, True))
    x = (np.arange(N) + 0.5) * h
    v = np.tile(np.sin(2 * np.pi * k * x)[:, None], (1, N))
    u = [np.zeros((N, N)), v]
    p = np.zeros((N + 1, N + 1))
    rh = Rheology(K=nu, n=1.0, tau_y=0.0, m=1e4, reg_power=False)
    r = step(g, u, p, dt, rh, params=SolverParams(rtol=1e-13), theta=theta)
    z = dt * nu * 4.0 * np.sin(np.pi * k * h) ** 2 / h ** 2
    R = (1.0 - (1.0 - theta) * z) / (1.0 + theta * z)
    np.testing.assert_allclose(r.u[1], R * v, atol=1e-11)
    np.testing.assert_allclose(r.u[0], 0.0, atol=1e-12)
    # Crank-Nicolson keeps this stiff mode flipping sign with |R| near 1,
    # backward Euler damps it
    if theta == 0.5:
        assert R < -0.5
    if theta == 1.0:
        assert 0.0 < R < 0.1
