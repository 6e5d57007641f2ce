"""Pins for the oracle's flow diagnostics (Sec. III A steady criterion,
Sec. IV yield surfaces, zones and cessation, centre-line profiles and vortex
centres).

* |tau| in simple shear u_x = s y: the stress of Eq. 23 in closed form,
  (2^n K (s/2)^n + tau_y)(1 - exp(-m s / 2)) (|gamma_dot| = s / 2 in the
  scaled norm), tending to K s^n + tau_y, the textbook shear stress.
* zones of a hand-made mask: stagnant, plug and attached components with
  their sizes, and a component wrapping around a periodic axis.
* the centre line of an x-invariant field is its profile.
* the discrete stream function of u = (d psi/dy, -d psi/dx) converges to psi
  at second order, and the vortex centre to the extremum of psi
  (x^3 (1-x)^2 y^2 (1-y)^3 peaks at (0.6, 0.4)); the same in the centre plane
  of a 3D field.
* the steady criterion holds at once for plane Couette flow, which is an
  exact steady state of the step; a box at rest is unyielded from the start.
"""

import numpy as np
import pytest

from oracle.diagnostics import (centreline, run_cessation, run_to_steady, step_change, stream_function,
                                stress_norm, vortex_centre, zones)
from oracle.grid import Grid
from oracle.step import Rheology


@pytest.mark.parametrize("nexp,reg", [(1.0, True), (0.5, True), (1.5, True), (1.0, False)])
def test_stress_norm_in_simple_shear(nexp, reg):
    s, K, tau, m = 0.8, 0.7, 0.3, 50.0
    N = 8
    wall = np.zeros((2, 2, 2))
    wall[1, 1, 0] = s  # top wall at y = 1 moves with u_x = s
    g = Grid((N, N), 1.0 / N, periodic=(True, False), wall_u=wall)
    y = (np.arange(N) + 0.5) / N
    u = [np.tile(s * y, (N, 1)), np.zeros((N, N))]
    rh = Rheology(K=K, n=nexp, tau_y=tau, m=m, reg_power=reg)
    gd = s / 2.0
    F = 1.0 - np.exp(-m * gd)
    if reg:
        expect = (2.0 ** nexp * K * gd ** nexp + tau) * F
    else:
        expect = 2.0 ** nexp * K * gd ** nexp + tau * F
    np.testing.assert_allclose(stress_norm(u, g, rh), expect, rtol=1e-13)
    # unregularised limit: the shear stress K s^n + tau_y
    rh_inf = Rheology(K=K, n=nexp, tau_y=tau, m=1e12, reg_power=reg)
    np.testing.assert_allclose(stress_norm(u, g, rh_inf), K * s ** nexp + tau, rtol=1e-12)


def test_zones_of_a_hand_made_mask():
    wall = np.zeros((2, 2, 2))
    wall[1, 1, 0] = 1.0  # lid: top wall
    g = Grid((8, 6), 1.0 / 8, wall_u=wall)
    m = np.zeros((8, 6), dtype=bool)
    m[2:5, 0:2] = True   # touches the bottom wall: stagnant, 6 cells
    m[3:5, 3] = True     # interior: plug, 2 cells
    m[6, 5] = True       # touches only the lid: attached, 1 cell
    m[0, 3] = True       # touches the left wall at rest: stagnant, 1 cell
    labels, comps = zones(m, g)
    kinds = sorted((c["kind"], c["size"]) for c in comps)
    assert kinds == [("attached", 1), ("plug", 2), ("stagnant", 1), ("stagnant", 6)]
    assert np.all((labels >= 0) == m)
    # a band across a periodic axis is one component
    gp = Grid((8, 6), 1.0 / 8, periodic=(True, False))
    mp = np.zeros((8, 6), dtype=bool)
    mp[0, 2] = mp[7, 2] = True
    _, cp = zones(mp, gp)
    assert len(cp) == 1 and cp[0]["size"] == 2 and cp[0]["kind"] == "plug"


def test_centreline_of_an_x_invariant_field():
    g = Grid((10, 7), 0.1)
    prof = np.linspace(-1.0, 2.0, 7) ** 3
    u = [np.tile(prof, (10, 1)), np.zeros((10, 7))]
    np.testing.assert_array_equal(centreline(u, g, 0, 1), prof)
    g3 = Grid((6, 4, 5), 0.2)
    u3 = [np.broadcast_to(prof[:5], (6, 4, 5)).copy(), np.zeros((6, 4, 5)), np.zeros((6, 4, 5))]
    np.testing.assert_array_equal(centreline(u3, g3, 0, 2), prof[:5])


def _psi(x, y):
    return -(x ** 3) * (1 - x) ** 2 * y ** 2 * (1 - y) ** 3


def _vel(x, y):
    dpsi_dy = -(x ** 3) * (1 - x) ** 2 * (2 * y * (1 - y) ** 3 - 3 * y ** 2 * (1 - y) ** 2)
    dpsi_dx = -(3 * x ** 2 * (1 - x) ** 2 - 2 * x ** 3 * (1 - x)) * y ** 2 * (1 - y) ** 3
    return dpsi_dy, -dpsi_dx


@pytest.mark.parametrize("d", [2, 3])
def test_stream_function_and_vortex_centre_converge(d):
    errs, cerrs = [], []
    for N in (32, 64, 128):
        h = 1.0 / N
        c = (np.arange(N) + 0.5) * h
        if d == 2:
            X, Y = np.meshgrid(c, c, indexing="ij")
            ux, uy = _vel(X, Y)
            u = [ux, uy]
            g = Grid((N, N), h)
        else:
            X, _, Z = np.meshgrid(c, c[:4], c, indexing="ij")
            ux, uz = _vel(X, Z)
            u = [ux, np.zeros_like(ux), uz]
            g = Grid((N, 4, N), h)
        psi = stream_function(u, g)
        xn = np.arange(N + 1) * h
        XN, YN = np.meshgrid(xn, xn, indexing="ij")
        errs.append(np.max(np.abs(psi - _psi(XN, YN))))
        x0, y0, _ = vortex_centre(psi, h)
        cerrs.append(max(abs(x0 - 0.6), abs(y0 - 0.4)))
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.6, errs
    assert cerrs[-1] < 2e-3 and cerrs[-1] < cerrs[0], cerrs


def test_steady_criterion_and_rest():
    N = 8
    wall = np.zeros((2, 2, 2))
    wall[1, 1, 0] = 1.0
    g = Grid((N, N), 1.0 / N, periodic=(True, False), wall_u=wall)
    y = (np.arange(N) + 0.5) / N
    u = [np.tile(y, (N, 1)), np.zeros((N, N))]
    p = np.zeros((N + 1, N + 1))
    rh = Rheology(K=0.7, n=1.0, tau_y=0.0, m=1e4, reg_power=False)
    _, _, steps, ok = run_to_steady(g, u, p, 0.05, rh, tol=1e-9, max_steps=5)
    assert ok and steps == 1
    assert step_change([np.ones(3)], [np.ones(3)]) == 0.0
    # a Bingham fluid at rest in a resting box is unyielded before any step
    gb = Grid((N, N), 1.0 / N)
    zero = [np.zeros((N, N)), np.zeros((N, N))]
    rb = Rheology(K=1.0, n=1.0, tau_y=2.0, m=1e3)
    out = run_cessation(gb, zero, p, 0.01, rb, max_steps=3)
    assert out[2] == 0 and out[3] == 0.0
