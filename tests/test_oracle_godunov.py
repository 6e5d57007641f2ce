"""Pins for the oracle's Godunov predictor (Sec. III A, Eqs. 11-14).

* Colella's limited slope is fourth-order accurate where the limiter is
  inactive: on smooth monotone data the slope converges to h u' at O(h^4)
  (Sec. III A names the fourth-order slope S).  A wrong weight on the limited
  neighbour slopes leaves an O(1) error.
* The limiter introduces no new extrema: the extrapolated face values
  u_i +- slope_i / 2 lie between the neighbouring cell values (TVD).
* The full predictor with its transverse terms is second-order accurate
  (Sec. III A: the approximate projection method is second order): a field
  that does not vary along z and is carried by a uniform oblique velocity
  (U, V, w(x, y)) is a passive scalar w translated by (U, V).  Along every
  axis the face states of w need the transverse term of the other axis, so
  a wrong transverse term (or a wrong slope) drops the convergence of the
  translated w to first order.
"""

import math

import numpy as np
import pytest

from oracle.grid import Grid
from oracle.godunov import limited_slopes
from oracle.multigrid import SolverParams
from oracle.step import Rheology, step


def _centres(n, h):
    return (np.arange(n) + 0.5) * h


@pytest.mark.parametrize("axis", [0, 1])
def test_limited_slope_is_fourth_order_on_smooth_monotone_data(axis):
    errs = []
    for n in (16, 32, 64, 128):
        h = 1.0 / n
        shape = [4, 4]
        shape[axis] = n
        g = Grid(tuple(shape), h)
        x = _centres(n, h)
        prof = np.exp(x) + 0.25 * x * x  # increasing, no inflection in [0, 1]
        dprof = np.exp(x) + 0.5 * x
        u = np.broadcast_to(prof.reshape([-1 if a == axis else 1 for a in range(2)]), shape).copy()
        s = limited_slopes(u, g, axis, [[0.0, 0.0], [0.0, 0.0]])
        # three cells from each wall the stencil sees no ghost
        inner = [slice(None)] * 2
        inner[axis] = slice(3, n - 3)
        ref = np.broadcast_to(dprof.reshape([-1 if a == axis else 1 for a in range(2)]), shape)
        errs.append(np.max(np.abs(s[tuple(inner)] / h - ref[tuple(inner)])))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert errs[-1] < 1e-8
    assert min(orders) > 3.7, orders


def test_limited_slope_creates_no_new_extrema():
    rng = np.random.default_rng(5)
    n = 40
    g = Grid((n, 4), 1.0 / n)
    # steps, plateaus and noise: every kind of data the limiter must tame
    prof = np.where(np.arange(n) < n // 2, 1.0, -0.5) + 0.3 * (np.arange(n) > 30)
    prof = prof + 0.05 * rng.normal(size=n) * (np.arange(n) % 7 == 0)
    u = np.tile(prof[:, None], (1, 4))
    s = limited_slopes(u, g, 0, [[0.0, 0.0], [0.0, 0.0]])[:, 0]
    for i in range(1, n - 1):
        lo = min(prof[i - 1], prof[i], prof[i + 1])
        hi = max(prof[i - 1], prof[i], prof[i + 1])
        for face in (prof[i] - 0.5 * s[i], prof[i] + 0.5 * s[i]):
            assert lo - 1e-15 <= face <= hi + 1e-15
        # a local extremum gets a zero slope
        if (prof[i] - prof[i - 1]) * (prof[i + 1] - prof[i]) <= 0.0:
            assert s[i] == 0.0


def _translate_error(n, T=0.25, U=1.0, V=0.5):
    """Mean absolute error of w after time T against its exact translation."""
    h = 1.0 / n
    nz = 4
    g = Grid((n, n, nz), h, periodic=(True, True, True))
    X, Y, _ = np.meshgrid(_centres(n, h), _centres(n, h), _centres(nz, h), indexing="ij")

    def w0(x, y):
        return 0.5 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)

    u = [np.full(X.shape, U), np.full(X.shape, V), w0(X, Y)]
    p = np.zeros((n + 1, n + 1, nz + 1))
    # eta = 0: the viscous operator is the identity, so one smoothing sweep
    # per level solves it exactly and the solves stay cheap
    rh = Rheology(K=0.0, n=1.0, tau_y=0.0, m=1.0)
    prm = SolverParams(nu1=1, nu2=1, nu_bottom=1)
    dt = 0.5 * h  # Courant numbers 0.5 and 0.25
    for _ in range(int(round(T / dt))):
        r = step(g, u, p, dt, rh, params=prm)
        u, p = r.u, r.p
    # the carrier velocity is reproduced exactly
    assert np.max(np.abs(u[0] - U)) == 0.0 and np.max(np.abs(u[1] - V)) == 0.0
    return float(np.mean(np.abs(u[2] - w0(X - U * T, Y - V * T))))


def test_oblique_translation_is_second_order():
    e16, e32, e64 = (_translate_error(n) for n in (16, 32, 64))
    o1, o2 = math.log2(e16 / e32), math.log2(e32 / e64)
    assert o1 > 1.8 and o2 > 1.8, (e16, e32, e64)
