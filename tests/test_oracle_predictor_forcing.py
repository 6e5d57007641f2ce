"""Evidence for leaving the stress divergence out of the edge-state forcing
by default (Sec. III A, Eq. 14).

Eq. 14 extrapolates the face states with the explicit forcing
(-G p + div tau)/rho.  With the regularised viscosity, eta reaches
tau_y m / 2 where the strain rate vanishes, so the explicit stress term in
the extrapolation carries dt eta / h^2 >> 1 and the step is unstable at the
configured time step: on the 32^2 Bingham cavity (n = 1, Re = 1, Bi = 2,
Pa = 1e4, the 64^2 workload's parameters) at CFL 0.5 the paper's form blows
up within a few steps, while at CFL 0.2 it stays bounded and within a few
per cent of the form without the term, the difference falling with dt.
The stress still enters the step through the semi-implicit solve of Eq. 16.
"""

import numpy as np

from oracle.grid import Grid
from oracle.step import Rheology, step
from paper_1803_00417_gb300.inputs import cavity


def _run(cfl, nsteps):
    cfg = cavity((32, 32), Re=1.0, Bi=2.0, Pa=1e4, nexp=1.0, cfl=cfl)
    g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
    rh = Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    zero = [np.zeros(cfg["n"]) for _ in range(2)]
    p0 = np.zeros((33, 33))
    u, p, ub, pb = zero, p0, zero, p0
    umax, diff = [], []
    for _ in range(nsteps):
        r = step(g, u, p, cfg["dt"], rh, predictor_visc=True)
        rb = step(g, ub, pb, cfg["dt"], rh)
        u, p, ub, pb = r.u, r.p, rb.u, rb.p
        umax.append(max(float(np.max(np.abs(c))) for c in u))
        if not np.isfinite(umax[-1]) or umax[-1] > 1e6:
            break
        num = sum(float(np.sum((a - b) ** 2)) for a, b in zip(u, ub))
        diff.append(np.sqrt(num / sum(float(np.sum(b ** 2)) for b in ub)))
    return umax, diff


def test_paper_form_forcing_blows_up_at_cfl_half():
    umax, _ = _run(0.5, 10)
    assert max(umax) > 1e3  # the lid speed is 1


def test_paper_form_forcing_is_bounded_at_small_dt():
    umax2, diff2 = _run(0.2, 12)
    umax1, diff1 = _run(0.1, 12)
    assert max(umax2) < 1.5 and max(umax1) < 1.5  # of the order of the lid speed
    assert max(diff2) < 0.05
    assert max(diff1) < 0.5 * max(diff2)  # the difference shrinks with dt
