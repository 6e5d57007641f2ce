"""Flow diagnostics of the paper's start-up, steady-state and cessation study
(Sec. III A steady criterion; Sec. IV yield surfaces, stagnant and plug zones,
cessation time; Sec. IV/V centre-line profiles and vortex centres).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

* ``stress_norm``   |tau| = 2 eta |gamma_dot| at cells (tau = 2 eta gamma_dot,
                    Eq. 4; |.| the scaled norm of Eq. 1).  A cell is unyielded
                    where |tau| <= tau_y (Sec. IV: the yield surface is the
                    contour |tau| = tau_0).
* ``zones``         connected components (cells sharing a face) of the
                    unyielded cells, each classified as stagnant (it touches
                    a wall at rest), plug (it touches no wall) or attached
                    (it touches moving walls only).  Sec. IV: stagnant zones
                    are connected to no-slip walls, plug zones move in the
                    interior and touch no wall.
* ``step_change``   max |u^{m+1} - u^m| / max |u^m|: the steady criterion of
                    Sec. III A, whose pointwise quotient is undefined where
                    u^m = 0, read with the maxima taken separately.
* ``run_to_steady`` / ``run_cessation``  the start-up and cessation study of
                    Sec. IV: step until the change falls below the tolerance;
                    then hold every wall at rest and step until no cell is
                    yielded, t_c = the time since the lid stopped.
* ``centreline``    a velocity component along the line through the box
                    centre parallel to one axis.
* ``stream_function`` / ``vortex_centre``  psi at the nodes of the plane
                    through the centre (2D: the whole box; 3D: normal to y),
                    integrated from the low wall of the last in-plane axis,
                    d psi / d(last axis) = u_first; the primary vortex centre is
                    the extremum of psi with the largest magnitude, refined by
                    a parabola through its neighbours along each axis.
"""

from collections import deque

import numpy as np

from .grid import Grid
from .multigrid import SolverParams
from .rheology import strain_rate_norm, viscosity
from .step import step


def stress_norm(u, grid, rheo):
    """|tau| = 2 eta(g) g at every cell, g = |gamma_dot|."""
    g = strain_rate_norm(u, grid)
    eta = viscosity(g, rheo.K, rheo.n, rheo.tau_y, rheo.m, rheo.reg_power)
    return 2.0 * eta * g


def unyielded(u, grid, rheo):
    return stress_norm(u, grid, rheo) <= rheo.tau_y


def zones(mask, grid):
    """Components of the True cells of ``mask`` (face neighbours), found by
    breadth-first search.  Returns (labels, comps): labels[cell] = component
    index or -1; comps[k] = dict(size, kind) with kind 'stagnant', 'plug' or
    'attached'."""
    d = grid.d
    labels = -np.ones(grid.n, dtype=np.int64)
    comps = []
    for start in zip(*np.nonzero(mask)):
        if labels[start] >= 0:
            continue
        k = len(comps)
        labels[start] = k
        q = deque([start])
        size, rest, moving = 0, False, False
        while q:
            c = q.popleft()
            size += 1
            for a in range(d):
                for s in (-1, 1):
                    nb = list(c)
                    nb[a] += s
                    if nb[a] < 0 or nb[a] >= grid.n[a]:
                        if grid.periodic[a]:
                            nb[a] %= grid.n[a]
                        else:
                            wall = grid.wall_u[a, 0 if s < 0 else 1]
                            if np.any(wall != 0.0):
                                moving = True
                            else:
                                rest = True
                            continue
                    nb = tuple(nb)
                    if mask[nb] and labels[nb] < 0:
                        labels[nb] = k
                        q.append(nb)
        kind = "stagnant" if rest else ("attached" if moving else "plug")
        comps.append(dict(size=size, kind=kind))
    return labels, comps


def step_change(u_new, u_old):
    num = max(float(np.max(np.abs(a - b))) for a, b in zip(u_new, u_old))
    den = max(float(np.max(np.abs(b))) for b in u_old)
    return num / den if den > 0 else np.inf


def run_to_steady(grid, u, p, dt, rheo, tol=1e-5, max_steps=1000, params=None):
    """Step from (u, p) until step_change < tol.  Returns (u, p, steps, reached)."""
    params = params or SolverParams()
    for m in range(1, max_steps + 1):
        r = step(grid, u, p, dt, rheo, params=params)
        ch = step_change(r.u, u)
        u, p = r.u, r.p
        if ch < tol:
            return u, p, m, True
    return u, p, max_steps, False


def resting(grid):
    """The same box with every wall at rest (the lid stopped)."""
    return Grid(grid.n, grid.h, grid.periodic, np.zeros_like(grid.wall_u))


def run_cessation(grid, u, p, dt, rheo, max_steps=1000, params=None, damp_steps=0):
    """Hold every wall at rest and step until max |tau| <= tau_y, the first
    ``damp_steps`` steps with theta = 1 (backward Euler), the rest with the
    Crank-Nicolson weighting.  Returns
    (u, p, steps, t_c, t_c_interp, history of max |tau| / tau_y): t_c is the
    time of the first step at which no cell is yielded, t_c_interp the
    linear interpolation of max |tau| / tau_y = 1 between the last two
    steps."""
    params = params or SolverParams()
    g0 = resting(grid)
    hist = [float(np.max(stress_norm(u, g0, rheo))) / rheo.tau_y]
    if hist[0] <= 1.0:
        return u, p, 0, 0.0, 0.0, hist
    for m in range(1, max_steps + 1):
        r = step(g0, u, p, dt, rheo, params=params, theta=1.0 if m <= damp_steps else 0.5)
        u, p = r.u, r.p
        hist.append(float(np.max(stress_norm(u, g0, rheo))) / rheo.tau_y)
        if hist[-1] <= 1.0:
            a, b = hist[-2], hist[-1]
            frac = (a - 1.0) / (a - b) if a > b else 1.0
            return u, p, m, m * dt, (m - 1 + frac) * dt, hist
    return u, p, max_steps, np.inf, np.inf, hist


def centreline(u, grid, comp, along):
    """u[comp] along axis ``along`` through the box centre: for an even count
    the mean of the two middle cells of each other axis, for an odd one the
    middle cell."""
    a = u[comp]
    for b in reversed(range(grid.d)):
        if b == along:
            continue
        n = grid.n[b]
        if n % 2 == 0:
            a = 0.5 * (np.take(a, n // 2 - 1, axis=b) + np.take(a, n // 2, axis=b))
        else:
            a = np.take(a, n // 2, axis=b)
    return a


def stream_function(u, grid):
    """psi on the nodes of the centre plane.  2D: (n0+1, n1+1) nodes with
    psi(i, 0) = 0 and psi(i, j+1) = psi(i, j) + h u_x(x-face i, cell row j),
    u_x on an x-face the mean of its two cells (0 on the walls normal to x).
    3D: the same in the (x, z) plane normal to y through the centre, with
    u_x averaged over the middle cell layers as in ``centreline``."""
    d, h = grid.d, grid.h
    ux = u[0]
    if d == 3:
        n1 = grid.n[1]
        ux = 0.5 * (ux[:, n1 // 2 - 1, :] + ux[:, n1 // 2, :]) if n1 % 2 == 0 else ux[:, n1 // 2, :]
        na, nb = grid.n[0], grid.n[2]
    else:
        na, nb = grid.n[0], grid.n[1]
    face = np.zeros((na + 1, nb))
    face[1:na] = 0.5 * (ux[:-1] + ux[1:])
    psi = np.zeros((na + 1, nb + 1))
    psi[:, 1:] = h * np.cumsum(face, axis=1)
    return psi


def vortex_centre(psi, h):
    """(x, y) of the extremum of psi with the largest magnitude, refined by a
    parabola through its two neighbours along each axis (node k sits at
    k h), and psi there (the node value)."""
    k = np.unravel_index(int(np.argmax(np.abs(psi))), psi.shape)
    pos = []
    for a in range(2):
        x = k[a] * h
        if 0 < k[a] < psi.shape[a] - 1:
            lo = list(k)
            hi = list(k)
            lo[a] -= 1
            hi[a] += 1
            fm, f0, fp = psi[tuple(lo)], psi[k], psi[tuple(hi)]
            den = fm - 2.0 * f0 + fp
            if den != 0.0:
                x += 0.5 * h * (fm - fp) / den
        pos.append(x)
    return pos[0], pos[1], float(psi[k])
