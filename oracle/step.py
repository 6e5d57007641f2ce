"""One time step m -> m+1 of the approximate projection method (Sec. III A)
with the regularised Herschel-Bulkley viscosity (Sec. III B).

Order of the step:
 1. eta^m from u^m (Eq. 23).
 2. forcing F = (-G p^{m-1/2} + L_eta u^m + f) / rho at cells (Eq. 12 with
    div tau = L_eta u).
 3. face states u^L, u^R and the advection velocity u^adv (Eqs. 11-14).
 4. MAC projection: D^MAC G^MAC phi = D^MAC u^adv, u^MAC = u^adv - G^MAC phi.
    The paper names u^MAC without spelling this step out; the standard exact
    cell-centred MAC projection is the reading used.
 5. upwinding by u^MAC and the convective term; right-hand side of Eq. 16:
    b = u^m - dt [u^MAC . grad u~] + dt/rho (-G p + 1/2 L_eta u^m + f).
 6. (I - dt/(2 rho) L_eta^m) u* = b, walls at their (constant) velocity
    (Eq. 16; L_eta u = 2 div(eta gamma_dot)), by V-cycle-preconditioned
    BiCGStab (the paper leaves the solver to AMReX).  This is the
    Crank-Nicolson weighting of Eq. 15; ``theta`` generalises it to
    (I - theta dt/rho L_eta) u* = ... + (1 - theta) dt/rho L_eta u^m
    (theta = 1: backward Euler).
 7. nodal projection L phi = rho D(u*/dt + G p^{m-1/2}/rho) (Eq. 17),
    u^{m+1} = u* + dt/rho (G p^{m-1/2} - G phi), p^{m+1/2} = phi.
    Eq. 18 prints u^{m+1} = u* - dt/rho G phi, which is inconsistent with the
    G p term on the right-hand side of Eq. 17; the consistent update is used.
"""

import numpy as np

from .godunov import advective_term, face_states
from .grid import node_weights, nodes_full, nodes_unique, sl
from .multigrid import (CellPoisson, NodalPoisson, SolveStats, SolverParams, TensorViscous,
                        bicgstab_solve, mg_solve)
from .operators import (cell_grad_nodal, face_eta_all, mac_div, mac_grad, nodal_div, tensor_op)
from .rheology import cell_viscosity


class Rheology:
    def __init__(self, K=1.0, n=1.0, tau_y=0.0, m=1e4, reg_power=True):
        self.K = float(K)
        self.n = float(n)
        self.tau_y = float(tau_y)
        self.m = float(m)
        self.reg_power = bool(reg_power)

    @staticmethod
    def from_dimensionless(Re, n, HB, Pa):
        """Sec. IV: rho = U = L = 1 gives K = 2^(1-n)/Re, tau_y = HB/Re, m = Pa."""
        return Rheology(K=2.0 ** (1.0 - n) / Re, n=n, tau_y=HB / Re, m=Pa)


class StepResult:
    pass


def step(grid, u, p, dt, rheo, rho=1.0, f=None, params=None, keep=False, predictor_visc=False, theta=0.5):
    """Advance (u^m, p^{m-1/2}) by dt.  ``u`` is a list of d cell arrays, ``p``
    a nodal array of shape n+1 per axis.  Returns a StepResult with u, p and the
    solve statistics (and every intermediate field when ``keep``)."""
    params = params or SolverParams()
    d = grid.d
    u = [np.asarray(uc, dtype=np.float64) for uc in u]
    f = f if f is not None else [0.0] * d
    res = StepResult()

    eta = cell_viscosity(u, grid, rheo)
    p_u = nodes_unique(np.asarray(p, dtype=np.float64), grid)
    Gp = cell_grad_nodal(p_u, grid)
    Lu = tensor_op(u, face_eta_all(eta, grid), grid)
    F = [(-Gp[c] + (Lu[c] if predictor_visc else 0.0) + f[c]) / rho for c in range(d)]

    uL, uR, uadv = face_states(u, F, grid, dt)

    # MAC projection
    rhs_mac = mac_div(uadv, grid)
    phi_mac, st_mac = mg_solve(CellPoisson(grid), [np.zeros(grid.n)], [rhs_mac], params)
    umac = []
    for a in range(d):
        um = uadv[a] - mac_grad(phi_mac[0], grid, a)
        if not grid.periodic[a]:
            um[sl(d, a, 0)] = 0.0
            um[sl(d, a, grid.n[a])] = 0.0
        umac.append(um)

    A = advective_term(uL, uR, umac, grid)
    wl = 1.0 - theta  # weight of the explicit viscous term (1/2 in Eq. 15)
    rhs = [u[c] - dt * A[c] + (dt / rho) * (-Gp[c] + wl * Lu[c] + f[c]) for c in range(d)]

    beta = dt / (2.0 * rho) if theta == 0.5 else theta * dt / rho
    visc = TensorViscous(grid, eta, beta)
    ustar, st_visc = bicgstab_solve(visc, [uc.copy() for uc in u], rhs, params)

    unew, phi, rhs_nod, st_nod = nodal_project(grid, ustar, p_u, Gp, dt, rho, params)

    res.u = unew
    res.p = nodes_full(phi, grid)
    res.stats = {"mac": st_mac, "visc": st_visc, "nodal": st_nod}
    if keep:
        res.eta, res.Gp, res.Lu, res.F = eta, Gp, Lu, F
        res.uL, res.uR, res.uadv = uL, uR, uadv
        res.rhs_mac, res.phi_mac, res.umac = rhs_mac, phi_mac[0], umac
        res.A, res.rhs, res.ustar = A, rhs, ustar
        res.rhs_nod, res.phi = rhs_nod, phi
    return res


def nodal_project(grid, ustar, p_u, Gp, dt, rho=1.0, params=None):
    """Stage 7 (Eqs. 17-19): solve L phi = rho D(u*/dt + G p/rho) with the
    warm start p, then u^{m+1} = u* + dt/rho (G p - G phi) and p^{m+1/2} = phi.
    ``p_u`` holds the unique nodes of p^{m-1/2}, ``Gp`` its cell gradient.
    Returns (u^{m+1}, phi on the unique nodes, the right-hand side, stats)."""
    params = params or SolverParams()
    d = grid.d
    w = node_weights(grid)
    v = [ustar[c] / dt + Gp[c] / rho for c in range(d)]
    rhs_nod = rho * nodal_div(v, grid, w)
    phi, st_nod = mg_solve(NodalPoisson(grid), [p_u.copy()], [rhs_nod], params)
    Gphi = cell_grad_nodal(phi[0], grid)
    unew = [ustar[c] + (dt / rho) * (Gp[c] - Gphi[c]) for c in range(d)]
    return unew, phi[0], rhs_nod, st_nod


def cfl_dt(grid, u, cfl, u_ref=1.0):
    """dt = cfl h / max(max|u|, u_ref) (the paper is silent on the rule; the
    lid speed bounds it from below at start-up)."""
    umax = max(float(np.max(np.abs(uc))) for uc in u)
    return cfl * grid.h / max(umax, u_ref)
