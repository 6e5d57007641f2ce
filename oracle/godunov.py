"""Second-order Godunov (BCG-style) edge-state predictor, upwinding and the
advective term (Sec. III A, Eqs. 11-15).

Steps, in the order the paper gives them:

1. Colella's fourth-order monotonicity-limited slope S u along each axis.
2. Transverse terms (v du/dy)^ by "a separate extrapolation and upwinding":
   pre-states extrapolated in space and time along the transverse axis with the
   slope only, upwinded, then (mean normal velocity) x (difference of the
   upwinded states) / h.
3. Left/right face states (Eq. 14a-b) for all components, with the time
   derivative replaced through the momentum equation: normal term, transverse
   terms and the forcing (-G p + div tau + f)/rho.
4. A face advection velocity u^adv from the normal component by the Riemann
   rule, the MAC projection of it (``mac`` in ``step``), upwinding of all
   components with u^MAC, and the convective term [u^MAC . grad u~].

Readings where the text is silent or garbled:
* Eq. 14b prints "+ u dt/2" inside the right-state slope factor and Eq. 14a/b
  put the forcing inside -(dt/2rho)(...); the Taylor-consistent forms are used:
  u^R = u_{i+1} - (1/2 + u_{i+1} dt/(2h)) slope_{i+1} ...,  + (dt/2) F;
* Riemann rule: u^L if u^L > 0 and u^L + u^R > 0; u^R if u^R < 0 and
  u^L + u^R < 0; else 0.  Tangential components follow the sign of that
  normal velocity, taking the mean of L and R when it is exactly zero;
* on a wall face both states equal the wall velocity.
"""

import numpy as np

from .grid import pad_cells, sl, velocity_wall_vals


def limited_slopes(uc, grid, a, wall_vals):
    """Colella (1985) fourth-order limited slope along axis a (per-cell
    increment; S u = slope / h).  Two wall ghost layers are used."""
    d = grid.d
    up = pad_cells(uc, 2, grid, "dirichlet", wall_vals)
    n = grid.n[a]
    inner = [slice(2, -2)] * d

    def along(lo, hi):
        idx = list(inner)
        idx[a] = slice(lo, hi)
        return up[tuple(idx)]

    # quantities on padded positions 1..n+2 (cells -1..n)
    um = along(0, n + 2)
    u0 = along(1, n + 3)
    upl = along(2, n + 4)
    dL = u0 - um
    dR = upl - u0
    dC = 0.5 * (upl - um)
    dlim = np.where(dL * dR > 0.0, 2.0 * np.minimum(np.abs(dL), np.abs(dR)), 0.0)
    df = np.sign(dC) * np.minimum(np.abs(dC), dlim)
    # fourth-order slope on cells 0..n-1 (positions 1..n of these arrays)
    c = sl(d, a, slice(1, n + 1))
    d4 = (4.0 / 3.0) * dC[c] - (1.0 / 6.0) * (df[sl(d, a, slice(2, n + 2))] + df[sl(d, a, slice(0, n))])
    return np.sign(d4) * np.minimum(np.abs(d4), dlim[c])


def riemann(uL, uR):
    """Upwind normal velocity from left/right normal states."""
    s = uL + uR
    return np.where((uL > 0.0) & (s > 0.0), uL, np.where((uR < 0.0) & (s < 0.0), uR, 0.0))


def upwind(uL, uR, vel):
    """State selected by the sign of the face velocity (mean when zero)."""
    return np.where(vel > 0.0, uL, np.where(vel < 0.0, uR, 0.5 * (uL + uR)))


def _cells_to_faces_lr(q, grid, a):
    """Left (cell i-1) and right (cell i) values of a cell array on the a-faces
    0..n_a.  Outside-of-domain entries (wall faces) are filled with NaN and must
    be overwritten by the caller; periodic axes wrap."""
    d = grid.d
    n = grid.n[a]
    if grid.periodic[a]:
        left = np.concatenate([q[sl(d, a, slice(n - 1, n))], q], axis=a)
        right = np.concatenate([q, q[sl(d, a, slice(0, 1))]], axis=a)
    else:
        nanslab = np.full_like(q[sl(d, a, slice(0, 1))], np.nan)
        left = np.concatenate([nanslab, q], axis=a)
        right = np.concatenate([q, nanslab], axis=a)
    return left, right


def _set_walls(arr, grid, a, lo_val, hi_val):
    if not grid.periodic[a]:
        arr[sl(grid.d, a, 0)] = lo_val
        arr[sl(grid.d, a, grid.n[a])] = hi_val
    return arr


def face_states(u, F, grid, dt):
    """Left/right states of every component on every face (Eq. 14) and the
    upwinded normal advection velocity u^adv.

    Returns (uL, uR, uadv) with uL[a][c], uR[a][c] of face shape along a and
    uadv[a] the normal component on a-faces."""
    d, h = grid.d, grid.h
    slopes = [[limited_slopes(u[c], grid, a, velocity_wall_vals(grid, c)) for c in range(d)]
              for a in range(d)]  # slopes[a][c]

    # --- transverse terms from pre-states (slope-only extrapolation) ---
    hats = [[None] * d for _ in range(d)]  # hats[b][c] = (u_b d_b u_c)^ at cells
    for b in range(d):
        fac_L = 0.5 - u[b] * dt / (2.0 * h)
        fac_R = 0.5 + u[b] * dt / (2.0 * h)
        pL, pR = [], []
        for c in range(d):
            ext_L = u[c] + fac_L * slopes[b][c]
            ext_R = u[c] - fac_R * slopes[b][c]
            L, _ = _cells_to_faces_lr(ext_L, grid, b)
            _, R = _cells_to_faces_lr(ext_R, grid, b)
            wl, wh = grid.wall_u[b, 0, c], grid.wall_u[b, 1, c]
            pL.append(_set_walls(L, grid, b, wl, wh))
            pR.append(_set_walls(R, grid, b, wl, wh))
        vb = riemann(pL[b], pR[b])
        for c in range(d):
            st = vb if c == b else upwind(pL[c], pR[c], vb)
            lo = sl(d, b, slice(0, -1))
            hi = sl(d, b, slice(1, None))
            hats[b][c] = 0.5 * (vb[hi] + vb[lo]) * (st[hi] - st[lo]) / h

    # --- full traces along each axis ---
    uL = [[None] * d for _ in range(d)]
    uR = [[None] * d for _ in range(d)]
    uadv = []
    for a in range(d):
        fac_L = 0.5 - u[a] * dt / (2.0 * h)
        fac_R = 0.5 + u[a] * dt / (2.0 * h)
        for c in range(d):
            trans = np.zeros(grid.n)
            for b in range(d):
                if b != a:
                    trans += hats[b][c]
            common = -0.5 * dt * trans + 0.5 * dt * F[c]
            ext_L = u[c] + fac_L * slopes[a][c] + common
            ext_R = u[c] - fac_R * slopes[a][c] + common
            L, _ = _cells_to_faces_lr(ext_L, grid, a)
            _, R = _cells_to_faces_lr(ext_R, grid, a)
            wl, wh = grid.wall_u[a, 0, c], grid.wall_u[a, 1, c]
            uL[a][c] = _set_walls(L, grid, a, wl, wh)
            uR[a][c] = _set_walls(R, grid, a, wl, wh)
        ua = riemann(uL[a][a], uR[a][a])
        uadv.append(_set_walls(ua, grid, a, 0.0, 0.0))
    return uL, uR, uadv


def advective_term(uL, uR, umac, grid):
    """[u^MAC . grad u~]_c = sum_a (mean of u^MAC_a on the two a-faces)
    (u~_c(i+1/2) - u~_c(i-1/2)) / h, with u~ upwinded by u^MAC."""
    d, h = grid.d, grid.h
    A = [np.zeros(grid.n) for _ in range(d)]
    for a in range(d):
        lo = sl(d, a, slice(0, -1))
        hi = sl(d, a, slice(1, None))
        vbar = 0.5 * (umac[a][hi] + umac[a][lo])
        for c in range(d):
            ut = upwind(uL[a][c], uR[a][c], umac[a])
            A[c] += vbar * (ut[hi] - ut[lo]) / h
    return A
