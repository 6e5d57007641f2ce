"""Discrete operators of the step (Sec. III A), written from their definitions.

* ``tensor_op``      L_eta u = div(eta (grad u + grad u^T)) = div(2 eta gamma_dot)
                     (Eqs. 15-16; the paper writes tau = 2 eta gamma_dot).
* ``cell_grad_nodal`` cell-centred G p from nodal p (Sec. III A: the pressure
                     gradient at cell centres is a finite difference of nodes).
* ``nodal_div``      D of a cell-centred field at nodes (Eq. 17).
* ``nodal_lap``      L: the bilinear/trilinear finite-element Laplacian at
                     nodes, a second-order approximation of div grad (Eq. 17).
* ``mac_div``, ``mac_grad``, ``cell_lap``  the face-based divergence, gradient
                     and their composition for the MAC projection.

Readings (the paper is silent on the stencils):
* face eta is the arithmetic mean of the two cells; a wall face takes the
  interior cell's eta;
* the flux of component c through an a-face is
  eta_f (d_a u_c + d_c u_a): the normal derivative is the two-cell difference,
  the tangential one (c != a) the mean of the two cells' central differences;
  on a wall face the tangential derivative of the wall-normal velocity is that
  of its boundary value, zero;
* nodal operators obey natural (Neumann) conditions at walls: the divergence at
  a wall node sums only interior cells and is normalised by the node's dual
  cell fraction w_n, the Laplacian uses even reflection.
"""

import itertools

import numpy as np

from .grid import pad_cells, pad_nodes, sl, velocity_wall_vals


def _shift(d, axis, lo, hi):
    """Interior slice of a 1-ghost padded array shifted along ``axis``."""
    idx = [slice(1, -1)] * d
    idx[axis] = slice(lo, hi)
    return tuple(idx)


def face_eta(eta, grid, a):
    """eta on faces normal to axis a: mean of the two cells; wall faces take
    the interior value (even reflection of the cell field)."""
    ep = pad_cells(eta, 1, grid, "neumann")
    d = grid.d
    idx_lo = [slice(1, -1)] * d
    idx_hi = [slice(1, -1)] * d
    idx_lo[a] = slice(0, -1)
    idx_hi[a] = slice(1, None)
    return 0.5 * (ep[tuple(idx_lo)] + ep[tuple(idx_hi)])


def tangential_face_derivative(ua_pad, grid, a, c):
    """(d_c u_a) on faces normal to a (c != a): mean of the central c-differences
    in the two cells sharing the face; zero on wall faces (the boundary value of
    the wall-normal velocity does not vary along the wall)."""
    d, h = grid.d, grid.h
    # central c-difference at every cell along a incl. one ghost layer on each side
    lo = [slice(1, -1)] * d
    hi = [slice(1, -1)] * d
    lo[a] = slice(None)
    hi[a] = slice(None)
    lo[c] = slice(0, -2)
    hi[c] = slice(2, None)
    dc = (ua_pad[tuple(hi)] - ua_pad[tuple(lo)]) / (2.0 * h)
    X = 0.5 * (dc[sl(d, a, slice(0, -1))] + dc[sl(d, a, slice(1, None))])
    if not grid.periodic[a]:
        X[sl(d, a, 0)] = 0.0
        X[sl(d, a, grid.n[a])] = 0.0
    return X


def normal_face_difference(uc_pad, grid, a):
    """(u(i+1) - u(i))/h on faces normal to a, from a 1-ghost padded array."""
    d = grid.d
    lo = [slice(1, -1)] * d
    hi = [slice(1, -1)] * d
    lo[a] = slice(0, -1)
    hi[a] = slice(1, None)
    return (uc_pad[tuple(hi)] - uc_pad[tuple(lo)]) / grid.h


def pad_velocity(u, grid, homogeneous=False):
    return [pad_cells(u[c], 1, grid, "dirichlet", velocity_wall_vals(grid, c, homogeneous))
            for c in range(grid.d)]


def face_eta_all(eta, grid):
    return [face_eta(eta, grid, a) for a in range(grid.d)]


def tensor_op(u, eta_f, grid, homogeneous=False):
    """(L_eta u)_c = sum_a [F_ac(i+1/2) - F_ac(i-1/2)] / h,
    F_ac = eta_f (d_a u_c + d_c u_a) on a-faces (for c = a: 2 eta_f d_a u_a).
    ``eta_f[a]`` holds eta on the a-faces."""
    d, h = grid.d, grid.h
    up = pad_velocity(u, grid, homogeneous)
    out = []
    for c in range(d):
        acc = np.zeros(grid.n)
        for a in range(d):
            ef = eta_f[a]
            nrm = normal_face_difference(up[c], grid, a)
            if a == c:
                flux = ef * (2.0 * nrm)
            else:
                flux = ef * (nrm + tangential_face_derivative(up[a], grid, a, c))
            acc += (flux[sl(d, a, slice(1, None))] - flux[sl(d, a, slice(0, -1))]) / h
        out.append(acc)
    return out


def tensor_cross_part(u, eta_f, grid, c, homogeneous=False):
    """The part of (L_eta u)_c that involves the other components only:
    sum_{a != c} [eta_f d_c u_a]^{i+1/2}_{i-1/2} / h."""
    d, h = grid.d, grid.h
    acc = np.zeros(grid.n)
    for a in range(d):
        if a == c:
            continue
        ua = pad_cells(u[a], 1, grid, "dirichlet", velocity_wall_vals(grid, a, homogeneous))
        flux = eta_f[a] * tangential_face_derivative(ua, grid, a, c)
        acc += (flux[sl(d, a, slice(1, None))] - flux[sl(d, a, slice(0, -1))]) / h
    return acc


def cell_grad_nodal(p_unique, grid):
    """G p at cells: along axis a, the mean over the 2^(d-1) node pairs of the
    cell of (p_+ - p_-)/h."""
    d, h = grid.d, grid.h
    pp = pad_nodes(p_unique, grid)  # ghost nodes; periodic wraps
    # full node set 0..n along each axis (index +1 in padded array)
    full = pp[tuple(slice(1, grid.n[a] + 2) for a in range(d))]
    G = []
    for a in range(d):
        g = (full[sl(d, a, slice(1, None))] - full[sl(d, a, slice(0, -1))]) / h
        for b in range(d):
            if b != a:
                g = 0.5 * (g[sl(d, b, slice(0, -1))] + g[sl(d, b, slice(1, None))])
        G.append(g)
    return G


def nodal_div(v, grid, weights):
    """D v at unique nodes: (1 / (w_n 2^(d-1) h)) sum over the existing
    adjacent cells of sum_a s_a v_a, s_a = +1 for a cell on the high side of the
    node along a, -1 on the low side.  Cells outside a wall count as zero
    (impermeable wall, natural boundary condition); periodic axes wrap."""
    d, h = grid.d, grid.h
    acc = np.zeros(grid.node_shape)
    for a in range(d):
        vp = pad_cells(v[a], 1, grid, "zero")  # periodic axes still wrap
        for corner in itertools.product((0, 1), repeat=d):
            # cell at node index + corner - 1 (padded: node index + corner)
            idx = tuple(slice(corner[b], corner[b] + grid.node_shape[b]) for b in range(d))
            s = 1.0 if corner[a] == 1 else -1.0
            acc += s * vp[idx]
    return acc / (weights * (2 ** (d - 1)) * h)


def fe_stencil(d):
    """Coefficients of the FE Laplacian (times h^2) at offsets in {-1,0,1}^d:
    2D: centre -8/3, the 8 neighbours 1/3;  3D: centre -8/3, faces 0, edges
    1/6, corners 1/12."""
    st = {}
    for o in itertools.product((-1, 0, 1), repeat=d):
        k = sum(1 for v in o if v != 0)
        if k == 0:
            st[o] = -8.0 / 3.0
        elif d == 2:
            st[o] = 1.0 / 3.0
        else:
            st[o] = {1: 0.0, 2: 1.0 / 6.0, 3: 1.0 / 12.0}[k]
    return st


def nodal_lap(phi, grid):
    """L phi at unique nodes (strong form, even reflection at walls)."""
    d = grid.d
    pp = pad_nodes(phi, grid)
    st = fe_stencil(d)
    acc = np.zeros(phi.shape)
    for o, w in st.items():
        if w == 0.0:
            continue
        idx = tuple(slice(1 + o[b], 1 + o[b] + phi.shape[b]) for b in range(d))
        acc += w * pp[idx]
    return acc / (grid.h * grid.h)


def mac_div(faces, grid):
    """D^MAC: sum_a (u_a(i+1/2) - u_a(i-1/2)) / h from face-normal velocities."""
    d = grid.d
    acc = np.zeros(grid.n)
    for a in range(d):
        f = faces[a]
        acc += (f[sl(d, a, slice(1, None))] - f[sl(d, a, slice(0, -1))]) / grid.h
    return acc


def mac_grad(phi, grid, a):
    """G^MAC phi on a-faces: (phi(i+1) - phi(i))/h; zero on wall faces (the
    homogeneous Neumann condition of the MAC potential)."""
    pp = pad_cells(phi, 1, grid, "neumann")
    return normal_face_difference(pp, grid, a)


def cell_lap(phi, grid):
    """Cell-centred Laplacian D^MAC G^MAC with homogeneous Neumann walls."""
    return mac_div([mac_grad(phi, grid, a) for a in range(grid.d)], grid)
