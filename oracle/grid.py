"""Uniform grid, boundary ghosts and colourings for the oracle.

The paper leaves boundary treatment aside (Sec. III A: initialisation and
boundary treatments are ignored there).  The readings used here are:

* walls are no-slip with a prescribed wall velocity (the lid of the cavity in
  Sec. IV); a cell-centred ghost across a wall is the odd reflection
  ``g = 2 u_b - u_mirror`` (second ghost layer mirrors the second interior cell);
* a periodic axis wraps;
* ghosts are filled axis by axis, x then y then z (later fills overwrite
  corners);
* scalar potentials (MAC phi, nodal phi) obey homogeneous Neumann conditions at
  walls, i.e. even reflection.
"""

import numpy as np


class Grid:
    """A box of ``n[a]`` cells of side ``h`` along each axis ``a``.

    ``periodic[a]`` selects a periodic axis; otherwise both ends are walls.
    ``wall_u[a][s][c]`` is component ``c`` of the wall velocity on the low
    (``s=0``) or high (``s=1``) wall normal to axis ``a``; its normal component
    must be zero (impermeable walls).
    """

    def __init__(self, n, h, periodic=None, wall_u=None):
        self.n = tuple(int(v) for v in n)
        self.d = len(self.n)
        assert self.d in (2, 3)
        self.h = float(h)
        self.periodic = tuple(bool(p) for p in (periodic or [False] * self.d))
        if wall_u is None:
            wall_u = np.zeros((self.d, 2, self.d))
        self.wall_u = np.asarray(wall_u, dtype=np.float64).reshape(self.d, 2, self.d)
        for a in range(self.d):
            if self.periodic[a]:
                assert self.n[a] % 2 == 0, "periodic axes need an even cell count"
            assert self.wall_u[a, 0, a] == 0.0 and self.wall_u[a, 1, a] == 0.0

    # ---- shapes -----------------------------------------------------------------
    @property
    def cell_shape(self):
        return self.n

    @property
    def node_shape(self):
        """Unique nodes: ``n+1`` along a wall axis, ``n`` along a periodic axis."""
        return tuple(self.n[a] if self.periodic[a] else self.n[a] + 1 for a in range(self.d))

    def face_shape(self, a):
        """Faces normal to axis ``a``: ``n[a]+1`` positions along ``a`` (for a
        periodic axis face ``n[a]`` duplicates face 0)."""
        s = list(self.n)
        s[a] += 1
        return tuple(s)

    def coarsen(self):
        return Grid([v // 2 for v in self.n], 2 * self.h, self.periodic, np.zeros_like(self.wall_u))

    def can_coarsen(self):
        """Coarsen by two while every axis is even and keeps at least 2 cells
        (a deep hierarchy keeps the bottom problem small enough for a fixed
        number of smoothing sweeps to solve it)."""
        return all(v % 2 == 0 and v // 2 >= 2 for v in self.n)


def sl(d, axis, s):
    """Index tuple selecting slice ``s`` along ``axis`` of a d-dim array."""
    idx = [slice(None)] * d
    idx[axis] = s
    return tuple(idx)


def pad_cells(a, G, grid, kind, wall_vals=None):
    """Pad a cell-centred array with ``G`` ghost layers on every side.

    ``kind`` is ``"dirichlet"`` (odd reflection about the wall value
    ``wall_vals[axis][side]``, zero if None) or ``"neumann"`` (even reflection).
    Periodic axes wrap.  Axes are filled in order so corners take the last fill.
    """
    d = grid.d
    a = np.asarray(a, dtype=np.float64)
    out = np.zeros(tuple(s + 2 * G for s in a.shape))
    out[tuple(slice(G, G + s) for s in a.shape)] = a
    for ax in range(d):
        n = grid.n[ax]
        for g in range(1, G + 1):
            lo_ghost, hi_ghost = G - g, G + n - 1 + g
            lo_mirror, hi_mirror = G + g - 1, G + n - g
            if grid.periodic[ax]:
                out[sl(d, ax, lo_ghost)] = out[sl(d, ax, G + n - g)]
                out[sl(d, ax, hi_ghost)] = out[sl(d, ax, G + g - 1)]
            elif kind == "dirichlet":
                ub0 = 0.0 if wall_vals is None else wall_vals[ax][0]
                ub1 = 0.0 if wall_vals is None else wall_vals[ax][1]
                out[sl(d, ax, lo_ghost)] = 2.0 * ub0 - out[sl(d, ax, lo_mirror)]
                out[sl(d, ax, hi_ghost)] = 2.0 * ub1 - out[sl(d, ax, hi_mirror)]
            elif kind == "neumann":
                out[sl(d, ax, lo_ghost)] = out[sl(d, ax, lo_mirror)]
                out[sl(d, ax, hi_ghost)] = out[sl(d, ax, hi_mirror)]
            elif kind == "zero":
                out[sl(d, ax, lo_ghost)] = 0.0
                out[sl(d, ax, hi_ghost)] = 0.0
            else:
                raise ValueError(kind)
    return out


def velocity_wall_vals(grid, c, homogeneous=False):
    """Wall values of velocity component ``c`` as ``[axis][side]``."""
    if homogeneous:
        return None
    return [[grid.wall_u[a, 0, c], grid.wall_u[a, 1, c]] for a in range(grid.d)]


def pad_nodes(p, grid):
    """Pad a unique-node array with one ghost node per side: even reflection
    (homogeneous Neumann) across a wall, wrap along a periodic axis."""
    d = grid.d
    out = np.zeros(tuple(s + 2 for s in p.shape))
    out[tuple(slice(1, 1 + s) for s in p.shape)] = p
    for ax in range(d):
        m = p.shape[ax]
        if grid.periodic[ax]:
            out[sl(d, ax, 0)] = out[sl(d, ax, m)]
            out[sl(d, ax, m + 1)] = out[sl(d, ax, 1)]
        else:
            out[sl(d, ax, 0)] = out[sl(d, ax, 2)]
            out[sl(d, ax, m + 1)] = out[sl(d, ax, m - 1)]
    return out


def node_weights(grid):
    """w_n = product over wall axes of 1/2 on a wall node (1 otherwise): the
    fraction of the node's dual cell inside the domain.  Used for the
    compatibility condition of the singular nodal problem."""
    w = np.ones(grid.node_shape)
    for ax in range(grid.d):
        if not grid.periodic[ax]:
            w[sl(grid.d, ax, 0)] *= 0.5
            w[sl(grid.d, ax, grid.n[ax])] *= 0.5
    return w


def nodes_full(p_unique, grid):
    """Expand a unique-node array to ``n+1`` nodes per axis (periodic axes
    repeat node 0 at the end)."""
    out = p_unique
    for ax in range(grid.d):
        if grid.periodic[ax]:
            out = np.concatenate([out, out[sl(grid.d, ax, slice(0, 1))]], axis=ax)
    return out


def nodes_unique(p_full, grid):
    out = p_full
    for ax in range(grid.d):
        if grid.periodic[ax]:
            out = out[sl(grid.d, ax, slice(0, grid.n[ax]))]
    return np.ascontiguousarray(out)


def parity_colour(shape):
    """Red-black colour of each point: (sum of indices) mod 2."""
    idx = np.indices(shape)
    return idx.sum(axis=0) % 2


def multicolour(shape):
    """2^d colours by index parity per axis: colour = sum_a (i_a mod 2) 2^a.
    No two points of one colour are neighbours in the 3^d-point stencil."""
    idx = np.indices(shape)
    return sum(((idx[a] % 2) << a) for a in range(len(shape)))
