"""Geometric multigrid for the three linear solves of the step.

The paper uses AMReX's cell- and node-based (and tensor) multigrid solvers
(Sec. III D) without specifying them, so this module states its own plain
V-cycle, written the textbook way:

    V(l): nu1 smoothing sweeps; r = b - A x; restrict r; solve the coarse error
          equation by V(l+1) from zero; prolong and add; nu2 sweeps.
    coarsest level: an exact dense solve when it has at most DENSE_MAX
    unknowns (the usual case: 2^d cells), else ``nu_bottom`` smoothing sweeps.
    stop when ||b - A x||_inf <= rtol ||b||_inf (||b|| after removing the mean
    of a singular problem's right-hand side).

Problems:
* ``CellPoisson``   MAC potential: cell-centred Laplacian, Neumann walls,
                    red-black Gauss-Seidel, restriction by averaging the 2^d
                    children, cell-centred multilinear prolongation.
* ``TensorViscous`` (I - dt/(2 rho) L_eta) u = b for all components at once,
                    Dirichlet walls; one sweep = for each component c, red
                    then black Gauss-Seidel on u_c with the other components'
                    current values in the cross terms; coarse eta = mean of
                    the children.
* ``NodalPoisson``  FE nodal Laplacian, Neumann walls, 2^d-colour Gauss-Seidel
                    (the 3^d stencil couples diagonal neighbours, so two
                    colours would not be independent), full-weighting
                    restriction, multilinear prolongation.
Singular problems (MAC, nodal) subtract the (weighted) mean of the right-hand
side and pin the mean of the iterate after every cycle and the bottom solve.
"""

import numpy as np

from .grid import Grid, multicolour, node_weights, pad_cells, pad_nodes, parity_colour, sl
from .operators import (cell_lap, face_eta_all, fe_stencil, nodal_lap, tensor_cross_part, tensor_op)


class SolverParams:
    def __init__(self, rtol=1e-10, max_cycles=200, nu1=2, nu2=2, nu_bottom=40):
        self.rtol = rtol
        self.max_cycles = max_cycles
        self.nu1 = nu1
        self.nu2 = nu2
        self.nu_bottom = nu_bottom


class SolveStats:
    def __init__(self, cycles, r0, rnorm, bnorm, converged):
        self.cycles = cycles
        self.r0 = r0
        self.rnorm = rnorm
        self.bnorm = bnorm
        self.converged = converged

    def __repr__(self):
        return (f"SolveStats(cycles={self.cycles}, r0={self.r0:.3e}, rnorm={self.rnorm:.3e}, "
                f"bnorm={self.bnorm:.3e}, converged={self.converged})")


def build_levels(grid):
    levels = [grid]
    while levels[-1].can_coarsen():
        levels.append(levels[-1].coarsen())
    return levels


def restrict_cells(r, fine):
    """Mean of the 2^d fine children of each coarse cell."""
    d = fine.d
    out = r
    for a in range(d):
        out = 0.5 * (out[sl(d, a, slice(0, None, 2))] + out[sl(d, a, slice(1, None, 2))])
    return out


def restrict_faces(ef, fine):
    """Coarse-face coefficients: on each coarse a-face, the mean of the 2^(d-1)
    fine a-faces that tile it (no averaging across the face, so a coefficient
    jump along a grid plane stays sharp on coarse levels)."""
    d = fine.d
    out = []
    for a in range(d):
        f = ef[a][sl(d, a, slice(0, None, 2))]
        for b in range(d):
            if b != a:
                f = 0.5 * (f[sl(d, b, slice(0, None, 2))] + f[sl(d, b, slice(1, None, 2))])
        out.append(f)
    return out


def prolong_cells(e, coarse, kind):
    """Cell-centred multilinear interpolation: a fine child takes 3/4 of its
    parent and 1/4 of the parent's neighbour on its side, per axis; ghosts by
    ``kind`` (odd reflection for Dirichlet error, even for Neumann)."""
    d = coarse.d
    out = pad_cells(e, 1, coarse, kind)
    for a in range(d):
        n = coarse.n[a]
        c = out[sl(d, a, slice(1, n + 1))]
        lo = out[sl(d, a, slice(0, n))]
        hi = out[sl(d, a, slice(2, n + 2))]
        shape = list(c.shape)
        shape[a] = 2 * n
        f = np.empty(shape)
        f[sl(d, a, slice(0, None, 2))] = 0.75 * c + 0.25 * lo
        f[sl(d, a, slice(1, None, 2))] = 0.75 * c + 0.25 * hi
        out = f
    return out


def restrict_nodes(r, fine):
    """Full weighting (1/4, 1/2, 1/4 per axis) onto coarse nodes, with even
    reflection at walls and wrap on periodic axes."""
    d = fine.d
    out = r
    for a in range(d):
        m = out.shape[a]
        ext = np.concatenate([out[sl(d, a, slice(1, 2))] if not fine.periodic[a] else out[sl(d, a, slice(m - 1, m))],
                              out,
                              out[sl(d, a, slice(m - 2, m - 1))] if not fine.periodic[a] else out[sl(d, a, slice(0, 1))]],
                             axis=a)
        # fine node k sits at ext index k+1; coarse node I uses fine 2I-1, 2I, 2I+1
        mc = fine.n[a] // 2 + (0 if fine.periodic[a] else 1)
        cen = ext[sl(d, a, slice(1, 2 * mc, 2))]
        lo = ext[sl(d, a, slice(0, 2 * mc - 1, 2))]
        hi = ext[sl(d, a, slice(2, 2 * mc + 1, 2))]
        out = 0.5 * cen + 0.25 * (lo + hi)
    return out


def prolong_nodes(e, coarse):
    """Multilinear interpolation from coarse to fine nodes (coarse node I is
    fine node 2I; in-between fine nodes take the mean of their two parents)."""
    d = coarse.d
    out = e
    for a in range(d):
        m = out.shape[a]
        if coarse.periodic[a]:
            nxt = np.concatenate([out[sl(d, a, slice(1, m))], out[sl(d, a, slice(0, 1))]], axis=a)
            mf = 2 * m
            shape = list(out.shape)
            shape[a] = mf
            f = np.empty(shape)
            f[sl(d, a, slice(0, None, 2))] = out
            f[sl(d, a, slice(1, None, 2))] = 0.5 * (out + nxt)
        else:
            mf = 2 * (m - 1) + 1
            shape = list(out.shape)
            shape[a] = mf
            f = np.empty(shape)
            f[sl(d, a, slice(0, None, 2))] = out
            f[sl(d, a, slice(1, None, 2))] = 0.5 * (out[sl(d, a, slice(0, m - 1))] + out[sl(d, a, slice(1, m))])
        out = f
    return out


def _max_abs(xs):
    return max(float(np.max(np.abs(x))) if x.size else 0.0 for x in xs)


class CellPoisson:
    """Cell-centred Laplacian A phi = div grad phi with homogeneous Neumann
    walls (the MAC projection's potential equation).  Always singular."""

    singular = True

    def __init__(self, grid):
        self.levels = build_levels(grid)
        self.counts = []
        for g in self.levels:
            ones = np.ones(g.n)
            op = pad_cells(ones, 1, g, "zero")
            cnt = np.zeros(g.n)
            for a in range(g.d):
                cnt += op[_nb(g.d, a, -1)] + op[_nb(g.d, a, +1)]
            self.counts.append(cnt)
        self.colours = [parity_colour(g.n) for g in self.levels]

    def apply(self, l, x):
        return [cell_lap(x[0], self.levels[l])]

    def smooth(self, l, x, b):
        g = self.levels[l]
        for col in (0, 1):
            xp = pad_cells(x[0], 1, g, "zero")
            s = np.zeros(g.n)
            for a in range(g.d):
                s += xp[_nb(g.d, a, -1)] + xp[_nb(g.d, a, +1)]
            new = (s - g.h * g.h * b[0]) / self.counts[l]
            m = self.colours[l] == col
            x[0][m] = new[m]

    def restrict(self, l, r):
        return [restrict_cells(r[0], self.levels[l])]

    def prolong_add(self, l, x, e):
        x[0] += prolong_cells(e[0], self.levels[l + 1], "neumann")

    def zeros(self, l):
        return [np.zeros(self.levels[l].n)]

    def mean(self, l, x):
        return [float(np.mean(x[0]))]

    def sub_mean(self, l, x):
        x[0] -= np.mean(x[0])


def _nb(d, a, s):
    """Slice of a 1-ghost padded cell array giving the neighbour at offset s
    along axis a for every interior cell."""
    idx = [slice(1, -1)] * d
    idx[a] = slice(1 + s, (-1 + s) if (-1 + s) != 0 else None)
    return tuple(idx)


class TensorViscous:
    """(I - beta L_eta) u = b, beta = dt / (2 rho), all d components coupled
    through the cross terms of L_eta (Eq. 16).  Level 0 carries the wall
    velocities (unless ``hom0``), coarse levels the homogeneous error
    equation."""

    singular = False

    def __init__(self, grid, eta, beta, hom0=False):
        self.levels = build_levels(grid)
        self.beta = beta
        self.hom0 = hom0
        self.etas = [face_eta_all(eta, grid)]
        for l in range(1, len(self.levels)):
            self.etas.append(restrict_faces(self.etas[-1], self.levels[l - 1]))
        self.colours = [parity_colour(g.n) for g in self.levels]
        self.walls = [[[_wall_mask(g, a, s) for s in (-1, 1)] for a in range(g.d)] for g in self.levels]

    def apply(self, l, u):
        g = self.levels[l]
        Lu = tensor_op(u, self.etas[l], g, homogeneous=(l > 0 or self.hom0))
        return [u[c] - self.beta * Lu[c] for c in range(g.d)]

    def smooth(self, l, u, b):
        g = self.levels[l]
        d, h = g.d, g.h
        eta = self.etas[l]
        hom = l > 0 or self.hom0
        for c in range(d):
            cross = tensor_cross_part(u, eta, g, c, homogeneous=hom)
            for col in (0, 1):
                up = pad_cells(u[c], 1, g, "zero")
                offd = np.zeros(g.n)
                diag = np.zeros(g.n)
                for a in range(d):
                    kappa = 2.0 if a == c else 1.0
                    ef = eta[a]
                    w = kappa * ef / (h * h)
                    for s, fsl in ((-1, slice(0, -1)), (+1, slice(1, None))):
                        wf = w[sl(d, a, fsl)]
                        nb = up[_nb(d, a, s)]
                        wall = self.walls[l][a][0 if s < 0 else 1]
                        ub = 0.0 if hom else g.wall_u[a, 0 if s < 0 else 1, c]
                        offd += np.where(wall, 2.0 * wf * ub, wf * nb)
                        diag += np.where(wall, 2.0 * wf, wf)
                new = (b[c] + self.beta * (offd + cross)) / (1.0 + self.beta * diag)
                m = self.colours[l] == col
                u[c][m] = new[m]

    def restrict(self, l, r):
        return [restrict_cells(rc, self.levels[l]) for rc in r]

    def prolong_add(self, l, x, e):
        for c in range(len(x)):
            x[c] += prolong_cells(e[c], self.levels[l + 1], "dirichlet")

    def zeros(self, l):
        return [np.zeros(self.levels[l].n) for _ in range(self.levels[l].d)]


def _wall_mask(g, a, s):
    """Cells whose face on side s of axis a is a wall."""
    m = np.zeros(g.n, dtype=bool)
    if not g.periodic[a]:
        m[sl(g.d, a, 0 if s < 0 else g.n[a] - 1)] = True
    return m


class NodalPoisson:
    """FE nodal Laplacian L phi = f with Neumann walls (Eq. 17).  Singular; the
    compatibility weights are the dual-cell fractions w_n."""

    singular = True

    def __init__(self, grid):
        self.levels = build_levels(grid)
        self.weights = [node_weights(g) for g in self.levels]
        self.colours = [multicolour(g.node_shape) for g in self.levels]
        self.stencil = fe_stencil(grid.d)

    def apply(self, l, x):
        return [nodal_lap(x[0], self.levels[l])]

    def smooth(self, l, x, b):
        g = self.levels[l]
        d = g.d
        ncol = 2 ** d
        for col in range(ncol):
            pp = pad_nodes(x[0], g)
            s = np.zeros(x[0].shape)
            for o, wgt in self.stencil.items():
                if wgt == 0.0 or all(v == 0 for v in o):
                    continue
                idx = tuple(slice(1 + o[k], 1 + o[k] + x[0].shape[k]) for k in range(d))
                s += wgt * pp[idx]
            new = (g.h * g.h * b[0] - s) / self.stencil[(0,) * d]
            m = self.colours[l] == col
            x[0][m] = new[m]

    def restrict(self, l, r):
        return [restrict_nodes(r[0], self.levels[l])]

    def prolong_add(self, l, x, e):
        x[0] += prolong_nodes(e[0], self.levels[l + 1])

    def zeros(self, l):
        return [np.zeros(self.levels[l].node_shape)]

    def sub_mean(self, l, x):
        w = self.weights[l]
        x[0] -= float(np.sum(w * x[0]) / np.sum(w))


def _residual(prob, l, x, b):
    Ax = prob.apply(l, x)
    return [b[c] - Ax[c] for c in range(len(b))]


DENSE_MAX = 128


def _flat(xs):
    return np.concatenate([x.ravel() for x in xs])


def _unflat(v, like):
    out, k = [], 0
    for a in like:
        out.append(v[k:k + a.size].reshape(a.shape))
        k += a.size
    return out


def _bottom_dense(prob, l, x, b):
    """x = exact solution of the level-l problem for right-hand side b (the
    affine part of a level with wall values is moved to the right).  Singular
    problems are solved with their (weighted) mean-zero constraint appended as
    a bordered row and column."""
    cache = prob.__dict__.setdefault("_dense_cache", {})
    key = (l, bool(getattr(prob, "hom0", False)))
    like = prob.zeros(l)
    if key not in cache:
        z = prob.zeros(l)
        a0 = _flat(prob.apply(l, z))
        n = a0.size
        M = np.zeros((n, n))
        for k in range(n):
            e = np.zeros(n)
            e[k] = 1.0
            M[:, k] = _flat(prob.apply(l, _unflat(e, like))) - a0
        if prob.singular:
            w = _flat([prob.weights[l]]) if isinstance(prob, NodalPoisson) else np.ones(n)
            B = np.zeros((n + 1, n + 1))
            B[:n, :n] = M
            B[:n, n] = w
            B[n, :n] = w
            M = B
        cache[key] = (M, a0)
    M, a0 = cache[key]
    rhs = _flat(b) - a0
    if prob.singular:
        rhs = np.concatenate([rhs, [0.0]])
    sol = np.linalg.solve(M, rhs)[:a0.size]
    for xc, sc in zip(x, _unflat(sol, like)):
        xc[...] = sc


def vcycle(prob, l, x, b, params):
    if l == len(prob.levels) - 1:
        if prob.singular:
            b = [bc.copy() for bc in b]
            prob.sub_mean(l, b)
        if sum(a.size for a in x) <= DENSE_MAX:
            _bottom_dense(prob, l, x, b)
        else:
            for _ in range(params.nu_bottom):
                prob.smooth(l, x, b)
        if prob.singular:
            prob.sub_mean(l, x)
        return
    for _ in range(params.nu1):
        prob.smooth(l, x, b)
    r = _residual(prob, l, x, b)
    rc = prob.restrict(l, r)
    ec = prob.zeros(l + 1)
    vcycle(prob, l + 1, ec, rc, params)
    prob.prolong_add(l, x, ec)
    for _ in range(params.nu2):
        prob.smooth(l, x, b)


def mg_solve(prob, x, b, params):
    """Iterate V-cycles until ||b - A x||_inf <= rtol ||b||_inf.  ``x`` (a list
    of arrays) is updated in place and returned with a SolveStats."""
    b = [np.array(bc, dtype=np.float64) for bc in b]
    if prob.singular:
        prob.sub_mean(0, b)
        prob.sub_mean(0, x)
    bnorm = _max_abs(b)
    rn = _max_abs(_residual(prob, 0, x, b))
    r0 = rn
    if bnorm == 0.0:
        bnorm = rn
    tol = params.rtol * bnorm
    cycles = 0
    while rn > tol and cycles < params.max_cycles:
        vcycle(prob, 0, x, b, params)
        cycles += 1
        if prob.singular:
            prob.sub_mean(0, x)
        rn = _max_abs(_residual(prob, 0, x, b))
    return x, SolveStats(cycles, r0, rn, bnorm, rn <= tol)


def _dot(a, b):
    return sum(float(np.sum(x * y)) for x, y in zip(a, b))


def bicgstab_solve(prob, x, b, params):
    """BiCGStab (van der Vorst 1992) on (I - beta L_eta) u = b, right-
    preconditioned by one V-cycle of the homogeneous operator from a zero
    guess.  The V-cycle alone is not a convergent iteration for every
    viscosity field the regularised law produces (at large contrast the
    component-wise smoother with frozen cross terms can diverge), but it is a
    good preconditioner.  Stops when the recursive residual meets
    ||r||_inf <= rtol ||b||_inf and the true residual confirms it; otherwise
    restarts from the true residual.  ``cycles`` counts BiCGStab iterations
    (two V-cycles each)."""
    b = [np.array(bc, dtype=np.float64) for bc in b]
    pre = TensorViscous.__new__(TensorViscous)
    pre.__dict__.update(prob.__dict__)
    pre.hom0 = True
    d = len(b)

    def A0(e):
        return pre.apply(0, e)

    def M(r):
        e = pre.zeros(0)
        vcycle(pre, 0, e, [rc.copy() for rc in r], params)
        return e

    bnorm = _max_abs(b)
    r = _residual(prob, 0, x, b)
    rn = _max_abs(r)
    r0 = rn
    if bnorm == 0.0:
        bnorm = rn
    tol = params.rtol * bnorm
    it = 0
    while rn > tol and it < params.max_cycles:
        rhat = [rc.copy() for rc in r]
        rho = alpha = omega = 1.0
        v = [np.zeros_like(rc) for rc in r]
        p = [np.zeros_like(rc) for rc in r]
        while it < params.max_cycles:
            rho1 = _dot(rhat, r)
            if rho1 == 0.0:
                break
            beta = (rho1 / rho) * (alpha / omega)
            p = [r[c] + beta * (p[c] - omega * v[c]) for c in range(d)]
            phat = M(p)
            v = A0(phat)
            den = _dot(rhat, v)
            if den == 0.0:
                break
            alpha = rho1 / den
            s = [r[c] - alpha * v[c] for c in range(d)]
            shat = M(s)
            t = A0(shat)
            tt = _dot(t, t)
            omega = _dot(t, s) / tt if tt > 0.0 else 0.0
            x = [x[c] + alpha * phat[c] + omega * shat[c] for c in range(d)]
            r = [s[c] - omega * t[c] for c in range(d)]
            rho = rho1
            it += 1
            if _max_abs(r) <= tol or omega == 0.0:
                break
        r = _residual(prob, 0, x, b)
        rn = _max_abs(r)
    return x, SolveStats(it, r0, rn, bnorm, rn <= tol)
