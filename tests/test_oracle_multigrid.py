"""Pins for the oracle's multigrid (the paper's solves use AMReX multigrid,
Sec. III D; the V-cycle itself is this project's reading).

Fixed by: dense direct solves of the same operators on tiny grids, exactness
of a Gauss-Seidel colour sweep at the points it updates, and exactness of the
grid transfers on linear fields."""

import numpy as np
import pytest

from oracle.grid import Grid, multicolour, node_weights, parity_colour
from oracle.multigrid import (CellPoisson, NodalPoisson, SolverParams, TensorViscous, mg_solve,
                              prolong_cells, prolong_nodes, restrict_cells, restrict_nodes)


def _dense(apply, shapes):
    """Matrix of the linear map apply (list of arrays -> list of arrays) and
    its affine offset apply(0)."""
    sizes = [int(np.prod(s)) for s in shapes]
    N = sum(sizes)

    def unflat(v):
        out, k = [], 0
        for s, z in zip(shapes, sizes):
            out.append(v[k:k + z].reshape(s).copy())
            k += z
        return out

    def flat(xs):
        return np.concatenate([x.ravel() for x in xs])

    b0 = flat(apply(unflat(np.zeros(N))))
    M = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        M[:, k] = flat(apply(unflat(e))) - b0
    return M, b0, unflat, flat


def _solve_singular(M, b, w):
    """Solve M x = b with the constraint sum w x = 0 (bordered system)."""
    N = M.shape[0]
    B = np.zeros((N + 1, N + 1))
    B[:N, :N] = M
    B[:N, N] = w
    B[N, :N] = w
    rhs = np.concatenate([b, [0.0]])
    return np.linalg.solve(B, rhs)[:N]


P = SolverParams(rtol=1e-13, max_cycles=400)


@pytest.mark.parametrize("n", [(8, 8), (8, 4), (4, 4, 4)])
def test_cell_poisson_mg_matches_dense(n):
    g = Grid(n, 1.0 / max(n))
    prob = CellPoisson(g)
    rng = np.random.default_rng(1)
    b = rng.normal(size=n)
    b -= b.mean()
    M, b0, unflat, flat = _dense(lambda x: prob.apply(0, x), [n])
    ref = _solve_singular(M, b.ravel(), np.ones(b.size))
    x, st = mg_solve(prob, [np.zeros(n)], [b], P)
    assert st.converged
    np.testing.assert_allclose(x[0].ravel(), ref, atol=1e-10 * np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [(8, 8), (4, 4, 4)])
def test_nodal_mg_matches_dense(n):
    g = Grid(n, 1.0 / max(n))
    prob = NodalPoisson(g)
    rng = np.random.default_rng(2)
    shape = g.node_shape
    w = node_weights(g)
    b = rng.normal(size=shape)
    b -= np.sum(w * b) / np.sum(w)
    M, b0, unflat, flat = _dense(lambda x: prob.apply(0, x), [shape])
    ref = _solve_singular(M, b.ravel(), w.ravel())
    x, st = mg_solve(prob, [np.zeros(shape)], [b], P)
    assert st.converged
    np.testing.assert_allclose(x[0].ravel(), ref, atol=1e-10 * np.max(np.abs(ref)))


@pytest.mark.parametrize("n,periodic", [((8, 8), None), ((8, 8), (True, False)), ((4, 4, 4), None)])
def test_tensor_viscous_mg_matches_dense(n, periodic):
    d = len(n)
    wall = np.zeros((d, 2, d))
    if not (periodic and periodic[d - 1]):
        wall[d - 1, 1, 0] = 1.0
    g = Grid(n, 1.0 / max(n), periodic=periodic, wall_u=wall)
    rng = np.random.default_rng(3)
    eta = np.exp(rng.uniform(-2, 2, size=n))
    prob = TensorViscous(g, eta, beta=0.05)
    b = [rng.normal(size=n) for _ in range(d)]
    M, b0, unflat, flat = _dense(lambda x: prob.apply(0, x), [n] * d)
    ref = np.linalg.solve(M, flat(b) - b0)  # affine: walls carry the lid velocity
    x, st = mg_solve(prob, [np.zeros(n) for _ in range(d)], b, P)
    assert st.converged
    np.testing.assert_allclose(flat(x), ref, atol=1e-10 * np.max(np.abs(ref)))


def test_gauss_seidel_colour_sweep_solves_its_points():
    # after the black half-sweep of component 0 the component-0 equation holds
    # exactly at every black cell (the other component is frozen meanwhile)
    n = (8, 8)
    wall = np.zeros((2, 2, 2))
    wall[1, 1, 0] = 1.0
    g = Grid(n, 0.125, wall_u=wall)
    rng = np.random.default_rng(4)
    eta = np.exp(rng.uniform(-1, 1, size=n))
    prob = TensorViscous(g, eta, beta=0.3)
    u = [rng.normal(size=n) for _ in range(2)]
    b = [rng.normal(size=n) for _ in range(2)]
    red = parity_colour(n) == 0
    u0 = [x.copy() for x in u]
    prob.smooth(0, u0, b)  # one sweep: comp 0 red, black; then comp 1 red, black
    # the black half of comp 0 was solved with comp 1 still at its old values
    u_mid = [u0[0].copy(), u[1].copy()]
    r = [bb - aa for bb, aa in zip(b, prob.apply(0, u_mid))]
    assert np.max(np.abs(r[0][~red])) < 1e-12 * max(1.0, np.max(np.abs(b[0])))
    # nodal: one 2^d-colour sweep solves the last colour exactly
    gn = Grid((8, 8), 0.125)
    pn = NodalPoisson(gn)
    x = [rng.normal(size=gn.node_shape)]
    f = [rng.normal(size=gn.node_shape)]
    pn.smooth(0, x, f)
    res = f[0] - pn.apply(0, x)[0]
    last = multicolour(gn.node_shape) == 3
    assert np.max(np.abs(res[last])) < 1e-10


@pytest.mark.parametrize("d", [2, 3])
def test_transfers_exact_on_linear_fields(d):
    rng = np.random.default_rng(5)
    nf = (8,) * d
    fine = Grid(nf, 0.125)
    coarse = fine.coarsen()
    gv = rng.normal(size=d)
    # cell averages of a linear field restrict to the coarse cell value
    Xf = np.meshgrid(*[(np.arange(s) + 0.5) * fine.h for s in nf], indexing="ij")
    Xc = np.meshgrid(*[(np.arange(s) + 0.5) * coarse.h for s in coarse.n], indexing="ij")
    lf = sum(gv[a] * Xf[a] for a in range(d))
    lc = sum(gv[a] * Xc[a] for a in range(d))
    np.testing.assert_allclose(restrict_cells(lf, fine), lc, rtol=1e-13)
    # cell-centred multilinear prolongation reproduces a linear field in the interior
    pc = prolong_cells(lc, coarse, "neumann")
    inner = tuple(slice(1, -1) for _ in range(d))
    np.testing.assert_allclose(pc[inner], lf[inner], rtol=1e-13)
    # node transfers: full weighting and multilinear interpolation are exact on linears
    Xnf = np.meshgrid(*[np.arange(s + 1) * fine.h for s in nf], indexing="ij")
    Xnc = np.meshgrid(*[np.arange(s + 1) * coarse.h for s in coarse.n], indexing="ij")
    nf_l = sum(gv[a] * Xnf[a] for a in range(d))
    nc_l = sum(gv[a] * Xnc[a] for a in range(d))
    np.testing.assert_allclose(prolong_nodes(nc_l, coarse), nf_l, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(restrict_nodes(nf_l, fine)[inner], nc_l[inner], rtol=1e-13)
    # constants survive every transfer (even reflection at walls)
    np.testing.assert_allclose(restrict_nodes(np.full(fine.node_shape, 2.5), fine), 2.5)
    np.testing.assert_allclose(prolong_cells(np.full(coarse.n, 2.5), coarse, "neumann"), 2.5)


def test_singular_solve_mean_and_zero_rhs():
    g = Grid((8, 8), 0.125)
    prob = CellPoisson(g)
    x, st = mg_solve(prob, [np.zeros((8, 8))], [np.zeros((8, 8))], SolverParams())
    assert st.cycles == 0 and np.all(x[0] == 0.0)
    rng = np.random.default_rng(6)
    b = rng.normal(size=(8, 8))
    x, st = mg_solve(prob, [np.zeros((8, 8))], [b], SolverParams())
    assert st.converged and abs(np.mean(x[0])) < 1e-14


@pytest.mark.parametrize("n", [(8, 8), (4, 4, 4)])
def test_tensor_viscous_bicgstab_matches_dense(n):
    from oracle.multigrid import bicgstab_solve

    d = len(n)
    wall = np.zeros((d, 2, d))
    wall[d - 1, 1, 0] = 1.0
    g = Grid(n, 1.0 / max(n), wall_u=wall)
    rng = np.random.default_rng(8)
    # strong contrast, as the regularised law produces
    eta = np.exp(rng.uniform(-4, 4, size=n))
    prob = TensorViscous(g, eta, beta=0.05)
    b = [rng.normal(size=n) for _ in range(d)]
    M, b0, unflat, flat = _dense(lambda x: prob.apply(0, x), [n] * d)
    ref = np.linalg.solve(M, flat(b) - b0)
    x, st = bicgstab_solve(prob, [np.zeros(n) for _ in range(d)], b, P)
    assert st.converged
    np.testing.assert_allclose(flat(x), ref, atol=1e-10 * np.max(np.abs(ref)))
