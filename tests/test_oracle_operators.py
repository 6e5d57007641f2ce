"""Pins for the oracle's discrete operators (Sec. III A, Eqs. 12, 16, 17).

Fixed by: exact reproduction of polynomial fields by second-order stencils,
the bilinear/trilinear finite-element stiffness assembled by quadrature,
discrete integration-by-parts identities, and symmetry of the constant-
coefficient operator."""

import itertools

import numpy as np
import pytest

from oracle.grid import Grid, node_weights
from oracle.operators import (cell_grad_nodal, cell_lap, face_eta_all, fe_stencil, mac_div,
                              mac_grad, nodal_div, nodal_lap, tensor_op)


def _centres(n, h):
    return np.meshgrid(*[(np.arange(s) + 0.5) * h for s in n], indexing="ij")


def _nodes(n, h):
    return np.meshgrid(*[np.arange(s + 1) * h for s in n], indexing="ij")


def _inner(d, k=1):
    return tuple(slice(k, -k) for _ in range(d))


@pytest.mark.parametrize("d", [2, 3])
def test_tensor_op_constant_eta_quadratic_exact(d):
    # div(eta (grad u + grad u^T)) = eta (lap u + grad div u) for constant eta;
    # second-order stencils are exact on quadratics away from the walls.
    rng = np.random.default_rng(10 + d)
    n = (7,) * d
    h = 0.3
    g = Grid(n, h)
    X = _centres(n, h)
    # u_c = sum_{a<=b} Q[c,a,b] x_a x_b
    Q = rng.normal(size=(d, d, d))
    Q = 0.5 * (Q + Q.transpose(0, 2, 1))
    u = [sum(Q[c, a, b] * X[a] * X[b] for a in range(d) for b in range(d)) for c in range(d)]
    eta0 = 1.7
    Lu = tensor_op(u, face_eta_all(np.full(n, eta0), g), g)
    # d_a d_b u_c = 2 Q[c,a,b]
    for c in range(d):
        lap = sum(2 * Q[c, a, a] for a in range(d))
        graddiv = sum(2 * Q[a, a, c] for a in range(d))
        np.testing.assert_allclose(Lu[c][_inner(d, 2)], eta0 * (lap + graddiv), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("d", [2, 3])
def test_tensor_op_linear_eta_linear_u_exact(d):
    # u linear (u_c = sum_a B[c,a] x_a), eta = e0 + gvec.x: the result is
    # sum_a (d_a eta)(d_a u_c + d_c u_a) = sum_a gvec_a (B[c,a] + B[a,c]).
    # A transposed operand (B[c,a] twice) or a wrong face average fails this.
    rng = np.random.default_rng(20 + d)
    n = (6,) * d
    h = 0.25
    g = Grid(n, h)
    X = _centres(n, h)
    B = rng.normal(size=(d, d))
    gv = rng.normal(size=d)
    u = [sum(B[c, a] * X[a] for a in range(d)) for c in range(d)]
    eta = 5.0 + sum(gv[a] * X[a] for a in range(d))
    Lu = tensor_op(u, face_eta_all(eta, g), g)
    for c in range(d):
        expect = sum(gv[a] * (B[c, a] + B[a, c]) for a in range(d))
        np.testing.assert_allclose(Lu[c][_inner(d, 2)], expect, rtol=1e-11, atol=1e-11)


def _tensor_matrix(g, eta0):
    d = g.d
    n = g.n
    ef = face_eta_all(np.full(n, eta0), g)
    N = int(np.prod(n))
    M = np.zeros((d * N, d * N))
    for k in range(d * N):
        e = np.zeros(d * N)
        e[k] = 1.0
        u = [e[c * N:(c + 1) * N].reshape(n) for c in range(d)]
        Lu = tensor_op(u, ef, g, homogeneous=True)
        M[:, k] = np.concatenate([x.ravel() for x in Lu])
    return M


@pytest.mark.parametrize("d", [2, 3])
def test_tensor_op_constant_eta_periodic_is_self_adjoint(d):
    # With no walls and constant eta the stencil is the discrete version of the
    # self-adjoint, negative semi-definite div(2 eta D u): its matrix is symmetric
    # and its null space holds the uniform translations.
    n = (4,) * d
    g = Grid(n, 0.5, periodic=(True,) * d)
    M = _tensor_matrix(g, 1.3)
    np.testing.assert_allclose(M, M.T, atol=1e-12)
    ev = np.linalg.eigvalsh(M)
    assert np.max(ev) < 1e-10 and np.sum(np.abs(ev) < 1e-10) == d


@pytest.mark.parametrize("d", [2, 3])
def test_tensor_op_with_walls_is_dissipative(d):
    # Walls make the stencil non-symmetric next to the boundary (the tangential
    # derivative there uses the reflected ghost), but its symmetric part stays
    # negative definite, so (I - beta L) is invertible for every beta > 0.
    n = (4,) * d if d == 2 else (3, 4, 3)
    g = Grid(n, 0.5)
    M = _tensor_matrix(g, 1.3)
    assert np.max(np.linalg.eigvalsh(0.5 * (M + M.T))) < 0


def _fe_stiffness_stencil(d):
    """Assemble the Q1 stiffness row of an interior node by Gauss quadrature of
    grad(psi_i).grad(psi_j) over the 2^d elements around it (unit h), divided
    by the lumped mass 1 to give the strong-form stencil of -lap."""
    xg, wg = np.polynomial.legendre.leggauss(3)
    xg = 0.5 * (xg + 1.0)
    wg = 0.5 * wg

    def phi1(c, x):
        return x if c == 1 else 1.0 - x

    def dphi1(c):
        return 1.0 if c == 1 else -1.0

    st = {}
    # node at origin; element with lower corner e in {-1,0}^d
    for e in itertools.product((-1, 0), repeat=d):
        local0 = tuple(-v for v in e)  # origin's local vertex index
        for loc in itertools.product((0, 1), repeat=d):
            off = tuple(e[a] + loc[a] for a in range(d))
            val = 0.0
            for q in itertools.product(range(3), repeat=d):
                x = [xg[q[a]] for a in range(d)]
                w = np.prod([wg[q[a]] for a in range(d)])
                for a in range(d):
                    gi = dphi1(local0[a]) * np.prod([phi1(local0[b], x[b]) for b in range(d) if b != a])
                    gj = dphi1(loc[a]) * np.prod([phi1(loc[b], x[b]) for b in range(d) if b != a])
                    val += w * gi * gj
            st[off] = st.get(off, 0.0) + val
    return {k: -v for k, v in st.items()}  # strong form of +lap


@pytest.mark.parametrize("d", [2, 3])
def test_fe_stencil_is_assembled_q1_stiffness(d):
    ref = _fe_stiffness_stencil(d)
    st = fe_stencil(d)
    for o in itertools.product((-1, 0, 1), repeat=d):
        assert st[o] == pytest.approx(ref.get(o, 0.0), abs=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_nodal_lap_exact_on_quadratics(d):
    rng = np.random.default_rng(30 + d)
    n = (6,) * d
    h = 0.2
    g = Grid(n, h)
    X = _nodes(n, h)
    Q = rng.normal(size=(d, d))
    Q = 0.5 * (Q + Q.T)
    phi = sum(Q[a, b] * X[a] * X[b] for a in range(d) for b in range(d))
    L = nodal_lap(phi, g)
    np.testing.assert_allclose(L[_inner(d)], 2 * np.trace(Q), rtol=1e-11)


@pytest.mark.parametrize("d", [2, 3])
def test_nodal_div_and_cell_grad_exact_on_linear(d):
    rng = np.random.default_rng(40 + d)
    n = (5,) * d
    h = 0.3
    g = Grid(n, h)
    B = rng.normal(size=(d, d))
    Xc = _centres(n, h)
    v = [sum(B[c, a] * Xc[a] for a in range(d)) for c in range(d)]
    D = nodal_div(v, g, node_weights(g))
    np.testing.assert_allclose(D[_inner(d)], np.trace(B), rtol=1e-12)
    Xn = _nodes(n, h)
    gp = rng.normal(size=d)
    p = sum(gp[a] * Xn[a] for a in range(d))
    G = cell_grad_nodal(p, g)
    for a in range(d):
        np.testing.assert_allclose(G[a], gp[a], rtol=1e-12)


@pytest.mark.parametrize("d,periodic", [(2, None), (3, None), (2, (True, False)), (3, (False, True, False))])
def test_nodal_div_is_minus_adjoint_of_cell_grad(d, periodic):
    # sum_cells v . G p = - sum_nodes w_n p D v  (discrete integration by parts
    # with impermeable walls; w_n is the dual-cell fraction of the node)
    rng = np.random.default_rng(50 + d)
    n = (4,) * d
    g = Grid(n, 0.7, periodic=periodic)
    v = [rng.normal(size=n) for _ in range(d)]
    p = rng.normal(size=g.node_shape)
    w = node_weights(g)
    lhs = sum(np.sum(v[a] * G) for a, G in enumerate(cell_grad_nodal(p, g)))
    rhs = -np.sum(w * p * nodal_div(v, g, w))
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_nodal_lap_weighted_symmetric(d):
    # W L is the assembled (symmetric) FE stiffness; constants are its null space
    n = (4,) * d if d == 2 else (2, 4, 2)
    g = Grid(n, 0.5)
    shape = g.node_shape
    N = int(np.prod(shape))
    M = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        M[:, k] = nodal_lap(e.reshape(shape), g).ravel()
    WM = node_weights(g).ravel()[:, None] * M
    np.testing.assert_allclose(WM, WM.T, atol=1e-12)
    np.testing.assert_allclose(M @ np.ones(N), 0.0, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_fe_lap_close_to_div_grad(d):
    # L approximates D G to second order for smooth phi (the approximate
    # projection of Sec. III A): the max difference drops ~4x per refinement.
    errs = []
    for N in (8, 16, 32):
        g = Grid((N,) * d, 1.0 / N)
        X = _nodes(g.n, g.h)
        phi = np.prod([np.cos(np.pi * X[a]) for a in range(d)], axis=0)
        diff = nodal_lap(phi, g) - nodal_div(cell_grad_nodal(phi, g), g, node_weights(g))
        errs.append(np.max(np.abs(diff[_inner(d)])))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert rates[-1] > 1.85 and min(rates) > 1.6


@pytest.mark.parametrize("d", [2, 3])
def test_mac_div_grad_adjoint_and_cell_lap_quadratic(d):
    rng = np.random.default_rng(60 + d)
    n = (5,) * d
    h = 0.4
    g = Grid(n, h)
    phi = rng.normal(size=n)
    faces = []
    for a in range(d):
        f = rng.normal(size=g.face_shape(a))
        f[tuple(0 if b == a else slice(None) for b in range(d))] = 0.0
        f[tuple(n[a] if b == a else slice(None) for b in range(d))] = 0.0
        faces.append(f)
    lhs = sum(np.sum(faces[a] * mac_grad(phi, g, a)) for a in range(d))
    rhs = -np.sum(phi * mac_div(faces, g))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    X = _centres(n, h)
    q = sum((a + 1.0) * X[a] ** 2 for a in range(d))
    np.testing.assert_allclose(cell_lap(q, g)[_inner(d)], sum(2.0 * (a + 1.0) for a in range(d)), rtol=1e-11)
