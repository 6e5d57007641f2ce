"""The multigrid pieces' per-element device code, built for the host, against
the oracle on seeded fields: the viscous operator (I - beta L_eta) u and one
red-black sweep of each component (Eq. 16), the cell Poisson residual and
sweep, the nodal FE residual and 2^D-colour sweep (Eq. 17), and the cell,
face and nodal transfers.  The kernels run exactly this code; these checks
need no GPU and agree to rounding."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.grid import Grid
from oracle.multigrid import (CellPoisson, NodalPoisson, TensorViscous, prolong_cells, prolong_nodes,
                              restrict_cells, restrict_faces, restrict_nodes)
from oracle.operators import cell_lap, face_eta_all, nodal_lap
from paper_1803_00417_gb300.hbflow import from_device_layout, to_device_layout

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1803_00417_gb300", "csrc")
TOL = 1e-12


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("mg") / "mg_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "host", "mg_check.cu"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return exe


def rel(a, b):
    a = [np.asarray(x) for x in (a if isinstance(a, (list, tuple)) else [a])]
    b = [np.asarray(x) for x in (b if isinstance(b, (list, tuple)) else [b])]
    num = sum(float(np.sum((x - y) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(y ** 2)) for y in b)
    return np.sqrt(num / den) if den > 0 else np.sqrt(num)


@pytest.mark.parametrize("n,hom,seed", [((8, 6), 0, 51), ((8, 6), 1, 52), ((6, 4, 8), 0, 53), ((4, 8, 6), 1, 54)])
def test_multigrid_pieces_match_oracle(harness, tmp_path, n, hom, seed):
    rng = np.random.default_rng(seed)
    d = len(n)
    h = 1.0 / max(n)
    wall = rng.standard_normal((d, 2, d))
    for a in range(d):
        wall[a, :, a] = 0.0
    g = Grid(n, h, wall_u=wall)
    gc = g.coarsen()
    beta = 0.3 * h * h
    eta = np.exp(rng.standard_normal(n))
    u = [rng.standard_normal(n) for _ in range(d)]
    bv = [rng.standard_normal(n) for _ in range(d)]
    x, bc = rng.standard_normal(n), rng.standard_normal(n)
    xn, bn = rng.standard_normal(g.node_shape), rng.standard_normal(g.node_shape)
    ev = [rng.standard_normal(gc.n) for _ in range(d)]
    ec = rng.standard_normal(gc.n)
    en = rng.standard_normal(gc.node_shape)

    wu = np.zeros((3, 2, 3))
    wu[:d, :, :d] = wall
    src = tmp_path / "in.bin"
    with open(src, "wb") as f:
        np.array([d, *(list(n) + [1] * (3 - d)), hom], dtype=np.int32).tofile(f)
        np.array([h, beta], dtype=np.float64).tofile(f)
        wu.ravel().tofile(f)
        for arr in (eta, u, bv, x, bc, xn, bn, ev, ec, en):
            to_device_layout(arr).tofile(f)
    dst = tmp_path / "out.bin"
    r = subprocess.run([harness, str(src), str(dst)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    out = np.fromfile(dst, dtype=np.float64)
    pos = 0

    def take(shape, ncomp):
        nonlocal pos
        cnt = int(np.prod(shape)) * ncomp
        v = from_device_layout(out[pos:pos + cnt], tuple(shape), ncomp)
        pos += cnt
        return v

    visc = TensorViscous(g, eta, beta, hom0=bool(hom))
    assert rel(take(n, d), visc.apply(0, u)) < TOL
    us = [c.copy() for c in u]
    visc.smooth(0, us, bv)
    assert rel(take(n, d), us) < TOL
    assert rel(take(n, 1), [bc - cell_lap(x, g)]) < TOL
    xs = [x.copy()]
    CellPoisson(g).smooth(0, xs, [bc])
    assert rel(take(n, 1), xs) < TOL
    assert rel(take(g.node_shape, 1), [bn - nodal_lap(xn, g)]) < TOL
    xns = [xn.copy()]
    NodalPoisson(g).smooth(0, xns, [bn])
    assert rel(take(g.node_shape, 1), xns) < TOL
    assert rel(take(gc.n, d), [restrict_cells(c, g) for c in u]) < TOL
    fc = restrict_faces(face_eta_all(eta, g), g)
    for a in range(d):
        assert rel(take(gc.face_shape(a), 1), [fc[a]]) < TOL, a
    assert rel(take(n, d), [u[c] + prolong_cells(ev[c], gc, "dirichlet") for c in range(d)]) < TOL
    assert rel(take(n, 1), [x + prolong_cells(ec, gc, "neumann")]) < TOL
    assert rel(take(gc.node_shape, 1), [restrict_nodes(xn, g)]) < TOL
    assert rel(take(g.node_shape, 1), [xn + prolong_nodes(en, gc)]) < TOL
    # the FP32 finest level of the mixed mode (x-interior-first maps, face
    # viscosities formed from the cell viscosity): FP32 rounding of the same
    # operator and sweep
    assert rel(take(n, d), visc.apply(0, u)) < 1e-5
    assert rel(take(n, d), us) < 1e-5
    assert rel(take(n, 1), xs) < 1e-5
    assert rel(take(g.node_shape, 1), xns) < 1e-5
    assert pos == out.size
