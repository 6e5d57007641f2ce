"""The explicit stages' per-element device code, built for the host, against
the oracle on seeded states: viscosity (Eqs. 1, 23), G p and L_eta u, the
Godunov face states and u^adv (Eqs. 11-14), and the nodal right-hand side
(Eq. 17).  The kernels run exactly this code; these checks need no GPU and
agree to rounding (the GPU runs of the same comparisons are in
test_gpu_parity.py)."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.grid import Grid
from oracle.step import Rheology, step
from paper_1803_00417_gb300.hbflow import from_device_layout, to_device_layout
from paper_1803_00417_gb300.inputs import cavity, random_state

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1803_00417_gb300", "csrc")
TOL = 1e-12


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("explicit") / "explicit_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "host", "explicit_check.cu"), "-o",
                    exe], check=True, capture_output=True, text=True)
    return exe


def rel_l2(a, b):
    a = [np.asarray(x) for x in (a if isinstance(a, (list, tuple)) else [a])]
    b = [np.asarray(x) for x in (b if isinstance(b, (list, tuple)) else [b])]
    num = sum(float(np.sum((x - y) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(y ** 2)) for y in b)
    return np.sqrt(num / den) if den > 0 else np.sqrt(num)


@pytest.mark.parametrize("n,seed,over", [
    ((20, 12), 41, dict(Re=1.0, Bi=2.0, Pa=1e4, nexp=1.0)),
    ((18, 14), 42, dict(Re=1000.0, Bi=5.0, Pa=1e5, nexp=0.5)),
    ((10, 8, 6), 43, dict(Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)),
    ((7, 9, 5), 44, dict(Re=10.0, Bi=3.0, Pa=1e4, nexp=0.8)),
])
def test_explicit_stages_match_oracle(harness, tmp_path, n, seed, over):
    cfg = cavity(n, **over)
    d = len(cfg["n"])
    u, p = random_state(cfg["n"], seed=seed)
    g = Grid(cfg["n"], cfg["h"], wall_u=cfg["wall_u"])
    rh = Rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    dt = cfg["dt"]
    ref = step(g, u, p, dt, rh, keep=True)

    wu = np.zeros((3, 2, 3))
    wu[:d, :, :d] = np.asarray(cfg["wall_u"], dtype=np.float64).reshape(d, 2, d)
    nn = list(cfg["n"]) + [1] * (3 - d)
    src = tmp_path / "in.bin"
    with open(src, "wb") as f:
        np.array([d, *nn, 0], dtype=np.int32).tofile(f)
        np.array([cfg["h"], dt, 1.0, cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"], 0.0, 0.0, 0.0],
                 dtype=np.float64).tofile(f)
        wu.ravel().tofile(f)
        to_device_layout(u).tofile(f)
        to_device_layout(p).tofile(f)
        to_device_layout(ref.ustar).tofile(f)
    dst = tmp_path / "out.bin"
    r = subprocess.run([harness, str(src), str(dst)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    out = np.fromfile(dst, dtype=np.float64)

    shape = tuple(cfg["n"])
    ncell = int(np.prod(shape))
    pos = 0

    def take(count):
        nonlocal pos
        v = out[pos:pos + count]
        pos += count
        return v

    eta = from_device_layout(take(ncell), shape, 1)[0]
    Gp = from_device_layout(take(d * ncell), shape, d)
    Lu = from_device_layout(take(d * ncell), shape, d)
    assert rel_l2(eta, ref.eta) < 1e-13
    assert rel_l2(Gp, ref.Gp) < TOL
    assert rel_l2(Lu, ref.Lu) < TOL
    for a in range(d):
        fshape = tuple(v + (1 if b == a else 0) for b, v in enumerate(shape))
        nf = int(np.prod(fshape))
        uL = from_device_layout(take(d * nf), fshape, d)
        uR = from_device_layout(take(d * nf), fshape, d)
        ua = from_device_layout(take(nf), fshape, 1)[0]
        assert rel_l2(uL, ref.uL[a]) < TOL, a
        assert rel_l2(uR, ref.uR[a]) < TOL, a
        assert rel_l2(ua, ref.uadv[a]) < TOL, a
    nshape = tuple(v + 1 for v in shape)
    nrhs = from_device_layout(take(int(np.prod(nshape))), nshape, 1)[0]
    assert rel_l2(nrhs, ref.rhs_nod) < TOL
    assert pos == out.size
