"""The colour-split layout of the FP32 finest level of the mixed viscous solve
(Eq. 16's operator and its red-black Gauss-Seidel smoother), built for the
host: its per-slot functions give the natural-layout functions' results bit
for bit on seeded fields (sweeps, operator, transfers, conversions), and its
slot map visits every cell of a colour once.  No GPU needed."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1803_00417_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("split") / "split_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-I", CSRC,
                    os.path.join(HERE, "host", "split_check.cu"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return exe


# the smallest grid the layout takes, ragged odd y/z extents (no transfers),
# even grids with the coarse level, both wall conditions, more than 32 rows
# per plane (several x-wall warps, the last one partial), rows longer than one
# block's 256 threads (two segments), and rows of even length n0 / 2, where the
# sweep's 8-byte pair gather is checked too
@pytest.mark.parametrize("n,hom,seed", [((4, 3, 3), 0, 1), ((8, 6, 4), 0, 2), ((8, 6, 4), 1, 3),
                                        ((12, 7, 9), 0, 4), ((10, 5, 3), 1, 5), ((16, 16, 16), 0, 6),
                                        ((6, 9, 12), 1, 7), ((20, 8, 6), 0, 8), ((18, 70, 14), 1, 9),
                                        ((600, 5, 4), 0, 10), ((24, 10, 8), 1, 15), ((1100, 4, 3), 1, 11)])
def test_split_layout_matches_natural_bit_for_bit(harness, n, hom, seed):
    r = subprocess.run([harness, *map(str, n), str(hom), str(seed)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
