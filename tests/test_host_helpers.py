"""Host-side checks of device code that also compiles for the host: the FP64
comparisons and exact scalings done on bit patterns (against IEEE arithmetic,
bit for bit), the thread -> cell maps of the smoother and operator kernels
(every cell once), the viscous wall stencil's one-axis reflections (against
the general accessor, bit for bit), and the interior smoother and operator
with stored or cell-formed face viscosities (against the general point
forms).  Built with nvcc as a host program; no GPU needed."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1803_00417_gb300", "csrc")


def test_host_helpers(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "host_checks")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "host", "host_checks.cu"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().startswith("ok"), r.stdout
