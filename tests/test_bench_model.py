"""The roofline model bench.py reports: algorithmic bytes of one finest-level
launch of the viscous smoother (one component, one colour), counted by hand
from the kernel's reads and writes."""

import pytest

pytest.importorskip("numpy")

import bench  # noqa: E402


def test_smoother_bytes_cell_viscosity_fp32_3d():
    # other colour of u_c 1/2, two other components 2, eta 1, b_c of the
    # colour 1/2, u_c of the colour written 1/2: 4.5 floats per cell
    assert bench.visc_smoother_bytes(3, 1000, 4, True) == pytest.approx(18.0 * 1000)


def test_smoother_bytes_face_arrays():
    # FP64 with three face arrays: (1/2 + 2 + 1/2 + 3 + 1/2) doubles per cell
    assert bench.visc_smoother_bytes(3, 10, 8, False) == pytest.approx(52.0 * 10)
    # 2D FP32 with two face arrays: (1/2 + 1 + 1/2 + 2 + 1/2) floats
    assert bench.visc_smoother_bytes(2, 10, 4, False) == pytest.approx(18.0 * 10)


def test_traffic_per_cell_from_capture():
    # the DRAM bytes per cell taken from the 192^3 capture
    # (profiles/k_visc_smooth_cavity192.md: 144.2 MB read + 15.1 MB written)
    assert bench.SMOOTHER_DRAM_BYTES_PER_CELL == pytest.approx(22.5, abs=0.05)


def test_fused_sweep_bytes():
    # u_c, two other components, eta, b_c read once, u_c written once
    assert bench.fused_sweep_bytes(3, 1000, 4) == pytest.approx(24.0 * 1000)
