"""Host logic of the binding: arrays indexed [i, j(, k)] go to the library's
flat x-fastest, component-major layout and back unchanged."""

import numpy as np
import pytest

from paper_1803_00417_gb300.hbflow import from_device_layout, to_device_layout


@pytest.mark.parametrize("shape", [(5, 3), (4, 3, 2), (1, 7), (3, 1, 4)])
def test_layout_round_trip(shape):
    rng = np.random.default_rng(len(shape))
    d = len(shape)
    u = [rng.standard_normal(shape) for _ in range(d)]
    flat = to_device_layout(u)
    assert flat.shape == (d * int(np.prod(shape)),)
    back = from_device_layout(flat, shape, d)
    for a, b in zip(u, back):
        assert np.array_equal(a, b)


def test_x_is_fastest():
    a = np.arange(24, dtype=np.float64).reshape(2, 3, 4)  # a[i, j, k]
    flat = to_device_layout(a)
    # flat index i + 2 (j + 3 k)
    for i in range(2):
        for j in range(3):
            for k in range(4):
                assert flat[i + 2 * (j + 3 * k)] == a[i, j, k]
