"""Pins for the reference U-Net of the learned initial guess: its backward
pass against central finite differences in exact FP64, the convolution
against a direct loop, and shape/adjoint identities of the grid transfers."""

import itertools

import numpy as np
import pytest

import oracle.unet as U


@pytest.fixture
def exact():
    U.ROUND_BF16 = False
    yield
    U.ROUND_BF16 = True


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -3.14159, 1e-30])
    r = U.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0            # tie -> even (mantissa ...0)
    assert r[2] == 1.0 + 2 ** -7                  # representable
    assert r[3] == 1.0 + 2 ** -6                  # tie -> even (rounds up)
    assert abs(r[4] + 3.140625) < 1e-12
    assert r[5] > 0


@pytest.mark.parametrize("d", [2, 3])
def test_conv_matches_direct_loop(d, exact):
    rng = np.random.default_rng(d)
    n = (5,) * d
    x = rng.normal(size=n + (3,))
    W = rng.normal(size=(3 ** d, 4, 3))
    b = rng.normal(size=4)
    out = U.conv(x, W, b)
    for p in itertools.product(*[range(s) for s in n]):
        ref = b.copy()
        for t, off in enumerate(U.taps(d)):
            q = tuple(p[a] + off[a] for a in range(d))
            if all(0 <= q[a] < n[a] for a in range(d)):
                ref += W[t] @ x[q]
        np.testing.assert_allclose(out[p], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_transfers_are_adjoint(d, exact):
    rng = np.random.default_rng(10 + d)
    n = (4,) * d
    x = rng.normal(size=n + (2,))
    y = rng.normal(size=tuple(v // 2 for v in n) + (2,))
    # <pool x, y> = <x, pool^T y> and <up y, x> = <y, up^T x>
    assert np.sum(U.pool(x) * y) == pytest.approx(np.sum(x * U.pool_backward(y)), rel=1e-12)
    assert np.sum(U.upsample(y) * x) == pytest.approx(np.sum(y * U.upsample_backward(x)), rel=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_backward_matches_finite_differences(d, exact):
    rng = np.random.default_rng(20 + d)
    n = (8,) * d
    params = U.init_params(d, seed=3)
    for W, b in params:
        b += rng.normal(size=b.shape) * 0.1
    x = rng.normal(size=n + (1,))
    t = rng.normal(size=n + (1,))
    mask = np.ones(n + (1,))
    y, tape = U.forward(params, x, keep=True)
    loss, gy = U.mse_loss(y, t, mask)
    grads = U.backward(params, tape, gy)
    eps = 1e-6
    checked = 0
    for k in (0, 3, 7, 9, 13, 14):  # first, encoder, bottleneck, decoder, last conv, head
        for which in (0, 1):
            arr = params[k][which]
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp, _ = U.mse_loss(U.forward(params, x), t, mask)
                flat[idx] = old - eps
                lm, _ = U.mse_loss(U.forward(params, x), t, mask)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                an = grads[k][which].reshape(-1)[idx]
                assert an == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, which, idx)
                checked += 1
    assert checked >= 40
