"""The learned-guess network's CUDA kernels (BF16 tensor-core convolutions with
FP32 accumulation, forward and backward) against the CPU reference network of
oracle/unet.py with the same BF16 rounding points, and training sanity."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle.unet as U  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_00417_gb300 import build

    build.build()


def to_gpu_params(params):
    out = []
    for k, (W, b) in enumerate(params):
        if k == 0:
            Wg = np.zeros(W.shape[:2] + (16,))
            Wg[:, :, 0] = W[:, :, 0]
        else:
            Wg = W
        out += [Wg.ravel(), np.asarray(b).ravel()]
    return np.concatenate(out).astype(np.float32)


def from_gpu_params(flat, d):
    convs, head = U.layer_shapes(d)
    nt = 3 ** d
    out, off = [], 0
    for k, (ci, co) in enumerate(convs):
        cg = 16 if k == 0 else ci
        W = flat[off:off + nt * co * cg].reshape(nt, co, cg).astype(np.float64)
        off += nt * co * cg
        b = flat[off:off + co].astype(np.float64)
        off += co
        out.append([W[:, :, :ci], b, W])
    Wh = flat[off:off + 16].reshape(1, 1, 16).astype(np.float64)
    off += 16
    bh = flat[off:off + 1].astype(np.float64)
    out.append([Wh, bh, Wh])
    return out


def spatial_to_flat(a):
    """oracle array (*n) indexed [i, j(, k)] -> flat x-fastest."""
    return np.ascontiguousarray(a.transpose(tuple(range(a.ndim))[::-1])).ravel()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


def make_case(d, seed):
    rng = np.random.default_rng(seed)
    n = (16, 16) if d == 2 else (8, 8, 8)
    params = U.init_params(d, seed=seed)
    for p in params:
        p[1] = p[1] + rng.normal(size=p[1].shape) * 0.05
        p[0] = p[0].astype(np.float32).astype(np.float64)
        p[1] = p[1].astype(np.float32).astype(np.float64)
    x = rng.normal(size=n)
    t = rng.normal(size=n)
    return n, params, x, t


@pytest.mark.parametrize("d", [2, 3])
def test_forward_matches_reference(d):
    from paper_1803_00417_gb300.hbflow import UNet

    n, params, x, _ = make_case(d, 5 + d)
    net = UNet(n, train=False)
    net.set_params(to_gpu_params(params))
    xd = torch.tensor(spatial_to_flat(x).astype(np.float32), device="cuda")
    yd = torch.empty_like(xd)
    net.forward(xd, yd)
    torch.cuda.synchronize()
    y_ref = U.forward(params, U.bf16(x)[..., None])[..., 0]
    err = rel(yd.cpu().numpy(), spatial_to_flat(y_ref))
    assert err < 2e-2, err
    net.close()


@pytest.mark.parametrize("d", [2, 3])
def test_gradients_match_reference(d):
    from paper_1803_00417_gb300.hbflow import UNet

    n, params, x, t = make_case(d, 11 + d)
    net = UNet(n, train=True)
    net.set_params(to_gpu_params(params))
    xd = torch.tensor(spatial_to_flat(x).astype(np.float32), device="cuda")
    td = torch.tensor(spatial_to_flat(t).astype(np.float32), device="cuda")
    md = torch.ones_like(xd)
    gy = torch.empty_like(xd)
    net.zero_grads()
    net.forward(xd)
    loss_gpu = net.loss(td, md, gy)
    net.backward(gy)
    g_gpu = from_gpu_params(net.get_grads(), d)
    y_ref, tape = U.forward(params, U.bf16(x)[..., None], keep=True)
    loss_ref, gy_ref = U.mse_loss(y_ref, t[..., None], np.ones(n + (1,)))
    g_ref = U.backward(params, tape, gy_ref)
    assert loss_gpu == pytest.approx(loss_ref, rel=2e-2)
    for k in range(len(params)):
        for w in (0, 1):
            e = rel(g_gpu[k][w], g_ref[k][w])
            assert e < 6e-2, (k, w, e)
    # the first layer's unused (padded) input channels get exactly zero gradient
    assert np.all(g_gpu[0][2][:, :, 1:] == 0.0)
    net.close()


def test_training_reduces_loss():
    from paper_1803_00417_gb300.hbflow import UNet
    from paper_1803_00417_gb300.learned import train

    rng = np.random.default_rng(3)
    n = (16, 16)
    xs, ys = [], []
    for _ in range(8):
        x = rng.normal(size=n)
        # a smooth, linear target: a few Jacobi-like averages of the input
        y = x.copy()
        for _ in range(3):
            y = 0.25 * (np.roll(y, 1, 0) + np.roll(y, -1, 0) + np.roll(y, 1, 1) + np.roll(y, -1, 1))
        xs.append(spatial_to_flat(x).astype(np.float32))
        ys.append(spatial_to_flat(y).astype(np.float32))
    net = UNet(n, train=True, seed=1)
    hist = train(net, np.array(xs), np.array(ys), np.ones(256, dtype=np.float32), epochs=25, lr=2e-3, batch=2)
    assert hist[-1] < 0.5 * hist[0], hist
    net.close()


@pytest.mark.parametrize("d", [2, 3])
def test_tcgen05_path_matches(d):
    """The tcgen05 convolutions (TMEM accumulators) give the forward pass and
    the gradients of the mma.sync path and of the CPU reference network."""
    from paper_1803_00417_gb300.hbflow import UNet

    n, params, x, t = make_case(d, 21 + d)
    xd = torch.tensor(spatial_to_flat(x).astype(np.float32), device="cuda")
    td = torch.tensor(spatial_to_flat(t).astype(np.float32), device="cuda")
    md = torch.ones_like(xd)
    outs, grads = [], []
    for path in (0, 1):
        net = UNet(n, train=True)
        net.set_tensor_path(path)
        net.set_params(to_gpu_params(params))
        yd = torch.empty_like(xd)
        gy = torch.empty_like(xd)
        net.zero_grads()
        net.forward(xd, yd)
        net.loss(td, md, gy)
        net.backward(gy)
        net.tensor_status()
        outs.append(yd.cpu().numpy())
        grads.append(net.get_grads())
        net.close()
    y_ref = U.forward(params, U.bf16(x)[..., None])[..., 0]
    assert rel(outs[1], spatial_to_flat(y_ref)) < 2e-2
    assert rel(outs[1], outs[0]) < 1e-2
    assert rel(grads[1], grads[0]) < 3e-2
