"""Plain reference of the learned initial guess network (test infrastructure).

The paper has no learned component; this network is the initial-guess model
the task adds to the nodal projection solve (Sec. III A, Eq. 17).  Its
architecture is this project's reading of a "4-level U-Net, 16-32-64-128
channels, 3x3 convolutions, BF16 weights with FP32 accumulation":

    enc_l: conv3 -> ReLU -> conv3 -> ReLU          (l = 0..2, then the bottleneck)
    down:  2^d average pooling;  up: nearest upsampling, concatenate the skip
    dec_l: conv3 -> ReLU -> conv3 -> ReLU;  head: 1x1 conv, no activation

Tensors are channels-last numpy arrays (*spatial, C) in FP64.  ``bf16`` rounds
to bfloat16 (round to nearest even), applied where the CUDA path stores BF16:
weights, every activation that feeds a convolution, and the gradients that
feed the backward convolutions.  Arithmetic is FP64 otherwise.

Convolution taps are the 3^d offsets in lexicographic order (last axis
fastest); weights are laid out W[tap, c_out, c_in]; zero padding outside.
"""

import itertools

import numpy as np

CHANNELS = (16, 32, 64, 128)


ROUND_BF16 = True  # set False for exact FP64 (finite-difference checks)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    if not ROUND_BF16:
        return np.asarray(x, dtype=np.float64)
    a = np.asarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def taps(d):
    return list(itertools.product((-1, 0, 1), repeat=d))


def _shifted(x, off):
    """y[p] = x[p + off] with zeros outside (x: (*spatial, C))."""
    d = len(off)
    y = np.zeros_like(x)
    src = []
    dst = []
    for a in range(d):
        n = x.shape[a]
        o = off[a]
        if o >= 0:
            src.append(slice(o, n))
            dst.append(slice(0, n - o))
        else:
            src.append(slice(0, n + o))
            dst.append(slice(-o, n))
    y[tuple(dst)] = x[tuple(src)]
    return y


def conv(x, W, b):
    """out[p, co] = b[co] + sum_tap sum_ci x[p + off_tap, ci] W[tap, co, ci]."""
    d = x.ndim - 1
    out = np.zeros(x.shape[:-1] + (W.shape[1],)) + b
    for t, off in enumerate(taps(d)):
        out += _shifted(x, off) @ W[t].T
    return out


def conv_backward(x, W, g):
    """Gradients of conv for upstream g: (g_x, g_W, g_b)."""
    d = x.ndim - 1
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for t, off in enumerate(taps(d)):
        xs = _shifted(x, off)
        gW[t] = g.reshape(-1, g.shape[-1]).T @ xs.reshape(-1, xs.shape[-1])
        gx += _shifted(g @ W[t], tuple(-o for o in off))
    gb = g.reshape(-1, g.shape[-1]).sum(axis=0)
    return gx, gW, gb


def pool(x):
    d = x.ndim - 1
    out = x
    for a in range(d):
        idx0 = [slice(None)] * x.ndim
        idx1 = [slice(None)] * x.ndim
        idx0[a] = slice(0, None, 2)
        idx1[a] = slice(1, None, 2)
        out = 0.5 * (out[tuple(idx0)] + out[tuple(idx1)])
    return out


def pool_backward(g):
    d = g.ndim - 1
    out = g
    for a in range(d):
        out = np.repeat(out, 2, axis=a) * 0.5
    return out


def upsample(x):
    d = x.ndim - 1
    out = x
    for a in range(d):
        out = np.repeat(out, 2, axis=a)
    return out


def upsample_backward(g):
    d = g.ndim - 1
    out = g
    for a in range(d):
        idx0 = [slice(None)] * g.ndim
        idx1 = [slice(None)] * g.ndim
        idx0[a] = slice(0, None, 2)
        idx1[a] = slice(1, None, 2)
        out = out[tuple(idx0)] + out[tuple(idx1)]
    return out


def layer_shapes(d):
    """(c_in, c_out) of the 3^d convolutions in execution order, then the head."""
    c = CHANNELS
    convs = [(1, c[0]), (c[0], c[0]), (c[0], c[1]), (c[1], c[1]), (c[1], c[2]), (c[2], c[2]),
             (c[2], c[3]), (c[3], c[3]),
             (c[3] + c[2], c[2]), (c[2], c[2]), (c[2] + c[1], c[1]), (c[1], c[1]),
             (c[1] + c[0], c[0]), (c[0], c[0])]
    return convs, (c[0], 1)


def init_params(d, seed):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, FP64."""
    rng = np.random.default_rng(seed)
    convs, head = layer_shapes(d)
    nt = 3 ** d
    params = []
    for ci, co in convs:
        W = rng.normal(size=(nt, co, ci)) * np.sqrt(2.0 / (nt * ci))
        params.append([W, np.zeros(co)])
    Wh = rng.normal(size=(1, head[1], head[0])) * np.sqrt(1.0 / head[0])
    params.append([Wh, np.zeros(head[1])])
    return params


def forward(params, x, keep=False):
    """x: (*spatial, 1) input (spatial sizes divisible by 8).  Returns the
    (*spatial, 1) output and, with keep, the tape for backward."""
    P = [[bf16(W), b] for W, b in params]
    tape = []
    h = bf16(x)
    k = 0

    def block(h):
        nonlocal k
        for _ in range(2):
            W, b = P[k]
            z = conv(h, W, b)
            y = bf16(np.maximum(z, 0.0))
            tape.append((k, h, z))
            h = y
            k += 1
        return h

    skips = []
    for level in range(3):
        h = block(h)
        skips.append(h)
        h = bf16(pool(h))
    h = block(h)
    for level in (2, 1, 0):
        h = np.concatenate([bf16(upsample(h)), skips[level]], axis=-1)
        h = block(h)
    Wh, bh = P[k]
    y = h @ Wh[0].T + bh
    tape.append((k, h, None))
    if keep:
        return y, tape
    return y


def backward(params, tape, gy):
    """Gradients of every parameter for the upstream gradient gy of the output."""
    P = [[bf16(W), b] for W, b in params]
    grads = [None] * len(params)
    kh, hh, _ = tape[-1]
    Wh, _ = P[kh]
    grads[kh] = [(gy.reshape(-1, gy.shape[-1]).T @ hh.reshape(-1, hh.shape[-1]))[None],
                 gy.reshape(-1, gy.shape[-1]).sum(axis=0)]
    g = bf16(gy @ Wh[0])
    ti = len(tape) - 2
    # decoder blocks (levels 0, 1, 2 in reverse execution order), then the
    # bottleneck and encoder blocks
    skip_grads = {}

    def block_back(g):
        nonlocal ti
        for _ in range(2):
            k, hin, z = tape[ti]
            gz = g * (z > 0.0)
            gx, gW, gb = conv_backward(hin, P[k][0], gz)
            grads[k] = [gW, gb]
            g = bf16(gx)
            ti -= 1
        return g

    c = CHANNELS
    for level in (0, 1, 2):
        g = block_back(g)
        cu = g.shape[-1] - c[level]
        gup, gskip = g[..., :cu], g[..., cu:]
        skip_grads[level] = gskip
        g = bf16(upsample_backward(gup))
    g = block_back(g)
    for level in (2, 1, 0):
        g = bf16(pool_backward(g))
        g = bf16(g + skip_grads[level])
        g = block_back(g)
    return grads


def mse_loss(y, t, mask):
    """Mean over the masked points of (y - t)^2 and its gradient."""
    n = float(np.sum(mask))
    r = (y - t) * mask
    return float(np.sum(r * r) / n), 2.0 * r / n
