"""Training driver of the learned initial guess (marshalling only: the data
come from the library's solver, the network runs in the library's kernels).

Pairs (x, y) for the nodal projection solve of Eq. 17: x = r0 / |r0|_inf with
r0 = b - L p^{m-1/2} the warm-start residual, y = d / |d|_inf with
d = phi - p^{m-1/2} the correction the multigrid found.  The network learns the
direction of the correction; the library scales it by a least-squares step.  Both live on the (n+1)^d nodes and are
zero-padded to the network's box (multiples of 8)."""

import numpy as np

from .hbflow import HBFlow, UNet, from_device_layout
from .inputs import cavity, rheology_params


def net_box(n):
    """Smallest box of multiples of 8 holding the (n+1)^d nodes."""
    return tuple(((v + 1 + 7) // 8) * 8 for v in n)


def nodes_to_box(a_nodes, n, box):
    """Flat node array (x fastest, (n+1)^d) -> flat box array (x fastest)."""
    d = len(n)
    shp = tuple(v + 1 for v in n)
    arr = np.asarray(a_nodes, dtype=np.float64).reshape(shp[::-1])
    out = np.zeros(box[::-1], dtype=np.float32)
    out[tuple(slice(0, s) for s in shp[::-1])] = arr
    return out.ravel()


def coarse_cells(n, level):
    """Cells per axis of multigrid level ``level`` (halved per level)."""
    return tuple(v >> level for v in n)


def restrict_nodes(a_nodes, n):
    """Nodal full weighting onto the next coarser level (as the multigrid's
    nodal restriction): along x, then y, then z, coarse node I takes
    1/2 of fine node 2I and 1/4 of each of 2I - 1, 2I + 1, with the fine nodes
    beyond a wall mirrored back inside.  Flat x-fastest arrays; returns the
    coarse array and its cell counts."""
    d = len(n)
    shp = tuple(v + 1 for v in n)
    arr = np.asarray(a_nodes, dtype=np.float64).reshape(shp[::-1])
    for a in range(d):
        ax = d - 1 - a  # numpy axis of spatial axis a (x fastest = last)
        m = n[a]
        lo = np.abs(np.arange(0, m + 1, 2) - 1)
        hi = np.arange(0, m + 1, 2) + 1
        hi = np.where(hi > m, 2 * m - hi, hi)
        cen = np.take(arr, np.arange(0, m + 1, 2), axis=ax)
        arr = 0.5 * cen + 0.25 * (np.take(arr, lo, axis=ax) + np.take(arr, hi, axis=ax))
    return arr.ravel(), coarse_cells(n, 1)


def box_mask(n, box):
    return nodes_to_box(np.ones(int(np.prod([v + 1 for v in n]))), n, box)


def sample_params(rng, bi_max=20.0):
    """Bi ~ U[0, bi_max], n ~ U[0.5, 1.5], Re = 10^U[0,3] (dimensionless groups
    of Sec. IV), Pa = 1e4."""
    return dict(Re=10.0 ** rng.uniform(0, 3), nexp=rng.uniform(0.5, 1.5), Bi=rng.uniform(0, bi_max), Pa=1e4)


def generate_pairs(n, seeds, steps, skip=1, precision=0, stream=None, level=0):
    """Run cavities from rest with seeded random rheology and collect the
    nodal-solve pairs of every ``skip``-th step after the first, restricted to
    multigrid level ``level`` (the level the network will run on)."""
    import torch

    nL = coarse_cells(n, level)
    box = net_box(nL)
    xs, ys, info = [], [], []
    for seed in seeds:
        rng = np.random.default_rng(seed)
        cfg = cavity(tuple(n), **sample_params(rng))
        sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=precision, stream=stream)
        sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
        d = len(n)
        nn = int(np.prod(cfg["n"]))
        sim.set_field("U", np.zeros(d * nn))
        sim.set_field("P", np.zeros(int(np.prod([v + 1 for v in cfg["n"]]))))
        for s in range(steps):
            p_old = sim.get_field("P").copy()
            st = sim.step(cfg["dt"])
            if s >= 1 and (s - 1) % skip == 0:
                r0 = sim.get_field("NRES0")
                p_new = sim.get_field("P")
                nrm = float(np.max(np.abs(r0)))
                dphi = p_new - p_old
                rc, dc, nc = r0, dphi, tuple(n)
                for _ in range(level):
                    rc, _n = restrict_nodes(rc, nc)
                    dc, nc = restrict_nodes(dc, nc)
                dn = float(np.max(np.abs(dc)))
                if nrm > 0 and dn > 0:
                    xs.append(nodes_to_box(rc / nrm, nc, box))
                    ys.append(nodes_to_box(dc / dn, nc, box))
                    info.append(dict(seed=seed, step=s, cycles=st["nodal"]["cycles"]))
        sim.close()
    return np.array(xs), np.array(ys), info


def train(net, xs, ys, mask, epochs=20, lr=1e-3, batch=4, seed=0, log=None):
    """Adam on the masked MSE; returns the loss history (mean per epoch)."""
    import torch

    rng = np.random.default_rng(seed)
    dev = "cuda"
    m = torch.tensor(mask, device=dev)
    gy = torch.empty(net.points, dtype=torch.float32, device=dev)
    X = torch.tensor(xs, device=dev)
    Y = torch.tensor(ys, device=dev)
    hist = []
    net.zero_grads()
    for ep in range(epochs):
        order = rng.permutation(len(xs))
        tot = 0.0
        for q, i in enumerate(order):
            net.forward(X[i])
            tot += net.loss(Y[i], m, gy)
            net.backward(gy)
            if (q + 1) % batch == 0 or q == len(order) - 1:
                net.adam(lr=lr)
        hist.append(tot / len(xs))
        if log:
            log(ep, hist[-1])
    return hist
