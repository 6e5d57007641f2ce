"""Training driver of the learned initial guesses (marshalling only: the data
come from the library's solver, the restriction to a coarse level is the
library's multigrid restriction, the network runs in the library's kernels).

Nodal projection (Eq. 17): pairs (x, y) with x = r0 / |r0|_inf, r0 = b - L
p^{m-1/2} the warm-start residual, and y = d / |d|_inf, d = phi - p^{m-1/2}
the correction the multigrid found; both on the (n+1)^d nodes of the chosen
level.  Viscous solve (Eq. 16): per velocity component, x = the residual at
the start of the solve (after the previous-increment step) / its max norm
over all components, y = the correction the solver found / its max norm; on
the n^d cells of the chosen level.  The network learns the direction of the
correction; the library scales it by a least-squares step.  Arrays are
zero-padded to the network's box (multiples of 8)."""

import numpy as np

from .hbflow import HBFlow
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


def box_mask(n, box):
    return nodes_to_box(np.ones(int(np.prod([v + 1 for v in n]))), n, box)


def cell_mask(n, box):
    return cells_to_box(np.ones(int(np.prod(n))), n, box)


def sample_params(rng, bi_max=20.0):
    """Bi ~ U[0, bi_max], n ~ U[0.5, 1.5], Re = 10^U[0,3] (dimensionless groups
    of Sec. IV), Pa = 1e4."""
    return dict(Re=10.0 ** rng.uniform(0, 3), nexp=rng.uniform(0.5, 1.5), Bi=rng.uniform(0, bi_max), Pa=1e4)


def restrict_down(sim, kind, flat, level):
    """A flat field restricted ``level`` times by the library's multigrid
    restriction (kind 0 cell vector, 1 cell scalar, 2 nodes)."""
    import torch

    cur = torch.tensor(flat, device="cuda")
    n = sim.n
    d = len(n)
    for l in range(level):
        n = tuple(v // 2 for v in n)
        cnt = (d if kind == 0 else 1) * int(np.prod(n)) if kind != 2 else int(np.prod([v + 1 for v in n]))
        nxt = torch.empty(cnt, dtype=torch.float64, device="cuda")
        sim.restrict(kind, l, cur, nxt)
        cur = nxt
    torch.cuda.synchronize()
    return cur.cpu().numpy()


def cells_to_box(a_cells, n, box):
    """Flat cell array (x fastest, n^d) -> flat box array (x fastest)."""
    arr = np.asarray(a_cells, dtype=np.float64).reshape(tuple(n)[::-1])
    out = np.zeros(box[::-1], dtype=np.float32)
    out[tuple(slice(0, s) for s in tuple(n)[::-1])] = arr
    return out.ravel()


def cell_box(n):
    """Smallest box of multiples of 8 holding the n^d cells."""
    return tuple(((v + 7) // 8) * 8 for v in n)


def generate_pairs(n, seeds, steps, skip=1, precision=0, stream=None, level=0):
    """Run cavities from rest with seeded random rheology and collect the
    nodal-solve pairs of every ``skip``-th step after the first, restricted to
    multigrid level ``level`` (the level the network will run on)."""
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
                rc = restrict_down(sim, 2, r0, level)
                dc = restrict_down(sim, 2, p_new - p_old, level)
                nrm = float(np.max(np.abs(rc)))
                dn = float(np.max(np.abs(dc)))
                if nrm > 0 and dn > 0:
                    xs.append(nodes_to_box(rc / nrm, nL, box))
                    ys.append(nodes_to_box(dc / dn, nL, box))
                    info.append(dict(seed=seed, step=s, cycles=st["nodal"]["cycles"]))
        sim.close()
    return np.array(xs), np.array(ys), info


def generate_visc_pairs(n, seeds, steps, skip=1, stream=None, level=0):
    """Run mixed-precision cavities from rest with seeded random rheology and
    the previous-increment guess on, and collect the viscous-solve pairs of
    every ``skip``-th step after the second (one pair per velocity component),
    restricted to multigrid level ``level``."""
    from .hbflow import MIXED

    nL = coarse_cells(n, level)
    box = cell_box(nL)
    d = len(n)
    ncL = int(np.prod(nL))
    xs, ys, info = [], [], []
    for seed in seeds:
        rng = np.random.default_rng(seed)
        cfg = cavity(tuple(n), **sample_params(rng))
        sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED, stream=stream)
        sim.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
        sim.set_visc_guess(1)
        sim.set_visc_record(True)
        nn = int(np.prod(cfg["n"]))
        sim.set_field("U", np.zeros(d * nn))
        sim.set_field("P", np.zeros(int(np.prod([v + 1 for v in cfg["n"]]))))
        for s in range(steps):
            st = sim.step(cfg["dt"])
            if s >= 2 and (s - 2) % skip == 0:
                rc = restrict_down(sim, 0, sim.get_field("VRES0"), level)
                dc = restrict_down(sim, 0, sim.get_field("VCORR"), level)
                nrm = float(np.max(np.abs(rc)))
                dn = float(np.max(np.abs(dc)))
                if nrm > 0 and dn > 0:
                    for q in range(d):
                        xs.append(cells_to_box(rc[q * ncL:(q + 1) * ncL] / nrm, nL, box))
                        ys.append(cells_to_box(dc[q * ncL:(q + 1) * ncL] / dn, nL, box))
                    info.append(dict(seed=seed, step=s, iterations=st["visc"]["cycles"]))
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
