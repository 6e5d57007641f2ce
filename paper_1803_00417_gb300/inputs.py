"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the method: it only builds grids'
parameters and pseudo-random smooth fields.  Arrays are indexed ``[i, j(, k)]``
with numpy axis ``a`` = spatial direction ``a``.

Workloads (lid-driven cavities of Sec. IV / V C; dimensionless units
rho = U = L = 1, K = 2^(1-n)/Re, tau_y = Bi/Re, m = Pa):

* ``cavity64_bingham``  2D 64^2,  n=1,   Re=1,    Bi=2,  m=1e4
* ``cavity1024_hb``     2D 1024^2, n=0.5, Re=1000, Bi=5,  m=1e5
* ``cavity256_3d_hb``   3D 256^3, n=1.5, Re=100,  Bi=10, m=1e5, lid +x on z=1
"""

import numpy as np

WORKLOADS = {
    "cavity64_bingham": dict(n=(64, 64), nexp=1.0, Re=1.0, Bi=2.0, Pa=1e4),
    "cavity1024_hb": dict(n=(1024, 1024), nexp=0.5, Re=1000.0, Bi=5.0, Pa=1e5),
    "cavity256_3d_hb": dict(n=(256, 256, 256), nexp=1.5, Re=100.0, Bi=10.0, Pa=1e5),
}


def rheology_params(Re, nexp, Bi, Pa):
    """(K, n, tau_y, m) from the dimensionless groups of Sec. IV."""
    return (2.0 ** (1.0 - nexp) / Re, nexp, Bi / Re, Pa)


def lid_walls(d, lid=1.0):
    """wall_u[axis][side][comp]: zero except the lid (top wall normal to the last
    axis) moving with ``lid`` along x."""
    w = np.zeros((d, 2, d))
    w[d - 1, 1, 0] = lid
    return w


def cavity(name_or_n, **over):
    """A cavity workload: dict with n, h, d, wall_u, rheology (K, n, tau_y, m),
    and dt = 0.5 h (CFL 0.5 against the unit lid speed)."""
    if isinstance(name_or_n, str):
        cfg = dict(WORKLOADS[name_or_n])
    else:
        cfg = dict(n=tuple(name_or_n), nexp=1.0, Re=1.0, Bi=2.0, Pa=1e4)
    cfg.update(over)
    n = tuple(cfg["n"])
    d = len(n)
    h = 1.0 / max(n)
    K, nexp, tau_y, m = rheology_params(cfg["Re"], cfg["nexp"], cfg["Bi"], cfg["Pa"])
    return dict(n=n, d=d, h=h, wall_u=lid_walls(d, cfg.get("lid", 1.0)), K=K, nexp=nexp,
                tau_y=tau_y, m=m, dt=cfg.get("cfl", 0.5) * h, periodic=(False,) * d)


def smooth_field(shape, seed, kmax=8, amp=1.0, centred=True):
    """Sum of random Fourier modes with |k| <= kmax evaluated at cell centres
    (``centred``) or nodes of a unit-spaced box of ``shape`` points."""
    rng = np.random.default_rng(seed)
    d = len(shape)
    L = [float(s) if centred else float(s - 1) for s in shape]
    axes = [(np.arange(s) + (0.5 if centred else 0.0)) / L[a] for a, s in enumerate(shape)]
    X = np.meshgrid(*axes, indexing="ij")
    out = np.zeros(shape)
    nmodes = 12
    for _ in range(nmodes):
        k = rng.integers(-kmax, kmax + 1, size=d)
        if not np.any(k):
            continue
        ph = rng.uniform(0, 2 * np.pi)
        a = rng.normal() / np.sqrt(1.0 + float(np.dot(k, k)))
        out += a * np.cos(2 * np.pi * sum(k[i] * X[i] for i in range(d)) + ph)
    s = np.max(np.abs(out))
    return amp * out / s if s > 0 else out


def random_state(n, seed, amp=1.0, pamp=1.0):
    """Seeded smooth velocity (d cell arrays) and nodal pressure for a box of
    ``n`` cells.  The velocity is the curl of a random stream function (2D) or
    vector potential (3D) sampled at cell centres times a wall envelope, so it
    is nearly divergence-free and small at the walls."""
    n = tuple(n)
    d = len(n)
    rng = np.random.default_rng(seed)
    axes = [(np.arange(s) + 0.5) / s for s in n]
    X = np.meshgrid(*axes, indexing="ij")
    env = np.ones(n)
    for a in range(d):
        env *= (X[a] * (1.0 - X[a])) * 4.0
    h = [1.0 / s for s in n]
    u = []
    seeds = rng.integers(0, 2**31, size=4)
    if d == 2:
        psi = env * smooth_field(n, int(seeds[0]))
        gx = np.gradient(psi, h[0], axis=0)
        gy = np.gradient(psi, h[1], axis=1)
        u = [gy, -gx]
    else:
        A = [env * smooth_field(n, int(seeds[i])) for i in range(3)]
        dA = [[np.gradient(A[c], h[a], axis=a) for a in range(3)] for c in range(3)]
        u = [dA[2][1] - dA[1][2], dA[0][2] - dA[2][0], dA[1][0] - dA[0][1]]
    s = max(np.max(np.abs(c)) for c in u)
    u = [amp * c / s for c in u]
    p = pamp * smooth_field(tuple(v + 1 for v in n), int(seeds[3]), kmax=4, centred=False)
    return u, p


def batch_sweep(ncav=64, seed=0, sizes=(128, 256, 384, 512), bi=(0.0, 50.0), nexp=(0.3, 1.5), re=(1.0, 1000.0),
                pa=1e4):
    """A seeded parameter sweep of 2D lid-driven cavities: sizes drawn from
    ``sizes`` (square, cells per side), Bi uniform in ``bi``, n uniform in
    ``nexp``, Re log-uniform in ``re``, fixed m = ``pa``.  Returns a list of
    :func:`cavity` dicts (each with its own dt = 0.5 h)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(ncav):
        s = int(rng.choice(sizes))
        b = float(rng.uniform(*bi))
        ne = float(rng.uniform(*nexp))
        r = float(np.exp(rng.uniform(np.log(re[0]), np.log(re[1]))))
        c = cavity((s, s), Re=r, Bi=b, Pa=pa, nexp=ne)
        c.update(Re=r, Bi=b)
        out.append(c)
    return out
