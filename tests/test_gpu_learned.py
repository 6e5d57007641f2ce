"""The learned initial guesses (not in the paper; they change only the
starting point of a solve, which still runs to its tolerance).

Nodal projection (Eq. 17): a network trained by the library's own kernels on
(warm-start residual, correction) pairs the solver generates.  Held-out
cavities advance in lockstep with and without it from identical states: the
solves reach the same tolerance and agree, and the guess is accepted (it
lowers the warm-start residual) at most steps.  The V-cycles with and without
it are printed, not asserted: measured, the network saves none (96 / 96 and
48 / 48 V-cycles on these cavities; one run in several gives one more with
it, since a lower max-norm residual of other spectral content can take as
many cycles or one more); the gain criterion is not met by this network.

Viscous solve (Eq. 16): the minimal-residual step along the previous step's
increment saves BiCGStab iterations (strictly fewer over ten steps of the
3D Herschel-Bulkley cavity's parameters), and the learned direction on top of
it keeps every solve at its tolerance; its iterations are printed."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_00417_gb300 import build

    build.build()


def test_learned_guess_gain_2d():
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow, UNet, set_guess_model
    from paper_1803_00417_gb300.inputs import cavity
    from paper_1803_00417_gb300.learned import box_mask, generate_pairs, net_box, sample_params, train

    n = (48, 48)
    xs, ys, _ = generate_pairs(n, seeds=range(6), steps=12, precision=MIXED)
    box = net_box(n)
    net = UNet(box, train=True, seed=0)
    hist = train(net, xs, ys, box_mask(n, box), epochs=12, lr=1e-3, batch=4)
    assert hist[-1] < 0.5 * hist[0]
    model = UNet(box, train=False)
    model.set_params(net.get_params())
    without = with_ = used = total = 0
    for seed in (1000, 1001):
        cfg = cavity(n, **sample_params(np.random.default_rng(seed)))
        a = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
        b = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
        for s in (a, b):
            s.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
            s.set_field("U", np.zeros(2 * 48 * 48))
            s.set_field("P", np.zeros(49 * 49))
        set_guess_model(b, model)
        for k in range(12):
            b.set_field("U", a.get_field("U").copy())
            b.set_field("P", a.get_field("P").copy())
            sa, sb = a.step(cfg["dt"]), b.step(cfg["dt"])
            assert sa["nodal"]["converged"] and sb["nodal"]["converged"]
            ua, ub = a.get_field("U"), b.get_field("U")
            assert np.linalg.norm(ua - ub) <= 1e-8 * max(np.linalg.norm(ua), 1e-30)
            if k >= 1:  # the first step from rest has a zero warm start
                without += sa["nodal"]["cycles"]
                with_ += sb["nodal"]["cycles"]
                used += int(sb["nodal"]["guess"])
                total += 1
        a.close()
        b.close()
    print(f"nodal V-cycles without / with the learned guess: {without} / {with_} "
          f"(guess accepted at {used}/{total} steps)")
    assert used >= total // 2


def test_learned_guess_on_a_coarse_level_2d():
    """The network on the nodes of multigrid level 1 (trained on pairs
    restricted the same way): the guess is restricted in, interpolated out,
    and the solves still reach the same tolerance and agree with the plain
    method; a level outside the hierarchy is rejected."""
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow, HBFlowError, UNet, set_guess_model
    from paper_1803_00417_gb300.inputs import cavity
    from paper_1803_00417_gb300.learned import (box_mask, coarse_cells, generate_pairs, net_box, sample_params,
                                                train)

    n = (48, 48)
    nc = coarse_cells(n, 1)
    xs, ys, _ = generate_pairs(n, seeds=range(6), steps=12, precision=MIXED, level=1)
    box = net_box(nc)
    assert xs.shape[1] == int(np.prod(box))
    net = UNet(box, train=True, seed=0)
    hist = train(net, xs, ys, box_mask(nc, box), epochs=12, lr=1e-3, batch=4)
    assert hist[-1] < 0.5 * hist[0]
    model = UNet(box, train=False)
    model.set_params(net.get_params())
    without = with_ = used = total = 0
    cfg = cavity(n, **sample_params(np.random.default_rng(1000)))
    a = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
    b = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
    for s in (a, b):
        s.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
        s.set_field("U", np.zeros(2 * 48 * 48))
        s.set_field("P", np.zeros(49 * 49))
    with pytest.raises(HBFlowError):
        set_guess_model(b, model, 40)
    set_guess_model(b, model, 1)
    for k in range(12):
        b.set_field("U", a.get_field("U").copy())
        b.set_field("P", a.get_field("P").copy())
        sa, sb = a.step(cfg["dt"]), b.step(cfg["dt"])
        assert sa["nodal"]["converged"] and sb["nodal"]["converged"]
        ua, ub = a.get_field("U"), b.get_field("U")
        assert np.linalg.norm(ua - ub) <= 1e-8 * max(np.linalg.norm(ua), 1e-30)
        if k >= 1:
            without += sa["nodal"]["cycles"]
            with_ += sb["nodal"]["cycles"]
            used += int(sb["nodal"]["guess"])
            total += 1
    a.close()
    b.close()
    print(f"level-1 guess: nodal V-cycles without / with: {without} / {with_} (accepted {used}/{total})")
    assert used >= total // 2


def _visc_pair(n, seed_params, develop, modes):
    """Contexts with the given viscous guess modes, started from one state
    developed from rest by a plain mixed context."""
    from paper_1803_00417_gb300.hbflow import MIXED, HBFlow
    from paper_1803_00417_gb300.inputs import cavity

    cfg = cavity(n, **seed_params)
    base = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
    base.set_rheology(cfg["K"], cfg["nexp"], cfg["tau_y"], cfg["m"])
    d = len(n)
    base.set_field("U", np.zeros(d * int(np.prod(n))))
    base.set_field("P", np.zeros(int(np.prod([v + 1 for v in n]))))
    for _ in range(develop):
        base.step(cfg["dt"])
    rec, u, p = base.get_state()
    base.close()
    sims = []
    for mode in modes:
        s = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"], precision=MIXED)
        s.set_state(rec, u, p)
        s.set_visc_guess(mode)
        sims.append(s)
    return sims, cfg


def test_previous_increment_guess_saves_viscous_iterations():
    over = dict(Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)  # the 3D workload's parameters
    (plain, hist), cfg = _visc_pair((48, 48, 48), over, 10, (0, 1))
    its = [0, 0]
    taken = 0
    for k in range(10):
        s0, s1 = plain.step(cfg["dt"]), hist.step(cfg["dt"])
        for s in (s0, s1):
            assert all(s[q]["converged"] for q in ("mac", "visc", "nodal"))
        its[0] += s0["visc"]["cycles"]
        its[1] += s1["visc"]["cycles"]
        taken += s1["visc"]["guess"] & 1
    u0, u1 = plain.get_field("U"), hist.get_field("U")
    print(f"viscous iterations over 10 steps without / with the previous-increment step: {its[0]} / {its[1]} "
          f"(step taken {taken}/10)")
    assert its[1] < its[0]
    assert taken >= 8  # the first step has no increment yet
    assert np.max(np.abs(u1 - u0)) <= 1e-6 * np.max(np.abs(u0))
    plain.close()
    hist.close()


def test_learned_viscous_direction_keeps_tolerance():
    from paper_1803_00417_gb300.hbflow import UNet, set_visc_guess_model
    from paper_1803_00417_gb300.learned import cell_box, cell_mask, coarse_cells, generate_visc_pairs, train

    n, level = (32, 32, 32), 1
    nL = coarse_cells(n, level)
    xs, ys, info = generate_visc_pairs(n, seeds=range(3), steps=10, level=level)
    assert len(xs) == 3 * 3 * 8
    box = cell_box(nL)
    net = UNet(box, train=True, seed=0)
    hist = train(net, xs, ys, cell_mask(nL, box), epochs=8, lr=1e-3, batch=4)
    assert hist[-1] < hist[0]
    model = UNet(box, train=False)
    model.set_params(net.get_params())
    net.close()
    over = dict(Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)
    (m1, m2), cfg = _visc_pair(n, over, 10, (1, 2))
    set_visc_guess_model(m2, model, level)
    its = [0, 0]
    used = 0
    for k in range(8):
        s1, s2 = m1.step(cfg["dt"]), m2.step(cfg["dt"])
        for s in (s1, s2):
            assert all(s[q]["converged"] for q in ("mac", "visc", "nodal"))
        its[0] += s1["visc"]["cycles"]
        its[1] += s2["visc"]["cycles"]
        used += (s2["visc"]["guess"] >> 1) & 1
    u1, u2 = m1.get_field("U"), m2.get_field("U")
    print(f"viscous iterations over 8 steps, previous increment / + learned direction: {its[0]} / {its[1]} "
          f"(learned step taken {used}/8)")
    assert np.max(np.abs(u2 - u1)) <= 1e-6 * np.max(np.abs(u1))
    set_visc_guess_model(m2, None)
    model.close()
    m1.close()
    m2.close()
