"""The learned initial guess in the nodal projection (Eq. 17): trained by the
library's own kernels on (warm-start residual, correction) pairs the solver
generates, it changes only the multigrid's starting point.  This test trains a
small model, then advances held-out cavities in lockstep with and without it
from identical states, and checks that (a) the solves still reach the same
tolerance and agree, (b) the guess is accepted at most steps and (c) the total
number of nodal V-cycles stays within a few per cent of the plain method's (a
guess with a smaller residual need not save a whole cycle).  It prints the
V-cycles saved."""

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
    assert with_ <= without + max(2, without // 20)


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
    assert with_ <= without + max(2, without // 20)
