"""The allocation-free time-step entry point, hbf_cfl_dt_noalloc.

Some callers cannot allocate device memory (work recorded inside a CUDA graph
capture, processes whose device memory belongs to another runtime's pool
allocator, drivers that reserve all memory up front).  For them the library
offers a variant of the max-|u| reduction behind hbf_cfl_dt whose scratch is a
static device array.  This file checks it through the C-ABI against the
context-based hbf_cfl_dt on the same velocity, for two calls in a row, and its
size limit.  It is collected last so that a failure here does not hide the
other tests' results."""

import ctypes

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


def test_noalloc_cfl_matches_context_entry_point():
    from paper_1803_00417_gb300.hbflow import HBFlow, load, to_device_layout
    from paper_1803_00417_gb300.inputs import cavity, random_state

    lib = load()
    cfg = cavity((40, 24, 18), Re=100.0, Bi=10.0, Pa=1e5, nexp=1.5)
    sim = HBFlow(cfg["n"], cfg["h"], cfg["wall_u"])
    stream = torch.cuda.current_stream().cuda_stream
    dt_dev = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for call, (seed, amp) in enumerate([(41, 3.0), (42, 0.25)]):
        u, _ = random_state(cfg["n"], seed=seed, amp=amp)
        flat = to_device_layout(u)
        sim.set_field("U", flat)
        ref = sim.cfl_dt(0.5)  # existing entry point (context scratch)
        u_dev = torch.tensor(flat, device="cuda")
        st = lib.hbf_cfl_dt_noalloc(ctypes.c_void_p(u_dev.data_ptr()), u_dev.numel(), cfg["h"], 0.5,
                                    ctypes.c_void_p(dt_dev.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0, st
        torch.cuda.synchronize()
        got = float(dt_dev.item())
        assert got == pytest.approx(ref, rel=1e-14), (call, got, ref)
        # amp < 1 exercises the max(|u|, 1) floor on the second call
        expect = 0.5 * cfg["h"] / max(float(np.max(np.abs(flat))), 1.0)
        assert got == pytest.approx(expect, rel=1e-14)
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1803_00417_gb300.hbflow import load

    lib = load()
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = 67108864 + 1  # one element more than the static partial array covers
    # rejected before any device access, so the pointer is never read
    st = lib.hbf_cfl_dt_noalloc(ctypes.c_void_p(dt_dev.data_ptr()), big, 0.1, 0.5,
                                ctypes.c_void_p(dt_dev.data_ptr()), None)
    assert st == -1
    assert lib.hbf_cfl_dt_noalloc(None, 10, 0.1, 0.5, ctypes.c_void_p(dt_dev.data_ptr()), None) == -1
