"""The C-ABI library builds, loads and exports every entry point that
include/hbflow.h declares (no compute call: no GPU needed)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hbflow.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hbf_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_00417_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_step_boundary():
    names = _declared()
    for required in ("hbf_init_grid", "hbf_set_rheology", "hbf_step", "hbf_solve_viscous", "hbf_project"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    from paper_1803_00417_gb300.hbflow import SIGNATURES

    assert set(SIGNATURES) == set(_declared())


def test_argument_errors_need_no_gpu(lib):
    from paper_1803_00417_gb300 import hbflow

    L = hbflow.load()
    ctx = ctypes.c_void_p()
    n = (ctypes.c_int64 * 3)(8, 8, 1)
    # invalid dimension and size are rejected before any CUDA call
    assert L.hbf_init_grid(ctypes.byref(ctx), 4, n, 0.1, None, 0, None) == -1
    n_bad = (ctypes.c_int64 * 3)(1, 8, 1)
    assert L.hbf_init_grid(ctypes.byref(ctx), 2, n_bad, 0.1, None, 0, None) == -1
    assert L.hbf_init_grid(ctypes.byref(ctx), 2, n, -1.0, None, 0, None) == -1
    assert L.hbf_step(None, 0.1, None) == -1


def test_header_is_plain_c(tmp_path):
    """The boundary is a C header: it compiles as C99 and as C++ on its own."""
    import shutil
    import subprocess

    src = tmp_path / "use.c"
    src.write_text('#include "hbflow.h"\nint main(void) { return hbf_set_tail((hbf_ctx*)0, 0) == 0; }\n')
    inc = os.path.join(ROOT, "include")
    for cc, std in (("gcc", "-std=c99"), ("g++", "-std=c++17")):
        if shutil.which(cc) is None:
            pytest.skip(cc + " not found")
        lang = ["-x", "c++"] if cc == "g++" else []
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, *lang, "-c", str(src),
                            "-o", str(tmp_path / ("use_" + cc + ".o"))], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
