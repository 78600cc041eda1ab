"""The C-ABI library loads and exports every symbol include/gkb.h declares.

No compute calls: these run without a GPU. The library is built on demand
(nvcc cross-compiles sm_103a without a device).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gkb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gkb_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2001_10424_gb300 import build
    return build.build()


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for n in ("gkb_create", "gkb_set_problem", "gkb_solve", "gkb_stats", "gkb_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    import paper_2001_10424_gb300 as gk
    assert sorted(gk.EXPORTED) == declared_functions()


def test_defaults_and_argument_errors_without_gpu(libpath):
    import paper_2001_10424_gb300 as gk
    gk.load(libpath)
    o = gk.gkb_default_options()
    assert o.precision == gk.GKB_PREC_FP64 and o.inner == gk.GKB_INNER_GMG_PCG
    assert o.maxit == 1000 and o.smoother_degree == 2
    lib = gk.load()
    assert lib.gkb_create(None, ctypes.byref(o)) == gk.GKB_ERR_INVALID_ARG
    bad = gk.gkb_default_options()
    bad.tol_inner = -1.0
    h = ctypes.c_void_p()
    assert lib.gkb_create(ctypes.byref(h), ctypes.byref(bad)) == gk.GKB_ERR_INVALID_ARG
    assert lib.gkb_solve(None, None, None, 1e-8, 5, None, None, None, None) == gk.GKB_ERR_INVALID_ARG
    assert lib.gkb_destroy(None) == gk.GKB_ERR_INVALID_ARG
    assert gk.gkb_last_error(None) == "invalid handle"


def test_binding_rejects_non_float64():
    import numpy as np
    import paper_2001_10424_gb300 as gk
    with pytest.raises(TypeError):
        gk._ptr(np.zeros(4, dtype=np.float32))
    with pytest.raises(TypeError):
        gk._ptr(np.zeros((4, 4))[:, 1])


def test_options_struct_layout_matches_the_header(libpath):
    """gkb_default_options zeroes exactly sizeof(gkb_options) bytes before
    filling the fields: over a larger buffer of 0xAB bytes the untouched tail
    shows the C size, which the ctypes mirror must equal (the struct ends in
    an int and padding, both zero)."""
    import paper_2001_10424_gb300 as gk
    lib = gk.load(libpath)
    buf = (ctypes.c_ubyte * 1024)(*([0xAB] * 1024))
    assert lib.gkb_default_options(ctypes.cast(buf, ctypes.POINTER(gk.gkb_options))) == gk.GKB_OK
    raw = bytes(buf)
    end = max(i for i, v in enumerate(raw) if v != 0xAB) + 1
    c_size = (end + 7) // 8 * 8
    assert c_size == ctypes.sizeof(gk.gkb_options)
    o = gk.gkb_options.from_buffer_copy(raw[:ctypes.sizeof(gk.gkb_options)])
    assert o.viscous_form == gk.GKB_VISC_LAPLACE and o.cheb_hi == 1.1 and o.fgmres_restart == 30


def test_header_constants_match_the_binding():
    import paper_2001_10424_gb300 as gk
    src = open(os.path.join(ROOT, "include", "gkb.h")).read()
    consts = dict((k, int(v)) for k, v in re.findall(r"#define\s+(GKB_[A-Z0-9_]+)\s+(-?\d+)\b", src))
    assert "GKB_VISC_SYMGRAD" in consts and "GKB_INNER_FGMRES" in consts
    for name, val in consts.items():
        if hasattr(gk, name):
            assert getattr(gk, name) == val, name


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without the built library the binding raises."""
    import subprocess
    import sys
    code = ("import paper_2001_10424_gb300 as gk\n"
            "try:\n"
            "    gk.load(%r)\n"
            "except RuntimeError as e:\n"
            "    print('raised', e)\n" % str(tmp_path / "libgkb.so"))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("raised"), out.stdout + out.stderr
