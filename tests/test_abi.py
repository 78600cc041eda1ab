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
