"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/m1.h declares; the Python binding forwards to exactly those."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "m1.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(m1_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_14703_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["m1_create_grid", "m1_set_state", "m1_implicit_step", "m1_residual_norm",
                 "m1_get_state", "m1_destroy_grid"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_header(lib):
    from paper_2208_14703_gb300 import m1
    assert sorted(m1.EXPORTS) == sorted(s for s in declared_symbols() if s in m1.EXPORTS)
    assert set(m1.EXPORTS) <= set(declared_symbols())


def test_host_side_validation_without_gpu(lib):
    # argument validation happens before any CUDA call
    from paper_2208_14703_gb300 import m1
    p = m1.m1_default_params()
    assert (p.nu0, p.nu_l, p.m_pseudo, p.dtau0) == (3, 1, 3, 1e-3)
    bad = m1.make_desc(2, 100, 64, 1.0, 1.0, ["reflect"] * 4, lmax=4)   # 100 % 8 != 0
    h = ctypes.c_void_p()
    assert m1._lib.m1_create_grid(ctypes.byref(bad), None, ctypes.byref(h)) == m1.ERR_INVALID_ARG
    bad = m1.make_desc(2, 64, 64, 1.0, 1.0, ["periodic", "reflect", "reflect", "reflect"], lmax=2)
    assert m1._lib.m1_create_grid(ctypes.byref(bad), None, ctypes.byref(h)) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_create_grid(None, None, ctypes.byref(h)) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_destroy_grid(None) == m1.ERR_INVALID_ARG
