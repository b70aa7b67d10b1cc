"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/m1.h declares; the Python binding forwards to exactly those."""
import ctypes
import os
import re

import numpy as np
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


# (name, descriptor fields, also invalid for the single-level op entry points,
# which ignore lmax)
BAD_DESCS = [
    ("dim 3", dict(dim=3, nx=64, ny=64), True),
    ("1D with ny > 1", dict(dim=1, nx=64, ny=2), True),
    ("empty grid", dict(dim=2, nx=0, ny=64), True),
    ("negative size", dict(dim=2, nx=64, ny=-8), True),
    ("lmax 0", dict(dim=2, nx=64, ny=64, lmax=0), False),
    ("lmax 21", dict(dim=1, nx=1 << 20, ny=1, lmax=21), False),
    ("ny not divisible by 2^(lmax-1)", dict(dim=2, nx=64, ny=60, lmax=4), False),
    ("nx not divisible by 2^(lmax-1)", dict(dim=1, nx=100, ny=1, lmax=4), False),
    ("c = 0", dict(dim=2, nx=64, ny=64, c=0.0), True),
    ("a_r < 0", dict(dim=2, nx=64, ny=64, a_r=-1.0), True),
    ("C_v nan", dict(dim=2, nx=64, ny=64, c_v=float("nan")), True),
    ("zero length", dict(dim=2, nx=64, ny=64, lx=0.0), True),
    ("precision 2", dict(dim=2, nx=64, ny=64, precision=2), True),
    ("unpaired periodic y wall", dict(dim=2, nx=64, ny=64, bc=["reflect", "reflect", "periodic",
                                                                "inflow"]), True),
    ("more than 2^30 cells", dict(dim=2, nx=1 << 16, ny=1 << 15, lmax=1), False),
]


@pytest.mark.parametrize("name,kw,op", BAD_DESCS, ids=[n for n, _, _ in BAD_DESCS])
def test_invalid_descriptors_rejected_before_any_cuda_call(lib, name, kw, op):
    from paper_2208_14703_gb300 import m1
    args = dict(dim=2, nx=64, ny=64, lx=1.0, ly=1.0, bc=["reflect"] * 4, lmax=3)
    args.update(kw)
    d = m1.make_desc(args["dim"], args["nx"], args["ny"], args["lx"], args["ly"], args["bc"],
                     args["lmax"], c=args.get("c", 1.0), a_r=args.get("a_r", 1.0),
                     c_v=args.get("c_v", 1.0), precision=args.get("precision", m1.FP64))
    d.ny = args["ny"]
    h = ctypes.c_void_p()
    assert m1._lib.m1_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == m1.ERR_INVALID_ARG
    arr = (m1.GridDesc * 1)(d)
    assert m1._lib.m1_create_batch(arr, 1, None, ctypes.byref(h)) == m1.ERR_INVALID_ARG
    if op:
        buf = np.zeros(4 * 64 * 64)
        assert m1._lib.m1_op_level(ctypes.byref(d), None, 0.1, m1._ptr(buf), m1._ptr(buf), None,
                                   m1.OP_APPLY, 0.0, 0.5, m1._ptr(buf),
                                   None) == m1.ERR_INVALID_ARG


def test_invalid_batches_servers_and_parameters_rejected(lib):
    from paper_2208_14703_gb300 import m1
    h = ctypes.c_void_p()
    a = m1.make_desc(1, 64, 1, 1.0, 1.0, ["periodic"] * 4, 2)
    b = m1.make_desc(1, 64, 1, 1.0, 1.0, ["periodic"] * 4, 3)
    arr = (m1.GridDesc * 2)(a, b)                 # level counts differ
    assert m1._lib.m1_create_batch(arr, 2, None, ctypes.byref(h)) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_create_batch(arr, 0, None, ctypes.byref(h)) == m1.ERR_INVALID_ARG
    for budget, slots, lmax, prec, small in ((0, 4, 3, 0, 0), (1 << 20, 0, 3, 0, 0),
                                             (1 << 20, 4, 0, 0, 0), (1 << 20, 4, 3, 2, 0),
                                             (1 << 20, 4, 3, 0, -1)):
        assert m1._lib.m1_server_create(budget, slots, lmax, prec, None, small, None,
                                        ctypes.byref(h)) == m1.ERR_INVALID_ARG
    p = m1.m1_default_params(nu_l=2)              # the paper fixes one sweep per pseudo step
    assert m1._lib.m1_server_create(1 << 20, 4, 3, 0, ctypes.byref(p), 0, None,
                                    ctypes.byref(h)) == m1.ERR_INVALID_ARG
    p = m1.m1_default_params(dtau_rule=2)
    assert m1._lib.m1_server_create(1 << 20, 4, 3, 0, ctypes.byref(p), 0, None,
                                    ctypes.byref(h)) == m1.ERR_INVALID_ARG
    p = m1.m1_default_params(cycle=3)                # V, W and F only
    assert m1._lib.m1_server_create(1 << 20, 4, 3, 0, ctypes.byref(p), 0, None,
                                    ctypes.byref(h)) == m1.ERR_INVALID_ARG
    assert m1.m1_default_params().cycle == m1.CYCLE_V
    t = ctypes.c_ulonglong()
    assert m1._lib.m1_serve_submit(None, None, 1, 0.1, None, ctypes.byref(t)) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_serve_poll(None, 1, None, None) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_serve_wait(None, 1, 1.0) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_server_destroy(None) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_implicit_step(None, 0.1, None, None) == m1.ERR_INVALID_ARG


def test_invalid_3d_operator_arguments_rejected(lib):
    """The 3D single-level entry point validates before any device work."""
    from paper_2208_14703_gb300 import m1
    import numpy as np
    ok = m1.make_desc3(4, 4, 4, 1.0, 1.0, 1.0)
    s = np.zeros(5 * 64)
    sig = np.zeros(2 * 64)
    ms = ctypes.c_double()
    bad = [m1.make_desc3(0, 4, 4, 1.0, 1.0, 1.0), m1.make_desc3(4, 4, 4, 1.0, 0.0, 1.0),
           m1.make_desc3(4, 4, 4, 1.0, 1.0, 1.0, bc=("inflow",) + ("periodic",) * 5)]
    for d in bad:
        assert m1._lib.m1_op_level3(ctypes.byref(d), 0.1, sig.ctypes.data, s.ctypes.data, None,
                                    m1.OP3_APPLY, 1, s.ctypes.data, 0, None,
                                    ctypes.byref(ms)) == m1.ERR_INVALID_ARG
    for mode, rhs, sweeps, dt in ((7, None, 1, 0.1), (m1.OP3_RESIDUAL, None, 1, 0.1),
                                  (m1.OP3_JACOBI, s.ctypes.data, 0, 0.1),
                                  (m1.OP3_APPLY, None, 1, 0.0)):
        assert m1._lib.m1_op_level3(ctypes.byref(ok), dt, sig.ctypes.data, s.ctypes.data, rhs,
                                    mode, sweeps, s.ctypes.data, 0, None,
                                    ctypes.byref(ms)) == m1.ERR_INVALID_ARG


def test_probe_rejects_bad_arguments_without_gpu(lib):
    from paper_2208_14703_gb300 import m1
    out = ctypes.c_double()
    assert m1._lib.m1_probe_fma_peak(m1.FP64, None, 0, ctypes.byref(out)) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_probe_fma_peak(7, None, 3, ctypes.byref(out)) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_probe_fma_peak(m1.FP64, None, 3, None) == m1.ERR_INVALID_ARG
    # the elementwise check entry: argument errors are found before any launch
    assert m1._lib.m1_op_elementwise(m1.FN_RCP64, None, -1, None, None) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_op_elementwise(m1.FN_SQRT64, None, 5, None, None) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_op_elementwise(6, None, 0, None, None) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_op_elementwise(m1.FN_SQRT32, None, 0, None, None) == 0


def test_grid3_validation_without_gpu(lib):
    from paper_2208_14703_gb300 import m1
    h = ctypes.c_void_p()
    ok = m1.make_desc3(16, 16, 16, 1.0, 1.0, 1.0, ("reflect",) * 6)
    for lmax in (0, 6, 21):          # 16 is not divisible by 2^5; out of range
        assert m1._lib.m1_create_grid3(ctypes.byref(ok), lmax, None, ctypes.byref(h)) == \
            m1.ERR_INVALID_ARG
    bad = m1.make_desc3(16, 16, 16, 1.0, 1.0, 1.0, ("periodic", "reflect") + ("reflect",) * 4)
    assert m1._lib.m1_create_grid3(ctypes.byref(bad), 2, None, ctypes.byref(h)) == m1.ERR_INVALID_ARG
    bad = m1.make_desc3(16, 16, 16, 0.0, 1.0, 1.0, ("reflect",) * 6)
    assert m1._lib.m1_create_grid3(ctypes.byref(bad), 2, None, ctypes.byref(h)) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_create_grid3(None, 2, None, ctypes.byref(h)) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_destroy_grid3(None) == m1.ERR_INVALID_ARG
    assert m1._lib.m1_grid3_implicit_step(None, 0.1, None, None) == m1.ERR_INVALID_ARG
