"""Mixed precision (FP32 V-cycles in correction form inside FP64 defect
correction) against the FP64 oracle.  The mixed path is a different iteration,
so the comparison is of converged results: both solve A(v) = b, the oracle to a
relative residual of 1e-13, the mixed path refined to 1e-12 (its FP64 defect is
exact, so refinement goes past the FP32 precision); every field (E, Fx, Fy, T)
of the mixed result must lie within relative L2 1e-8 of the oracle's (F
normalised by c ||E||).  A tolerance of 1e-10 alone leaves about 1e-8 of error
on these inputs for any solver (the weakly damped total-energy mode), so the
refinement is what the bound tests.  At full size the oracle evaluates the
residual of the mixed result."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14703_gb300 import inputs

pytestmark = pytest.mark.gpu

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")

BOUND = 1e-8


def field_errors(got, ref, c=1.0):
    nE = np.linalg.norm(ref[0])
    return {"E": np.linalg.norm(got[0] - ref[0]) / nE,
            "Fx": np.linalg.norm(got[1] - ref[1]) / (c * nE),
            "Fy": np.linalg.norm(got[2] - ref[2]) / (c * nE),
            "T": np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(ref[3])}


def mixed_step(case, tol, lmax=None, max_cycles=20000):
    g = m1.grid_from_case(case, lmax=lmax, precision=m1.MIXED)
    st = g.implicit_step(case["dt"], m1.m1_default_params(tol=tol, max_cycles=max_cycles))
    out = np.stack(g.get_state())
    g.close()
    return out, st


# (name, input, L_max, oracle tolerance, mixed tolerance); the free-streaming
# beam sits closer to the FP64 rounding floor of its residual, so both stop earlier
CASES = [
    ("1d-gaussian-256", lambda: inputs.gaussian_1d(256), 4, 1e-13, 1e-12),
    ("2d-hot-square-64", lambda: inputs.hot_square_2d(64, lmax=4), 4, 1e-13, 1e-12),
    ("2d-hot-square-128", lambda: inputs.hot_square_2d(128, lmax=5), 5, 1e-13, 1e-12),
    ("2d-beam-64", lambda: inputs.beam_channel_2d(64, lmax=4), 4, 1e-12, 1e-11),
]


@pytest.mark.parametrize("name,make,lmax,otol,mtol", CASES)
def test_mixed_step_matches_fp64_oracle(name, make, lmax, otol, mtol):
    case = make()
    og = O.Grid.from_case(case)
    ref, ost, _, _ = O.implicit_step(og, case["dt"], case["sa"], case["ss"], case["state"],
                                     O.SolveParams(lmax=lmax, tol=otol))
    assert ost["status"] == 0
    out, st = mixed_step(case, mtol, lmax)
    assert st.status == 0
    err = field_errors(out, ref, case["desc"]["c"])
    print(name, "cycles mixed", st.cycles, "oracle", ost["cycles"], "errors", err)
    assert max(err.values()) <= BOUND, err
    # the oracle's own residual of the mixed result meets the tolerance
    b = O.rhs_of(og, case["state"])
    res = O.norm(og, O.residual(og, case["dt"], case["sa"], case["ss"], b, out))
    assert res <= mtol * ost["res0"] * 1.01
    assert np.all(out[0] > 0) and np.all(out[3] > 0)
    assert np.all(np.hypot(out[1], out[2]) <= out[0] * (1 + 1e-12))


def test_mixed_full_size_against_fp64_path():
    # the 1024^2 workload: the oracle's residual of the mixed result, and the
    # per-field difference from the FP64 GPU path (itself parity-checked)
    case = inputs.hot_square_2d(1024)
    out, st = mixed_step(case, 1e-10)
    assert st.status == 0
    g = m1.grid_from_case(case)
    st64 = g.implicit_step(case["dt"], m1.m1_default_params(tol=1e-10))
    ref = np.stack(g.get_state())
    g.close()
    og = O.Grid.from_case(case)
    b = O.rhs_of(og, case["state"])
    res = O.norm(og, O.residual(og, case["dt"], case["sa"], case["ss"], b, out))
    assert res <= 1e-10 * st64.res0 * 1.001
    err = field_errors(out, ref)
    print("1024^2 mixed cycles", st.cycles, "fp64 cycles", st64.cycles, "ms", st.ms, st64.ms,
          "errors", err)
    assert max(err.values()) <= BOUND, err
    assert np.all(out[0] > 0) and np.all(np.hypot(out[1], out[2]) <= out[0] * (1 + 1e-12))


def test_mixed_not_converged_and_admissible():
    case = inputs.beam_channel_2d(64, lmax=4)
    g = m1.grid_from_case(case, precision=m1.MIXED)
    st = g.implicit_step(case["dt"], m1.m1_default_params(max_cycles=3), allow_not_converged=True)
    out = np.stack(g.get_state())
    g.close()
    assert st.status == m1.ERR_NOT_CONVERGED and st.cycles == 3
    assert np.all(out[0] > 0) and np.all(np.hypot(out[1], out[2]) <= out[0] * (1 + 1e-12))


def test_mixed_beam_4096_configuration():
    """The mixed-precision configuration at full size: a 4096^2 beam in a
    channel (L_max = 10), one step to 1e-8 in mixed precision and in FP64.  The
    oracle evaluates the residual of the mixed result over the whole grid; the
    per-field difference to the FP64 GPU path (itself parity-checked against
    the oracle at smaller sizes) is reported and bounded."""
    case = inputs.beam_channel_2d(4096)
    out, st = mixed_step(case, 1e-8)
    assert st.status == 0
    g = m1.grid_from_case(case)
    st64 = g.implicit_step(case["dt"], m1.m1_default_params(tol=1e-8))
    ref = np.stack(g.get_state())
    g.close()
    assert st64.status == 0
    og = O.Grid.from_case(case)
    b = O.rhs_of(og, case["state"])
    res = O.norm(og, O.residual(og, case["dt"], case["sa"], case["ss"], b, out))
    assert res <= 1e-8 * st64.res0 * 1.001
    err = field_errors(out, ref)
    print("4096^2 beam mixed cycles", st.cycles, "fp64 cycles", st64.cycles, "ms", st.ms,
          st64.ms, "errors", err)
    # the two paths take the same cycles (same residual history up to FP32
    # rounding of the corrections), so their results agree far below tol
    assert st.cycles == st64.cycles
    assert max(err.values()) <= BOUND, err
    assert np.all(out[0] > 0) and np.all(np.hypot(out[1], out[2]) <= out[0] * (1 + 1e-12))


# tol 1e-8: tol ||r_0|| lies far above the double-word noise floor, so the
# cycles form their defect in double-word FP32 (m1_kernels.cu, k_defect_dw)
DW_CASES = [
    ("2d-hot-square-128", lambda: inputs.hot_square_2d(128, lmax=5), 5),
    ("2d-beam-64", lambda: inputs.beam_channel_2d(64, lmax=4), 4),
    ("1d-gaussian-256", lambda: inputs.gaussian_1d(256, tol=1e-8), 4),
]


@pytest.mark.parametrize("name,make,lmax", DW_CASES, ids=[c[0] for c in DW_CASES])
def test_mixed_step_with_double_word_defect_matches_oracle(name, make, lmax):
    """At tol 1e-8 the mixed path takes the same cycles as the oracle's FP64 step
    and lands within 1e-8 of it per field (step parity of the mixed path)."""
    case = make()
    og = O.Grid.from_case(case)
    ref, ost, _, _ = O.implicit_step(og, case["dt"], case["sa"], case["ss"], case["state"],
                                     O.SolveParams(lmax=lmax, tol=1e-8))
    out, st = mixed_step(case, 1e-8, lmax)
    assert st.status == 0 and st.cycles == ost["cycles"], (st.cycles, ost["cycles"])
    err = field_errors(out, ref, case["desc"]["c"])
    print(name, st.cycles, "cycles", err)
    assert max(err.values()) <= BOUND, err


# The mixed path forms the cycles' defect in double words when
# tol ||r_0|| > 5e-12 diag ||b|| (m1_api.cu, make_ctl).  The difference between
# the double-word and the FP64 defect is largest at converged states (general
# values in every term of A); pin it there, on the hot square and the beam, at
# least 50 times below that threshold.
DW_FLOOR_CASES = [
    ("hot-square-256", lambda: inputs.hot_square_2d(256, lmax=6)),
    ("beam-window-256", lambda: inputs.beam_channel_crop(256, full=1024, lmax=6)),
]


@pytest.mark.parametrize("name,make", DW_FLOOR_CASES, ids=[c[0] for c in DW_FLOOR_CASES])
def test_double_word_defect_floor_at_converged_state(name, make):
    case = make()
    og = O.Grid.from_case(case)
    b = O.rhs_of(og, case["state"])
    g = m1.grid_from_case(case, precision=m1.FP64)
    g.implicit_step(case["dt"], m1.m1_default_params(tol=case["tol"]))
    v = np.stack(g.get_state())
    g.close()
    desc = m1.desc_from_case(case)
    sig = np.stack([case["sa"], case["ss"]])
    r64, _ = m1.m1_op_level(desc, case["dt"], sig, v, b, mode=m1.OP_RESIDUAL, inflow=case["inflow"])
    rdw, _ = m1.m1_op_level(desc, case["dt"], sig, v, b, mode=m1.OP_RESIDUAL_DW,
                            inflow=case["inflow"])
    d = case["desc"]
    diag = 1 + d["c"] * case["dt"] * d["nx"] / d["lx"] + d["c"] * case["dt"] * d["ny"] / d["ly"]
    floor = O.norm(og, rdw - r64) / (diag * O.norm(og, b))
    print(name, "double-word defect floor", floor, "x diag ||b||")
    assert floor <= 5e-12 / 50
