"""Element-wise parity at the full sizes of the workloads: the GPU step
(Algorithm 4) against the oracle's step on the same input, run by the oracle's
all-core build (bit-for-bit the one-core oracle, tests/test_oracle_threads.py).

- the 2D plain-FP64 workload: 1024^2 hot square in lognormal opacities,
  L_max = 8, tol 1e-8.  Same cycle count, same residual history, and relative
  L2 <= 1e-10 on E, F (against c ||E||) and T;
- the mixed-precision generator (an f = 1 beam entering a channel through the
  lognormal medium): the 1024^2 window of its 4096^2 grid that holds the beam
  (west wall, centred on the channel), L_max = 8, tol 1e-8.  The mixed path
  per field (E, Fx, Fy, T) within 1e-8 of the oracle, and the FP64 path within
  1e-10, after the same number of cycles.

Each oracle step takes minutes of host time."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14703_gb300 import inputs

pytestmark = pytest.mark.gpu

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")

PARITY_FP64 = 1e-10
PARITY_MIXED = 1e-8


def field_errors(got, ref, c=1.0):
    nE = np.linalg.norm(ref[0])
    return {"E": np.linalg.norm(got[0] - ref[0]) / nE,
            "Fx": np.linalg.norm(got[1] - ref[1]) / (c * nE),
            "Fy": np.linalg.norm(got[2] - ref[2]) / (c * nE),
            "T": np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(ref[3])}


def oracle_step_all_cores(case):
    threads = O.use_all_cores(True)
    try:
        g = O.Grid.from_case(case)
        out = O.implicit_step(g, case["dt"], case["sa"], case["ss"], case["state"],
                              O.SolveParams(lmax=case["lmax"], tol=case["tol"]))
    finally:
        O.use_all_cores(False)
    return out, threads


def gpu_step(case, precision):
    g = m1.grid_from_case(case, precision=precision)
    st = g.implicit_step(case["dt"], m1.m1_default_params(tol=case["tol"]))
    out = np.stack(g.get_state())
    hist, _ = g.step_history(st.cycles + 1)
    g.close()
    return out, st, hist


def test_fp64_step_1024_matches_oracle():
    case = inputs.hot_square_2d(1024)
    out, st, hist = gpu_step(case, m1.FP64)
    (ref, ost, ohist, _), threads = oracle_step_all_cores(case)
    assert ost["status"] == 0 and st.status == 0
    assert st.cycles == ost["cycles"]
    np.testing.assert_allclose(hist, ohist, rtol=1e-9, atol=1e-13 * ohist[0])
    err = field_errors(out, ref)
    print(f"1024^2 FP64: {st.cycles} cycles (oracle on {threads} threads), errors {err}")
    assert max(err.values()) <= PARITY_FP64, err


def test_beam_window_1024_mixed_and_fp64_match_oracle():
    case = inputs.beam_channel_crop(1024)
    (ref, ost, _, _), threads = oracle_step_all_cores(case)
    assert ost["status"] == 0
    out64, st64, _ = gpu_step(case, m1.FP64)
    assert st64.status == 0 and st64.cycles == ost["cycles"]
    err64 = field_errors(out64, ref)
    outm, stm, _ = gpu_step(case, m1.MIXED)
    assert stm.status == 0
    errm = field_errors(outm, ref)
    print(f"beam window 1024^2: oracle {ost['cycles']} cycles on {threads} threads; FP64 "
          f"{st64.cycles} cycles, errors {err64}; mixed {stm.cycles} cycles, errors {errm}")
    assert max(err64.values()) <= PARITY_FP64, err64
    assert max(errm.values()) <= PARITY_MIXED, errm
    assert np.all(outm[0] > 0) and np.all(np.hypot(outm[1], outm[2]) <= outm[0] * (1 + 1e-12))
