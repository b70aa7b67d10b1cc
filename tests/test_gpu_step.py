"""Whole implicit steps (Algorithm 4) on the GPU through the C ABI against the
FP64 oracle: same cycle count, same residual history, and the new state within
the FP64 parity bound (relative L2 1e-10 on E, on F normalised by c ||E||, and
on T).  At the full 1024^2 size, where the oracle cannot run the step, the
result is checked by properties the oracle can evaluate: the oracle's residual
of the GPU state, admissibility, conservation and determinism."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14703_gb300 import inputs

pytestmark = pytest.mark.gpu

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")

PARITY = 1e-10


def rel_l2(got, ref, c=1.0):
    nE = np.linalg.norm(ref[0])
    return dict(E=np.linalg.norm(got[0] - ref[0]) / nE,
                F=np.linalg.norm(got[1:3] - ref[1:3]) / (c * nE),
                T=np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(ref[3]))


def gpu_step(case, params, lmax=None, allow_nc=False):
    g = m1.grid_from_case(case, lmax=lmax)
    st = g.implicit_step(case["dt"], params, allow_not_converged=allow_nc)
    out = np.stack(g.get_state())
    hist, dtau = g.step_history(st.cycles + 1)
    g.close()
    return out, st, hist, dtau


def oracle_step(case, lmax, tol, max_cycles=20000):
    g = O.Grid.from_case(case)
    return O.implicit_step(g, case["dt"], case["sa"], case["ss"], case["state"],
                           O.SolveParams(lmax=lmax, tol=tol, max_cycles=max_cycles))


STEP_CASES = [
    ("1d-gaussian-256", lambda: inputs.gaussian_1d(256), 4, 1e-10),
    ("2d-hot-square-64", lambda: inputs.hot_square_2d(64, lmax=4), 4, 1e-8),
    ("2d-hot-square-128", lambda: inputs.hot_square_2d(128, lmax=5), 5, 1e-8),
    ("2d-beam-64", lambda: inputs.beam_channel_2d(64, lmax=4), 4, 1e-8),
    ("2d-riemann-64", lambda: inputs.riemann_2d(64, cfl=150.0, lmax=3, tol=5e-3), 3, 5e-3),
    ("1d-lmax1", lambda: inputs.gaussian_1d(128, lmax=1), 1, 1e-8),
]


@pytest.mark.parametrize("name,make,lmax,tol", STEP_CASES)
def test_step_matches_oracle(name, make, lmax, tol):
    case = make()
    ref, ost, ohist, odtau = oracle_step(case, lmax, tol)
    assert ost["status"] == 0
    out, st, hist, dtau = gpu_step(case, m1.m1_default_params(tol=tol), lmax=lmax)
    assert st.status == 0 and st.cycles == ost["cycles"]
    # residual norms agree to 1e-9 relative down to the rounding floor of
    # evaluating b - A(v) in FP64 (about 1e-13 ||r_0|| here)
    np.testing.assert_allclose(hist, ohist, rtol=1e-9, atol=1e-13 * ohist[0])
    np.testing.assert_allclose(dtau[:st.cycles], odtau, rtol=1e-12)
    assert st.damped == ost["damped"]
    err = rel_l2(out, ref, case["desc"]["c"])
    assert max(err.values()) <= PARITY, err
    assert np.all(out[0] > 0) and np.all(out[3] > 0)
    assert np.all(np.hypot(out[1], out[2]) <= out[0] * (1 + 1e-12))


def test_fixed_cycles_match_oracle_before_convergence():
    # stop after 7 cycles (tol = 0): every intermediate quantity must agree
    case = inputs.hot_square_2d(64, lmax=4)
    ref, ost, ohist, _ = oracle_step(case, 4, 0.0, max_cycles=7)
    out, st, hist, _ = gpu_step(case, m1.m1_default_params(tol=0.0, max_cycles=7), lmax=4,
                                allow_nc=True)
    assert st.status == m1.ERR_NOT_CONVERGED and st.cycles == 7 == ost["cycles"]
    np.testing.assert_allclose(hist, ohist, rtol=1e-11, atol=1e-13 * ohist[0])
    assert max(rel_l2(out, ref).values()) <= 1e-12


def test_equilibrium_is_returned_unchanged():
    case = inputs.hot_square_2d(64, lmax=4)
    case["state"][3] = 1.3
    case["state"][0] = 1.3 ** 4
    out, st, _, _ = gpu_step(case, m1.m1_default_params())
    assert st.cycles == 0 and st.status == 0
    np.testing.assert_array_equal(out, case["state"])


def test_nonadmissible_input_is_rejected_and_state_kept():
    case = inputs.gaussian_1d(64, lmax=2)
    g = m1.grid_from_case(case)
    s = case["state"].copy()
    s[1, 0, 5] = 3 * s[0, 0, 5]
    with pytest.raises(m1.M1Error) as e:
        g.set_state(s[0], s[1], s[2], s[3])
    assert e.value.status == m1.ERR_NONADMISSIBLE_INPUT
    s[1, 0, 5] = 0.0
    s[0, 0, 7] = np.nan
    with pytest.raises(m1.M1Error):
        g.set_state(s[0], s[1], s[2], s[3])
    np.testing.assert_array_equal(np.stack(g.get_state()), case["state"])
    g.close()


def test_state_round_trip_is_bitwise():
    case = inputs.random_admissible_2d(96, 64, seed=12)
    g = m1.grid_from_case(case, lmax=3)
    np.testing.assert_array_equal(np.stack(g.get_state()), case["state"])
    g.close()


def test_residual_norm_matches_oracle():
    case = inputs.hot_square_2d(64, lmax=4)
    g = m1.grid_from_case(case)
    og = O.Grid.from_case(case)
    b = O.rhs_of(og, case["state"])
    r0 = O.norm(og, O.residual(og, case["dt"], case["sa"], case["ss"], b, case["state"]))
    assert g.residual_norm(case["dt"]) == pytest.approx(r0, rel=1e-12)
    st = g.implicit_step(case["dt"], m1.m1_default_params())
    out = np.stack(g.get_state())
    r1 = O.norm(og, O.residual(og, case["dt"], case["sa"], case["ss"], b, out))
    assert g.residual_norm(case["dt"]) == pytest.approx(r1, rel=1e-9)
    assert r1 <= 1e-8 * r0 * (1 + 1e-9) and st.res == pytest.approx(r1, rel=1e-9)
    g.close()


def test_consecutive_steps_match_oracle():
    case = inputs.gaussian_1d(256)
    og = O.Grid.from_case(case)
    g = m1.grid_from_case(case)
    v = case["state"]
    for _ in range(3):
        v, ost, _, _ = O.implicit_step(og, case["dt"], case["sa"], case["ss"], v,
                                       O.SolveParams(lmax=4, tol=1e-10))
        st = g.implicit_step(case["dt"], m1.m1_default_params(tol=1e-10))
        assert st.cycles == ost["cycles"]
    assert max(rel_l2(np.stack(g.get_state()), v).values()) <= PARITY
    g.close()


@pytest.mark.parametrize("rule", [0, 1])
def test_dtau_rules_match_oracle_over_steps(rule):
    """Five steps of the 1D bump whose fifth step runs away under the printed
    dtau rule: per step the same cycle count and status as the oracle under
    either rule (the printed rule's run-away step ends at max_cycles on both),
    and the same state after the step the oracle converges."""
    case = inputs.bump_case(1, 1024, 7001, 50.0, 4, 1e-8)
    og = O.Grid.from_case(case)
    g = m1.grid_from_case(case)
    v = case["state"]
    p = m1.m1_default_params(tol=1e-8, max_cycles=400, dtau_rule=rule)
    for k in range(5):
        v, ost, _, _ = O.implicit_step(og, case["dt"], case["sa"], case["ss"], v,
                                       O.SolveParams(lmax=4, tol=1e-8, max_cycles=400,
                                                     dtau_rule=rule))
        st = g.implicit_step(case["dt"], p, allow_not_converged=True)
        assert st.cycles == ost["cycles"] and st.status == ost["status"], k
        if ost["status"] == 0:
            assert max(rel_l2(np.stack(g.get_state()), v).values()) <= PARITY, k
    g.close()


def test_full_size_step_properties():
    # the 1024^2 FP64 workload with L_max = 8, tol 1e-8
    case = inputs.hot_square_2d(1024)
    out, st, hist, _ = gpu_step(case, m1.m1_default_params(tol=case["tol"]))
    assert st.status == 0 and st.cycles > 0
    og = O.Grid.from_case(case)
    b = O.rhs_of(og, case["state"])
    r = O.residual(og, case["dt"], case["sa"], case["ss"], b, out)
    res = O.norm(og, r)
    assert res <= case["tol"] * hist[0] * (1 + 1e-6)
    assert res == pytest.approx(st.res, rel=1e-6)
    assert np.all(out[0] > 0) and np.all(out[3] > 0)
    assert np.all(np.hypot(out[1], out[2]) <= out[0] * (1 + 1e-12))
    # reflecting walls: E + C_v T changes by exactly -sum(r_E + r_T)
    e0 = (case["state"][0] + case["state"][3]).sum()
    e1 = (out[0] + out[3]).sum()
    assert abs((e1 - e0) + (r[0] + r[3]).sum()) <= 1e-12 * e0
    # a second run is bitwise identical (deterministic reductions, no atomics on data)
    out2, st2, _, _ = gpu_step(case, m1.m1_default_params(tol=case["tol"]))
    assert st2.cycles == st.cycles
    np.testing.assert_array_equal(out2, out)


def test_not_converged_keeps_last_admissible_iterate():
    case = inputs.hot_square_2d(64, lmax=4)
    out, st, _, _ = gpu_step(case, m1.m1_default_params(max_cycles=3), allow_nc=True)
    assert st.status == m1.ERR_NOT_CONVERGED and st.cycles == 3
    assert np.all(out[0] > 0) and np.all(np.hypot(out[1], out[2]) <= out[0] * (1 + 1e-12))


@pytest.mark.parametrize("lmax", [1, 2, 3, 4])
def test_paper_beam_matches_oracle(lmax):
    """The beam of Section 4.1 in nondimensional form (no matter, an f = 1 beam
    at 45 degrees through the west wall, CFL 2000, tolerance 1e-2) at 64^2: the
    same cycle count, residual history and damped cells as the oracle."""
    case = inputs.paper_beam_2d(64, lmax=lmax)
    ref, ost, ohist, _ = oracle_step(case, lmax, case["tol"])
    assert ost["status"] == 0
    out, st, hist, _ = gpu_step(case, m1.m1_default_params(tol=case["tol"]), lmax=lmax)
    assert st.status == 0 and st.cycles == ost["cycles"] and st.damped == ost["damped"]
    np.testing.assert_allclose(hist, ohist, rtol=1e-9, atol=1e-13 * ohist[0])
    assert max(rel_l2(out, ref).values()) <= PARITY
