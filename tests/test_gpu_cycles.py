"""W- and F-cycles (Section 6.3 names them as the alternatives to the paper's
V-cycle) on the GPU against the FP64 oracle run with the same cycle shape: same
cycle count, residual history and Delta tau_im sequence, and the new state
within the FP64 parity bound; with two grids every shape is the V-cycle bit for
bit; the mixed-precision path and batches take the same shapes."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14703_gb300 import inputs

pytestmark = pytest.mark.gpu

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")

PARITY = 1e-10
SHAPES = [("W", 1), ("F", 2)]


def rel_l2(got, ref):
    nE = np.linalg.norm(ref[0])
    return max(np.linalg.norm(got[0] - ref[0]) / nE, np.linalg.norm(got[1:3] - ref[1:3]) / nE,
               np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(ref[3]))


def gpu_step(case, params, precision=0):
    g = m1.grid_from_case(case, precision=precision)
    st = g.implicit_step(case["dt"], params, allow_not_converged=True)
    out = np.stack(g.get_state())
    hist, dtau = g.step_history(st.cycles + 1)
    g.close()
    return out, st, hist, dtau


CASES = [
    ("1d-gaussian-256", lambda: inputs.gaussian_1d(256), 1e-10),
    ("2d-hot-square-64", lambda: inputs.hot_square_2d(64, lmax=4), 1e-8),
    ("2d-ragged-periodic", lambda: inputs.random_admissible_2d(48, 40, seed=3, fmax=0.9, cfl=20,
                                                               bc=("periodic",) * 4, lmax=3),
     1e-8),
]


@pytest.mark.parametrize("shape_name,shape", SHAPES)
@pytest.mark.parametrize("name,make,tol", CASES)
def test_shape_step_matches_oracle(shape_name, shape, name, make, tol):
    case = make()
    lmax = case["lmax"]
    g = O.Grid.from_case(case)
    ref, ost, ohist, odtau = O.implicit_step(g, case["dt"], case["sa"], case["ss"], case["state"],
                                             O.SolveParams(lmax=lmax, tol=tol, cycle=shape))
    assert ost["status"] == 0
    out, st, hist, dtau = gpu_step(case, m1.m1_default_params(tol=tol, cycle=shape))
    assert st.status == 0 and st.cycles == ost["cycles"]
    np.testing.assert_allclose(hist, ohist, rtol=1e-9, atol=1e-13 * ohist[0])
    np.testing.assert_allclose(dtau[:st.cycles], odtau, rtol=1e-12)
    assert st.damped == ost["damped"]
    assert rel_l2(out, ref) <= PARITY


@pytest.mark.parametrize("shape_name,shape", SHAPES)
def test_shape_fixed_cycles_match_oracle_before_convergence(shape_name, shape):
    # five cycles with five grids (tol = 0): every intermediate quantity agrees
    case = inputs.hot_square_2d(128, lmax=5)
    g = O.Grid.from_case(case)
    ref, ost, ohist, _ = O.implicit_step(g, case["dt"], case["sa"], case["ss"], case["state"],
                                         O.SolveParams(lmax=5, tol=0.0, max_cycles=5,
                                                       cycle=shape))
    out, st, hist, _ = gpu_step(case, m1.m1_default_params(tol=0.0, max_cycles=5, cycle=shape))
    assert st.cycles == 5 == ost["cycles"]
    np.testing.assert_allclose(hist, ohist, rtol=1e-11, atol=1e-13 * ohist[0])
    assert rel_l2(out, ref) <= 1e-12


def test_shapes_coincide_with_two_grids():
    case = inputs.hot_square_2d(64, lmax=2)
    outs = [gpu_step(case, m1.m1_default_params(tol=1e-8, cycle=s)) for s in (0, 1, 2)]
    for out, st, hist, _ in outs[1:]:
        assert st.cycles == outs[0][1].cycles
        np.testing.assert_array_equal(out, outs[0][0])
        np.testing.assert_array_equal(hist, outs[0][2])


@pytest.mark.parametrize("shape_name,shape", SHAPES)
def test_mixed_precision_takes_the_shape(shape_name, shape):
    """The mixed path's W/F step agrees with the FP64 GPU step of the same shape
    within the mixed bound (relative L2 1e-8) and takes the same cycle count."""
    case = inputs.hot_square_2d(128, lmax=5)
    p = m1.m1_default_params(tol=1e-8, cycle=shape)
    ref, st64, _, _ = gpu_step(case, p, precision=m1.FP64)
    out, st32, _, _ = gpu_step(case, p, precision=m1.MIXED)
    assert st64.status == 0 and st32.status == 0
    assert abs(st32.cycles - st64.cycles) <= 1
    assert rel_l2(out, ref) <= 1e-8


@pytest.mark.parametrize("shape_name,shape", SHAPES)
def test_batched_shape_equals_alone(shape_name, shape):
    cases = [inputs.hot_square_2d(64, lmax=4),
             inputs.random_admissible_2d(96, 96, seed=5, fmax=0.8, cfl=20, bc=("reflect",) * 4,
                                         lmax=4)]
    p = m1.m1_default_params(tol=1e-8, cycle=shape)
    b = m1.batch_from_cases(cases)
    stats = b.implicit_step([c["dt"] for c in cases], p)
    outs = [np.stack(b.get_state(k)) for k in range(len(cases))]
    b.close()
    for k, c in enumerate(cases):
        alone, st, _, _ = gpu_step(c, p)
        assert stats[k].cycles == st.cycles
        np.testing.assert_array_equal(alone, outs[k])
