"""The all-core (OpenMP) build of the oracle gives bit-for-bit the results of
the one-core build: the same loops over the same cells, integer reductions and a
serial norm.  Checked on whole implicit steps (Algorithm 4: 1D and 2D, walls of
every kind, an inflow beam, V- and W-cycles) and on single kernels."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14703_gb300 import inputs

pytestmark = pytest.mark.skipif(not O.have_all_cores(), reason="no OpenMP in this compiler")


@pytest.fixture
def both():
    """Runs fn(...) on the one-core build, then the all-core build."""
    def run(fn):
        O.use_all_cores(False)
        a = fn()
        n = O.use_all_cores(True)
        try:
            b = fn()
        finally:
            O.use_all_cores(False)
        return a, b, n
    return run


def _step(case, **kw):
    g = O.Grid.from_case(case)
    p = O.SolveParams(lmax=case["lmax"], tol=case["tol"], **kw)
    v, st, hist, dt_hist = O.implicit_step(g, case["dt"], case["sa"], case["ss"], case["state"], p)
    return v, st, hist, dt_hist


@pytest.mark.parametrize("name,case,kw", [
    ("1d-gaussian", inputs.gaussian_1d(256), {}),
    ("2d-hot-square-64", inputs.hot_square_2d(64, lmax=4), {}),
    ("2d-beam-inflow-64", inputs.beam_channel_2d(64, lmax=4), {}),
    ("2d-hot-square-64-W", inputs.hot_square_2d(64, lmax=4), {"cycle": 1}),
])
def test_steps_bitwise_equal(both, name, case, kw):
    (v1, s1, h1, d1), (v2, s2, h2, d2), n = both(lambda: _step(case, **kw))
    assert n >= 1
    assert s1 == s2
    np.testing.assert_array_equal(v1, v2)
    np.testing.assert_array_equal(h1, h2)
    np.testing.assert_array_equal(d1, d2)


def test_kernels_bitwise_equal(both):
    case = inputs.random_admissible_2d(48, 40, seed=9, fmax=0.99, cfl=30,
                                       bc=("inflow", "reflect", "periodic", "periodic"))
    g = O.Grid.from_case(case)
    rng = np.random.default_rng(3)
    f = rng.normal(0, 1, case["state"].shape) * case["state"][0]
    b = O.rhs_of(g, case["state"])
    noise = rng.normal(0, 0.5, (4, 20, 24))

    def run():
        j, it = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, case["state"])
        p, _ = O.pseudo_time_smooth(g, case["dt"], case["sa"], case["ss"], f, case["state"], 0.7)
        r = O.residual(g, case["dt"], case["sa"], case["ss"], b, j)
        vc = O.restrict_state(g, case["state"])
        pc, nd = O.prolong_correct(g, vc + noise * vc[0], vc, case["state"])
        return j, it, p, r, O.norm(g, r), vc, pc, nd

    a, b2, _ = both(run)
    for x, y in zip(a, b2):
        np.testing.assert_array_equal(x, y)


def test_3d_step_bitwise_equal():
    from oracle import oracle3d as O3
    case = inputs.beam_3d(16, lmax=3)
    n = 16
    g = O3.Grid3(n, n, n, 1 / n, 1 / n, 1 / n, tuple(case["desc"]["bc"]), inflow=case["inflow"])
    p = O3.SolveParams3(lmax=3, tol=1e-8, cycle=1)
    O3.use_all_cores(False)
    a = O3.implicit_step(g, case["dt"], case["sa"], case["ss"], case["state"], p)
    assert O3.use_all_cores(True) >= 1
    try:
        b = O3.implicit_step(g, case["dt"], case["sa"], case["ss"], case["state"], p)
    finally:
        O3.use_all_cores(False)
    assert a[1] == b[1]
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[2], b[2])
