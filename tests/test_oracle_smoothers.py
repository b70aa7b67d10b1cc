"""Pins of the oracle's smoothers: Proposition 1 (Jacobi keeps the admissible
set), Proposition 2 (the split pseudo-time step keeps it), the admissible step
bound against brute-force bisection, the damped prolongation of Eq. (34), and
the unique fixed point of Algorithm 1 (Section 3.1)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14703_gb300 import inputs


def _admissible_all(v, c=1.0, slack=1e-14):
    return (np.all(v[0] > 0) and np.all(v[3] > 0)
            and np.all(np.hypot(v[1], v[2]) <= c * v[0] * (1 + slack)))


@pytest.mark.parametrize("seed,fmax,cfl,bc", [(1, 0.5, 10, "periodic"), (2, 0.999, 100, "reflect"),
                                              (3, 1.0, 1000, "periodic"), (4, 1.0, 50, "inflow")])
def test_jacobi_sweep_preserves_admissibility(seed, fmax, cfl, bc):
    case = inputs.random_admissible_2d(16, 12, seed=seed, fmax=fmax, cfl=cfl, bc=(bc,) * 4)
    g = O.Grid.from_case(case)
    v = case["state"]
    b = O.rhs_of(g, v)
    for _ in range(5):
        v, it = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, v)
        assert it >= 0
        assert _admissible_all(v)


@pytest.mark.parametrize("seed", range(4))
def test_pseudo_time_step_preserves_admissibility_for_any_source(seed):
    # the source f = A(v) + r is in general not admissible (Section 4.3); the
    # split step of Eq. (30) with the limited explicit half must still be.
    case = inputs.random_admissible_2d(12, 12, seed=seed, fmax=0.99, cfl=20)
    g = O.Grid.from_case(case)
    rng = np.random.default_rng(seed)
    f = rng.normal(0, 1, case["state"].shape) * case["state"][0]
    for dtau in (1e-3, 1.0, 1e3):
        u, it = O.pseudo_time_smooth(g, case["dt"], case["sa"], case["ss"], f, case["state"], dtau)
        assert it >= 0 and _admissible_all(u)


def test_max_admissible_step_against_bisection():
    rng = np.random.default_rng(7)
    for _ in range(400):
        E = 10 ** rng.uniform(-1, 1)
        f = rng.uniform(0, 1) if rng.uniform() < 0.8 else 1.0
        th = rng.uniform(0, 2 * np.pi)
        u = np.array([E, f * E * np.cos(th), f * E * np.sin(th), rng.uniform(0.5, 2)])
        d = rng.normal(0, 1, 4) * np.array([E, E, E, 1])
        t = O.max_admissible_step(u, d)

        def ok(tau):
            w = u + tau * d
            return w[0] > 0 and w[3] > 0 and np.hypot(w[1], w[2]) <= w[0] * (1 + 1e-12)
        if np.isinf(t):
            assert all(ok(x) for x in (1.0, 10.0, 1e3, 1e6))
            continue
        assert ok(t * (1 - 1e-9)) or t < 1e-12
        # just past t the state leaves S (or stays out for a while): check by bisection
        lo, hi = 0.0, t * (1 + 1e-6) + 1e-300
        if not ok(hi):
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                lo, hi = (mid, hi) if ok(mid) else (lo, mid)
            assert hi == pytest.approx(t, rel=1e-6, abs=1e-12)


def test_prolong_correct_damps_only_inadmissible_cells():
    rng = np.random.default_rng(3)
    g = O.Grid(2, 16, 16, 1 / 16, 1 / 16, bc=("reflect",) * 4)
    gc = g.coarse()
    case = inputs.random_admissible_2d(16, 16, seed=8, fmax=0.9)
    uf = case["state"]
    vc = O.restrict_state(g, uf)
    uc = vc + rng.normal(0, 0.5, vc.shape) * vc[0]
    out, nd = O.prolong_correct(g, uc, vc, uf)
    pe = O.prolong(g, uc - vc, O.KIND_DIFF)
    target = uf + pe
    adm = np.array([[O.admissible(target[:, j, i]) for i in range(16)] for j in range(16)])
    assert nd == int((~adm).sum()) and nd > 0
    np.testing.assert_array_equal(out[:, adm], target[:, adm])
    assert _admissible_all(out, slack=1e-12)
    # a damped cell lies on the segment u -> target, at half the admissible fraction
    for j, i in zip(*np.nonzero(~adm)):
        ts = O.max_admissible_step(uf[:, j, i], pe[:, j, i])
        np.testing.assert_allclose(out[:, j, i], uf[:, j, i] + 0.5 * min(1, ts) * pe[:, j, i],
                                   rtol=1e-14, atol=1e-14)
    assert gc.nx == 8


def test_jacobi_fixed_point_is_unique():
    # Algorithm 1 contracts (Section 3.1): two different initial guesses reach the
    # same fixed point, and the fixed point solves A(v) = b.
    case = inputs.random_admissible_2d(8, 8, seed=2, fmax=0.8, cfl=3)
    g = O.Grid.from_case(case)
    b = O.rhs_of(g, case["state"])
    v1 = case["state"].copy()
    v2 = case["state"].copy()
    v2[0] *= 3.0
    v2[1:3] *= -0.5
    for _ in range(2000):
        v1, _ = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, v1)
        v2, _ = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, v2)
    np.testing.assert_allclose(v1, v2, rtol=1e-12, atol=1e-12)
    r = O.residual(g, case["dt"], case["sa"], case["ss"], b, v1)
    assert O.norm(g, r) <= 1e-12 * O.norm(g, b)
