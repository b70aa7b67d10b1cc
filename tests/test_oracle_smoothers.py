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


# ---------------------------------------------------------------------------
# Pins of the pseudo-time step itself (Section 4.3, Eq. (29)/(30), Algorithm 3).
# The step is: explicit half u~ = u + tau_i f with tau_i = min(dtau, theta tau*_i)
# (reading R5: tau*_i the largest admissible step along f), then the implicit
# half u' + dtau A(u') = u~ by Jacobi sweeps started from u.  Each check below
# is stated in terms of A (pinned by the operator tests), the admissible step
# bound (pinned above by bisection) or a hand-derived closed form, never in
# terms of the smoother's own code; tests/test_oracle_mutations.py plants the
# plausible mistakes in a copy of the oracle and shows that each fails one of
# these checks.

def _smooth_case(seed=3, n=12, cfl=3.0):
    case = inputs.random_admissible_2d(n, n - 2, seed=seed, fmax=0.9, cfl=cfl)
    # moderate opacities keep the pseudo-time Jacobi iteration well contracting
    case["sa"] = np.clip(case["sa"], 1e-2, 5.0)
    case["ss"] = np.clip(case["ss"], 1e-2, 5.0)
    return case


def _admissible_direction(case, seed):
    """A source f inside the admissible cone (E_f > 0, |F_f| <= c E_f, T_f > 0),
    so that the explicit half is never limited: tau*_i is infinite."""
    rng = np.random.default_rng(seed)
    s = case["state"]
    f = np.empty_like(s)
    f[0] = s[0] * rng.uniform(0.2, 2.0, s[0].shape)
    th = rng.uniform(0, 2 * np.pi, s[0].shape)
    fr = rng.uniform(0, 0.95, s[0].shape)
    f[1], f[2] = fr * f[0] * np.cos(th), fr * f[0] * np.sin(th)
    f[3] = s[3] * rng.uniform(0.2, 2.0, s[0].shape)
    return f


def _tau(u, f, dtau, theta=0.5):
    """tau_i = min(dtau, theta tau*_i) per cell (reading R5)."""
    tau = np.empty(u.shape[1:])
    for j in range(u.shape[1]):
        for i in range(u.shape[2]):
            tau[j, i] = min(dtau, theta * O.max_admissible_step(u[:, j, i], f[:, j, i]))
    return tau


def check_implicit_half_solves_eq30(dtaus=(1e-3, 0.1, 1.0)):
    """With an admissible source (no limiting) and many Jacobi sweeps, one step
    solves u' + dtau A(u') = u + dtau f (Eq. (30)) to rounding."""
    case = _smooth_case()
    g = O.Grid.from_case(case)
    u = case["state"]
    f = _admissible_direction(case, 11)
    assert np.all(np.isinf(_tau(u, f, np.inf)))
    for dtau in dtaus:
        up, it = O.pseudo_time_smooth(g, case["dt"], case["sa"], case["ss"], f, u, dtau, m=1, nu=400)
        assert it >= 0
        lhs = up + dtau * O.apply_A(g, case["dt"], case["sa"], case["ss"], up)
        rhs = u + dtau * f
        err = np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs)
        assert err <= 1e-13, (dtau, err)


def check_limited_explicit_half(dtau=1.0):
    """With a source that leaves the admissible set, each cell's explicit half
    uses tau_i = min(dtau, tau*_i / 2) along f: the converged step solves
    u' + dtau A(u') = u + tau_i f cell by cell."""
    case = _smooth_case(seed=5)
    g = O.Grid.from_case(case)
    u = case["state"]
    rng = np.random.default_rng(12)
    f = rng.normal(0, 1, u.shape) * u[0] * np.array([4.0, 4.0, 4.0, 0.5])[:, None, None]
    tau = _tau(u, f, dtau)
    limited = tau < dtau
    assert limited.any() and (~limited).any()
    up, it = O.pseudo_time_smooth(g, case["dt"], case["sa"], case["ss"], f, u, dtau, m=1, nu=400)
    assert it >= 0
    lhs = up + dtau * O.apply_A(g, case["dt"], case["sa"], case["ss"], up)
    rhs = u + tau[None] * f
    err = np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs)
    assert err <= 1e-13, err


def check_small_dtau_is_explicit_euler():
    """As dtau -> 0 one pseudo-time step (one Jacobi sweep) is forward Euler of
    Eq. (29), du/dtau = f - A(u): u' = u + dtau (f - A(u)) + O(dtau^2)."""
    case = _smooth_case(seed=6)
    g = O.Grid.from_case(case)
    u = case["state"]
    rng = np.random.default_rng(13)
    f = O.apply_A(g, case["dt"], case["sa"], case["ss"], u) + rng.normal(0, 0.3, u.shape) * u[0]
    d = f - O.apply_A(g, case["dt"], case["sa"], case["ss"], u)
    # below the smallest admissible step no cell is limited
    d0 = 0.05 * float(_tau(u, f, np.inf).min())
    errs = []
    for dtau in (d0, 0.1 * d0):
        assert np.all(_tau(u, f, dtau) == dtau)
        up, _ = O.pseudo_time_smooth(g, case["dt"], case["sa"], case["ss"], f, u, dtau, m=1, nu=1)
        errs.append(np.linalg.norm(up - (u + dtau * d)) / (dtau * np.linalg.norm(d)))
    # first-order consistency: the relative defect is O(dtau), so it falls 10x
    assert errs[0] < 1e-3 and 0.05 < errs[1] / errs[0] < 0.2, errs


def check_steady_state_is_kept(dtaus=(1e-3, 1.0, 1e3)):
    """A steady state of Eq. (29) (f = A(u)) is returned unchanged by every
    pseudo-time step when A(u) lies in the admissible cone (no limiting)."""
    n = 16
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    E = 1.0 + 0.3 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    u = np.stack([E, 0.08 * E, -0.05 * E, E ** 0.25])
    sa = np.full((n, n), 0.7)
    ss = np.full((n, n), 1.3)
    g = O.Grid(2, n, n, 1 / n, 1 / n)
    dt = 0.5 / n
    f = O.apply_A(g, dt, sa, ss, u)
    assert np.all(np.isinf(_tau(u, f, np.inf)))
    for dtau in dtaus:
        up, it = O.pseudo_time_smooth(g, dt, sa, ss, f, u, dtau, m=3, nu=1)
        assert it >= 0
        np.testing.assert_allclose(up, u, rtol=1e-12, atol=0)


def _one_cell_root(Et, Tt, dtau, ka, c_v, a_r):
    """Bisection (200 halvings) for the gas temperature of one periodic cell:
    E'(1 + dtau) + dtau ka (E' - a_r T'^4) = Et and
    T'(1 + dtau c_v) - dtau ka (E' - a_r T'^4) = Tt; E' from the first."""
    def E_of(T):
        return (Et + dtau * ka * a_r * T ** 4) / (1 + dtau + dtau * ka)

    def g(T):
        return T * (1 + dtau * c_v) - dtau * ka * (E_of(T) - a_r * T ** 4) - Tt
    lo, hi = 0.0, max(Tt, 1.0) * 10
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if g(mid) < 0 else (lo, mid)
    T = 0.5 * (lo + hi)
    return E_of(T), T


def check_one_cell_closed_form():
    """One periodic cell in 1D is its own neighbour on both sides, so its
    transport terms cancel to A(u) = (E + src, (1 + k_t) F, C_v T - src) with
    src = k_a (E - a_r T^4).  For an admissible source the converged step is
    E', T' from the scalar gas balance (bisection), F' = (F + dtau f_F) /
    (1 + dtau (1 + k_t)); with sigma_a = 0, E' = (E + dtau f_E)/(1 + dtau) and
    T' = (T + dtau f_T)/(1 + dtau C_v).  One sweep (nu = 1) from u, with
    alpha = c dt / h, gives (E + dtau f_E + dtau alpha E) / (1 + dtau (1 +
    alpha)) for sigma = 0 (the initial guess of the Jacobi solve is u)."""
    h, dt, c_v, a_r = 1.0, 0.4, 1.0, 1.0
    g = O.Grid(1, 1, 1, h, 1.0, c_v=c_v, a_r=a_r)
    alpha = dt / h
    u = np.array([2.0, 0.6, 0.0, 1.1]).reshape(4, 1, 1)
    f = np.array([1.5, -0.9, 0.0, 0.7]).reshape(4, 1, 1)
    for sa, ssc in ((0.0, 0.0), (0.0, 3.0), (2.5, 0.5)):
        ka, kt = dt * sa, dt * (sa + ssc)
        for dtau in (0.3, 2.0, 40.0):
            up, it = O.pseudo_time_smooth(g, dt, np.full((1, 1), sa), np.full((1, 1), ssc), f, u,
                                          dtau, m=1, nu=300)
            assert it >= 0
            Et, Ft, Tt = u[0, 0, 0] + dtau * f[0, 0, 0], u[1, 0, 0] + dtau * f[1, 0, 0], \
                u[3, 0, 0] + dtau * f[3, 0, 0]
            if sa == 0.0:
                E1, T1 = Et / (1 + dtau), Tt / (1 + dtau * c_v)
            else:
                E1, T1 = _one_cell_root(Et, Tt, dtau, ka, c_v, a_r)
            F1 = Ft / (1 + dtau * (1 + kt))
            np.testing.assert_allclose(up[:, 0, 0], [E1, F1, 0.0, T1], rtol=1e-12, atol=1e-300)
        if sa == 0.0 and ssc == 0.0:
            dtau = 2.0
            up, _ = O.pseudo_time_smooth(g, dt, np.zeros((1, 1)), np.zeros((1, 1)), f, u, dtau,
                                         m=1, nu=1)
            E0, F0 = u[0, 0, 0], u[1, 0, 0]
            E1 = (E0 + dtau * f[0, 0, 0] + dtau * alpha * E0) / (1 + dtau * (1 + alpha))
            F1 = (F0 + dtau * f[1, 0, 0] + dtau * alpha * F0) / (1 + dtau * (1 + alpha))
            np.testing.assert_allclose(up[:2, 0, 0], [E1, F1], rtol=1e-14)


PSEUDO_TIME_PINS = (check_implicit_half_solves_eq30, check_limited_explicit_half,
                    check_small_dtau_is_explicit_euler, check_steady_state_is_kept,
                    check_one_cell_closed_form)


@pytest.mark.parametrize("pin", PSEUDO_TIME_PINS, ids=lambda p: p.__name__)
def test_pseudo_time_step_pin(pin):
    pin()
