"""Pins of the oracle's M1 closure (Section 2.1, Eq. (5)) against facts that do
not come from retyping the formula: Levermore's Lorentz-boost parametrisation
of the same closure, the isotropic and free-streaming limits, rotation
covariance and the trace/eigen structure of the pressure tensor."""
import numpy as np
import pytest

from oracle import oracle as O


def test_eddington_limits():
    # isotropic radiation: chi = 1/3; free streaming: chi = 1
    assert O.eddington_factor(0.0) == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert O.eddington_factor(1.0) == pytest.approx(1.0, rel=1e-15)


def test_eddington_matches_lorentz_boost():
    # Levermore (1984), cited in Section 2.1: an isotropic distribution boosted to
    # speed beta has f = 4 beta / (3 + beta^2) and chi = (1 + 3 beta^2) / (3 + beta^2).
    for beta in np.linspace(0.0, 1.0, 101):
        f = 4 * beta / (3 + beta ** 2)
        chi = (1 + 3 * beta ** 2) / (3 + beta ** 2)
        assert O.eddington_factor(f) == pytest.approx(chi, rel=2e-15, abs=1e-16)


def test_eddington_monotone_and_bounded():
    f = np.linspace(0, 1, 1001)
    chi = np.array([O.eddington_factor(x) for x in f])
    assert np.all(np.diff(chi) > 0)
    assert chi.min() >= 1 / 3 - 1e-16 and chi.max() <= 1 + 1e-16


def test_closure_isotropic_and_free_streaming():
    E = 2.5
    P = O.closure(E, 0.0, 0.0)
    np.testing.assert_allclose(P, [E / 3, 0.0, E / 3], rtol=1e-15)
    # f = 1 along a direction n: P = E n n^T
    th = 0.7
    n = np.array([np.cos(th), np.sin(th)])
    P = O.closure(E, E * n[0], E * n[1])
    np.testing.assert_allclose(P, [E * n[0] ** 2, E * n[0] * n[1], E * n[1] ** 2],
                               rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_closure_eigenstructure_and_rotation(seed):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        E = 10 ** rng.uniform(-3, 3)
        f = rng.uniform(0, 1)
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([np.cos(th), np.sin(th)])
        F = f * E * n
        Pxx, Pxy, Pyy = O.closure(E, F[0], F[1])
        P = np.array([[Pxx, Pxy], [Pxy, Pyy]])
        chi = O.eddington_factor(f)
        # eigenvalue chi E along the flux, (1 - chi)/2 E across it; trace of the
        # full 3x3 tensor (adding the out-of-plane (1 - chi)/2 E) is E
        np.testing.assert_allclose(P @ n, chi * E * n, rtol=1e-12, atol=1e-14 * E)
        m = np.array([-n[1], n[0]])
        np.testing.assert_allclose(P @ m, 0.5 * (1 - chi) * E * m, rtol=1e-12, atol=1e-14 * E)
        assert Pxx + Pyy + 0.5 * (1 - chi) * E == pytest.approx(E, rel=1e-13)
        # rotating the flux rotates the tensor
        a = rng.uniform(0, 2 * np.pi)
        Rm = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
        F2 = Rm @ F
        Q = O.closure(E, F2[0], F2[1])
        Q = np.array([[Q[0], Q[1]], [Q[1], Q[2]]])
        np.testing.assert_allclose(Q, Rm @ P @ Rm.T, rtol=1e-12, atol=1e-13 * E)


def test_closure_clamps_reduced_flux():
    # rounding may put |F| a few ulp above cE; the closure must stay finite
    E = 1.0
    P = O.closure(E, E * (1 + 4e-16), 0.0)
    assert np.all(np.isfinite(P)) and P[0] == pytest.approx(E, rel=1e-14)
