"""Pins of the oracle's operator A (Section 2.2 Eq. (6), Section 3.1 Eqs. (9)/(12),
[EXT] source terms from Eq. (3)) and of its local solve D^{-1}.

Independent references: the Rusanov flux-difference form of the scheme (the
paper's Eq. (6) is its expansion), telescoping conservation, the exact
upwind recurrence at f = 1, the equilibrium state, and a high-precision
bisection of the zero-dimensional source problem."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14703_gb300 import inputs


def _ghost_pad(g, v, axis_bc):
    """Pad a (4, ny, nx) state with one ghost layer using the stated ghost rules
    (periodic wrap; reflect = mirror with normal flux negated; neumann = copy)."""
    dim = g.dim
    s = v.copy()
    # x axis
    left, right = s[:, :, :1].copy(), s[:, :, -1:].copy()
    if axis_bc[0] == "periodic":
        left, right = s[:, :, -1:].copy(), s[:, :, :1].copy()
    elif axis_bc[0] == "reflect":
        left[1] *= -1
        right[1] *= -1
    s = np.concatenate([left, s, right], axis=2)
    if dim == 2:
        lo, hi = s[:, :1, :].copy(), s[:, -1:, :].copy()
        if axis_bc[1] == "periodic":
            lo, hi = s[:, -1:, :].copy(), s[:, :1, :].copy()
        elif axis_bc[1] == "reflect":
            lo[2] *= -1
            hi[2] *= -1
        s = np.concatenate([lo, s, hi], axis=1)
    return s


def _rusanov_flux_form(g, dt, sa, ss, v, axis_bc):
    """A(v) written as backward Euler of the conservation form with the Rusanov
    numerical flux Fhat = (Flux(U_L) + Flux(U_R))/2 - (c/2)(U_R - U_L), where
    U = (E, Fx, Fy) and the physical flux along x is (Fx, c^2 Pxx, c^2 Pxy)
    (along y: (Fy, c^2 Pxy, c^2 Pyy)), plus the backward-Euler sources."""
    c = g.c
    s = _ghost_pad(g, v, axis_bc)
    ny, nx = v.shape[1], v.shape[2]
    oy = 1 if g.dim == 2 else 0
    P = np.zeros((3,) + s.shape[1:])
    for j in range(s.shape[1]):
        for i in range(s.shape[2]):
            P[:, j, i] = O.closure(s[0, j, i], s[1, j, i], s[2, j, i], c)
    U = s[:3]

    def phys_flux(axis):
        if axis == 0:
            return np.stack([s[1], c * c * P[0], c * c * P[1]])
        return np.stack([s[2], c * c * P[1], c * c * P[2]])

    out = np.zeros_like(v)
    out[:3] = v[:3]
    for axis in ([0, 1] if g.dim == 2 else [0]):
        Fl = phys_flux(axis)
        h = g.hx if axis == 0 else g.hy
        if axis == 0:
            UL, UR = U[:, oy:oy + ny, :-1], U[:, oy:oy + ny, 1:]
            FL, FR = Fl[:, oy:oy + ny, :-1], Fl[:, oy:oy + ny, 1:]
            Fh = 0.5 * (FL + FR) - 0.5 * c * (UR - UL)          # faces i-1/2 .. nx-1/2
            out[:3] += dt / h * (Fh[:, :, 1:] - Fh[:, :, :-1])
        else:
            UL, UR = U[:, :-1, 1:-1], U[:, 1:, 1:-1]
            FL, FR = Fl[:, :-1, 1:-1], Fl[:, 1:, 1:-1]
            Fh = 0.5 * (FL + FR) - 0.5 * c * (UR - UL)
            out[:3] += dt / h * (Fh[:, 1:, :] - Fh[:, :-1, :])
    ka = c * dt * sa
    kt = c * dt * (sa + ss)
    src = ka * (v[0] - g.a_r * v[3] ** 4)
    out[0] += src
    out[1] += kt * v[1]
    out[2] += kt * v[2]
    out[3] = g.c_v * v[3] - src
    return out


@pytest.mark.parametrize("dim,bc", [(1, "periodic"), (1, "reflect"), (2, "periodic"),
                                    (2, "reflect"), (2, "neumann")])
def test_operator_equals_rusanov_flux_form(dim, bc):
    case = inputs.random_admissible_2d(12, 10, seed=3, dim=dim, bc=(bc,) * 4, fmax=0.95)
    g = O.Grid.from_case(case)
    A = O.apply_A(g, case["dt"], case["sa"], case["ss"], case["state"])
    ref = _rusanov_flux_form(g, case["dt"], case["sa"], case["ss"], case["state"], (bc, bc))
    scale = np.maximum(np.abs(ref).max(axis=(1, 2), keepdims=True), 1e-300)
    np.testing.assert_allclose(A / scale, ref / scale, rtol=0, atol=1e-13)


def test_operator_1d_source_free_matches_paper_rows():
    # with sigma = 0 in 1D, A must be the implicit HLL rows of Eq. (6) evaluated
    # at the given state: here compared through the flux form at random states
    case = inputs.random_admissible_2d(16, 1, seed=9, dim=1, fmax=0.99)
    case["sa"][:] = 0
    case["ss"][:] = 0
    g = O.Grid.from_case(case)
    A = O.apply_A(g, case["dt"], case["sa"], case["ss"], case["state"])
    ref = _rusanov_flux_form(g, case["dt"], case["sa"], case["ss"], case["state"],
                             ("periodic", "periodic"))
    np.testing.assert_allclose(A, ref, rtol=1e-13, atol=1e-13)
    assert np.all(A[2] == 0)


@pytest.mark.parametrize("bc", ["periodic", "reflect"])
def test_operator_conservation_identity(bc):
    # face fluxes telescope: sum A_E = sum E without sources (periodic or
    # reflecting); with sources sum (A_E + A_T) = sum (E + C_v T).
    case = inputs.random_admissible_2d(16, 16, seed=5, bc=(bc,) * 4)
    g = O.Grid.from_case(case)
    v = case["state"]
    A = O.apply_A(g, case["dt"], case["sa"], case["ss"], v)
    tot = (v[0] + g.c_v * v[3]).sum()
    assert (A[0] + A[3]).sum() == pytest.approx(tot, rel=1e-12)
    z = np.zeros_like(case["sa"])
    A0 = O.apply_A(g, case["dt"], z, z, v)
    assert A0[0].sum() == pytest.approx(v[0].sum(), rel=1e-12)
    if bc == "periodic":
        assert A0[1].sum() == pytest.approx(v[1].sum(), abs=1e-10 * np.abs(v[1]).sum())


def test_equilibrium_state_is_a_fixed_point():
    # E = a_r T^4 uniform, F = 0: every row of A(v) = b holds exactly
    n = 16
    T = 1.7
    case = inputs.random_admissible_2d(n, n, seed=1, bc=("reflect",) * 4)
    v = np.zeros((4, n, n))
    v[0] = T ** 4
    v[3] = T
    g = O.Grid.from_case(case)
    b = O.rhs_of(g, v)
    r = O.residual(g, case["dt"], case["sa"], case["ss"], b, v)
    assert np.abs(r).max() <= 64 * np.finfo(float).eps * np.abs(b).max()


def test_free_streaming_rows_are_the_upwind_recurrence():
    # 1D, sigma = 0, F = cE (f = 1, moving right): the E row collapses to the
    # implicit upwind scheme (1 + alpha) E_i - alpha E_{i-1} and the F row to c
    # times it (Section 2.2 with lambda = +c).
    n, c, dt = 20, 1.0, 3.0 / 20
    rng = np.random.default_rng(0)
    E = 10 ** rng.uniform(-1, 1, n)
    v = np.zeros((4, 1, n))
    v[0, 0] = E
    v[1, 0] = c * E
    v[3] = 1.0
    g = O.Grid(1, n, 1, 1.0 / n, 1.0, bc=("periodic",) * 4)
    z = np.zeros((1, n))
    A = O.apply_A(g, dt, z, z, v)
    alpha = c * dt * n
    up = (1 + alpha) * E - alpha * np.roll(E, 1)
    np.testing.assert_allclose(A[0, 0], up, rtol=1e-13, atol=1e-13 * E.max())
    np.testing.assert_allclose(A[1, 0], c * up, rtol=1e-13, atol=1e-13 * E.max())


def test_zero_dimensional_sources_against_bisection():
    # A uniform periodic state has no transport: the implicit step reduces to
    # (1 + k_a) E - k_a a_r T^4 = E^n,  C_v T - k_a (E - a_r T^4) = C_v T^n.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for (En, Tn, sa, cv) in [(1.0, 2.0, 3.0, 1.0), (50.0, 1.0, 1e3, 0.1), (1e-2, 1.5, 0.2, 5.0)]:
        n = 8
        v = np.zeros((4, 1, n))
        v[0] = En
        v[3] = Tn
        g = O.Grid(1, n, 1, 1.0 / n, 1.0, c_v=cv, bc=("periodic",) * 4)
        dt = 0.7
        sig = np.full((1, n), sa)
        # iterate to roundoff (tol = 0, a fixed 300 cycles): the stiff source makes
        # ||r_0|| large, so a relative stop would leave a visible absolute error
        out, st, _, _ = O.implicit_step(g, dt, sig, np.zeros((1, n)), v,
                                        O.SolveParams(lmax=2, tol=0.0, max_cycles=300))
        ka = mp.mpf(dt) * sa
        En_, Tn_, cv_ = mp.mpf(En), mp.mpf(Tn), mp.mpf(cv)
        # eliminate E: E = (E^n + ka T^4)/(1 + ka); g(T) = cv T - ka (E - T^4) - cv T^n

        def gfun(T):
            E = (En_ + ka * T ** 4) / (1 + ka)
            return cv_ * T - ka * (E - T ** 4) - cv_ * Tn_
        lo, hi = mp.mpf(0), mp.mpf(10) * (Tn_ + (En_ / 1) ** 0.25 + 1)
        for _ in range(200):
            mid = (lo + hi) / 2
            if gfun(mid) > 0:
                hi = mid
            else:
                lo = mid
        T = (lo + hi) / 2
        E = (En_ + ka * T ** 4) / (1 + ka)
        np.testing.assert_allclose(out[3], float(T), rtol=1e-14)
        np.testing.assert_allclose(out[0], float(E), rtol=1e-14)
        # total energy of the cell is exchanged, not created
        np.testing.assert_allclose(out[0] + cv * out[3], En + cv * Tn, rtol=1e-14)


def test_local_solve_reduces_to_paper_inverse_without_sources():
    # sigma = 0, (w0, w1) = (0, 1): D^{-1} = (1 + c dt/h)^{-1} I (proof of Prop. 1)
    beta = np.array([2.0, 0.3, -0.4, 1.1])
    diag = 7.5
    out, it = O.local_solve(0.0, 1.0, diag, 0.0, 0.0, 1.0, 1.0, beta)
    np.testing.assert_allclose(out[:3], beta[:3] / diag, rtol=1e-15)
    assert out[3] == pytest.approx(1.1, rel=1e-15) and it == 0


@pytest.mark.parametrize("w0,w1", [(0.0, 1.0), (1.0, 1e-3), (1.0, 10.0)])
def test_local_solve_satisfies_its_equations(w0, w1):
    rng = np.random.default_rng(11)
    for _ in range(200):
        diag = 1 + rng.uniform(0, 400)
        ka, ks = 10 ** rng.uniform(-3, 4), 10 ** rng.uniform(-3, 4)
        kt = ka + ks
        cv, ar = 10 ** rng.uniform(-1, 1), 1.0
        E = 10 ** rng.uniform(-2, 3)
        beta = np.array([E, 0.5 * E, -0.3 * E, 10 ** rng.uniform(-1, 1)])
        out, it = O.local_solve(w0, w1, diag, ka, kt, cv, ar, beta)
        assert it >= 0
        A, k = w0 + w1 * diag, w1 * ka
        e1 = A * out[0] + k * (out[0] - ar * out[3] ** 4) - beta[0]
        e3 = (w0 + w1 * cv) * out[3] - k * (out[0] - ar * out[3] ** 4) - beta[3]
        scale = max(abs(beta[0]), abs(beta[3]), k * ar * out[3] ** 4, A * out[0])
        assert abs(e1) <= 1e-13 * scale and abs(e3) <= 1e-13 * scale
        np.testing.assert_allclose(out[1:3] * (w0 + w1 * (diag + kt)), beta[1:3], rtol=1e-14)
        # admissibility of the output (E > 0, T > 0, |F| <= c E)
        assert out[0] > 0 and out[3] > 0 and np.hypot(out[1], out[2]) <= out[0]
