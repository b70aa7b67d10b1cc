"""Pins of the 3D oracle (oracle/m1_oracle3d.c), each a fact independent of its
own formulas: the closure against Levermore's parametrisation and its tensor
structure; states uniform along z (and y) reducing to the 2D (1D) oracle term by
term and, for the whole step, at the fixed point; invariance under a cyclic
permutation of the axes; conservation; equilibrium; R = 2^-3 P^T; admissibility
after every sweep and pseudo-time step (Propositions 1 and 2); dense Newton on a
4^3 grid; W- and F-cycles reaching the V-cycle's fixed point; inflow walls
reducing to the 2D oracle's, an f = 1 beam along z obeying the exact upwind
recurrence, and dense Newton with an inflow wall."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import oracle3d as O3


def random_state3(nx, ny, nz, seed, fmax=0.9, c=1.0):
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    E = 10.0 ** rng.uniform(-1.0, 1.0, shape)
    f = fmax * rng.uniform(0.0, 1.0, shape)
    d = rng.standard_normal((3,) + shape)
    d /= np.linalg.norm(d, axis=0)
    T = 10.0 ** rng.uniform(-0.3, 0.3, shape)
    return np.concatenate([E[None], f * c * E * d, T[None]])


def opacities(shape, seed, lo=-2.0, hi=2.0):
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(lo, hi, shape), 10.0 ** rng.uniform(lo, hi, shape)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ---- closure (Section 2.1, Eq. (5)) ----

@pytest.mark.parametrize("beta", [0.0, 0.2, 0.5, 0.8, 0.99])
def test_closure_eigenstructure_follows_levermore(beta):
    """Levermore's Lorentz-boost form of the M1 closure: f = 4b/(3 + b^2),
    chi = (1 + 3b^2)/(3 + b^2).  P has the eigenvalue chi E along n and
    (1 - chi) E / 2 (twice) across it; its trace is E."""
    f = 4 * beta / (3 + beta ** 2)
    chi = (1 + 3 * beta ** 2) / (3 + beta ** 2)
    rng = np.random.default_rng(int(100 * beta))
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    E = 2.5
    P = O3.closure(E, f * E * n)
    np.testing.assert_allclose(P, P.T, rtol=0, atol=1e-15)
    assert np.trace(P) == pytest.approx(E, rel=1e-14)
    np.testing.assert_allclose(P @ n, chi * E * n, rtol=0, atol=1e-14 * E)
    t = np.cross(n, rng.standard_normal(3))
    t /= np.linalg.norm(t)
    np.testing.assert_allclose(P @ t, 0.5 * (1 - chi) * E * t, rtol=0, atol=1e-14 * E)


def test_closure_rotates_with_the_flux():
    rng = np.random.default_rng(4)
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    F = np.array([0.3, -0.5, 0.6])
    np.testing.assert_allclose(O3.closure(1.7, q @ F), q @ O3.closure(1.7, F) @ q.T,
                               rtol=0, atol=1e-14)


# ---- reductions to the 2D and 1D oracle ----

@pytest.mark.parametrize("bc2", [("periodic",) * 4, ("reflect",) * 4,
                                 ("neumann", "reflect", "periodic", "periodic")])
def test_z_uniform_operator_is_the_2d_operator(bc2):
    """A state uniform along a periodic z axis with Fz = 0: the z faces cancel
    (diagonal c dt/hz against the two z neighbour terms), so every row equals the
    2D oracle's on each slice and the Fz row is zero."""
    nx, ny, nz, dt = 8, 6, 4, 0.05
    s2 = random_state3(nx, ny, 1, 7)[[0, 1, 2, 4], 0]          # (4, ny, nx) with Fz dropped
    s2[1:3] *= 0.9
    sa2, ss2 = opacities((ny, nx), 8)
    g2 = O.Grid(2, nx, ny, 1.0 / nx, 1.0 / ny, 1.0, 1.0, 1.0, bc2)
    a2 = O.apply_A(g2, dt, sa2, ss2, s2)
    g3 = O3.Grid3(nx, ny, nz, 1.0 / nx, 1.0 / ny, 0.3, bc2 + ("periodic", "periodic"))
    s3 = np.zeros(g3.shape)
    s3[[0, 1, 2, 4]] = s2[:, None]
    a3 = O3.apply_A(g3, dt, np.repeat(sa2[None], nz, 0), np.repeat(ss2[None], nz, 0), s3)
    for k in range(nz):
        assert rel(a3[[0, 1, 2, 4], k], a2) <= 1e-13
    assert np.abs(a3[3]).max() == 0.0


def test_yz_uniform_operator_is_the_1d_operator():
    nx, dt = 16, 0.2
    s1 = random_state3(nx, 1, 1, 9)[[0, 1, 4], 0, 0]           # E, Fx, T along x
    sa1, ss1 = opacities((nx,), 10)
    g1 = O.Grid(1, nx, 1, 1.0 / nx, 1.0, 1.0, 1.0, 1.0, ("reflect",) * 4)
    v1 = np.zeros((4, 1, nx))
    v1[0, 0], v1[1, 0], v1[3, 0] = s1
    a1 = O.apply_A(g1, dt, sa1[None], ss1[None], v1)
    g3 = O3.Grid3(nx, 2, 4, 1.0 / nx, 0.5, 0.25, ("reflect", "reflect") + ("periodic",) * 4)
    s3 = np.zeros(g3.shape)
    s3[0], s3[1], s3[4] = (x[None, None, :] for x in s1)
    sa3 = np.broadcast_to(sa1, (4, 2, nx))
    ss3 = np.broadcast_to(ss1, (4, 2, nx))
    a3 = O3.apply_A(g3, dt, sa3, ss3, s3)
    for k in range(4):
        for j in range(2):
            assert rel(a3[[0, 1, 4], k, j], a1[[0, 1, 3], 0]) <= 1e-13
    assert np.abs(a3[[2, 3]]).max() == 0.0


def test_z_uniform_step_reaches_the_2d_fixed_point():
    """The whole multigrid step of a z-uniform state reaches the 2D oracle's
    fixed point (the Jacobi iterates differ: the z neighbours lag one sweep)."""
    nx = ny = 8
    s2 = random_state3(nx, ny, 1, 11, fmax=0.6)[[0, 1, 2, 4], 0]
    sa2, ss2 = opacities((ny, nx), 12, -1.0, 1.0)
    dt = 4.0 / nx
    g2 = O.Grid(2, nx, ny, 1.0 / nx, 1.0 / ny, 1.0, 1.0, 1.0, ("reflect",) * 4)
    ref, st2, h2, _ = O.implicit_step(g2, dt, sa2, ss2, s2,
                                      O.SolveParams(lmax=2, tol=0.0, max_cycles=400))
    assert h2[-1] <= 1e-14 * h2[0]
    g3 = O3.Grid3(nx, ny, 2, 1.0 / nx, 1.0 / ny, 0.5, ("reflect",) * 4 + ("periodic",) * 2)
    s3 = np.zeros(g3.shape)
    s3[[0, 1, 2, 4]] = s2[:, None]
    out, st3, h3 = O3.implicit_step(g3, dt, np.repeat(sa2[None], 2, 0), np.repeat(ss2[None], 2, 0),
                                    s3, O3.SolveParams3(lmax=2, tol=0.0, max_cycles=400))
    assert h3[-1] <= 1e-14 * h3[0]
    for k in range(2):
        assert rel(out[[0, 1, 2, 4], k], ref) <= 1e-11
    assert np.abs(out[3]).max() <= 1e-14 * np.abs(out[0]).max()


# ---- symmetry, conservation, equilibrium ----

def test_cyclic_axis_permutation():
    """Renaming the axes (x, y, z) -> (z, x, y), with the flux components, the
    cell sizes and the walls, permutes the operator's result."""
    nx, ny, nz, dt = 6, 4, 8, 0.07
    s = random_state3(nx, ny, nz, 13)
    sa, ss = opacities((nz, ny, nx), 14)
    bc = ("reflect", "reflect", "periodic", "periodic", "neumann", "neumann")
    g = O3.Grid3(nx, ny, nz, 0.11, 0.13, 0.17, bc)
    a = O3.apply_A(g, dt, sa, ss, s)

    def perm(v):                      # new (x, y, z) = old (y, z, x); arrays are (.., z, y, x)
        return np.ascontiguousarray(v.transpose(0, 3, 1, 2) if v.ndim == 4 else v.transpose(2, 0, 1))

    def perm_fields(v):
        p = perm(v)
        return p[[0, 2, 3, 1, 4]]     # Fx' = Fy, Fy' = Fz, Fz' = Fx

    gp = O3.Grid3(ny, nz, nx, 0.13, 0.17, 0.11, bc[2:4] + bc[4:6] + bc[0:2])
    ap = O3.apply_A(gp, dt, perm(sa), perm(ss), perm_fields(s))
    assert rel(ap, perm_fields(a)) <= 1e-13


def test_conservation_of_energy_and_flux_sums():
    """Periodic walls, no matter: the face terms telescope, so sum A(v)_E = sum E
    and sum A(v)_F = sum F."""
    nx, ny, nz = 8, 6, 4
    s = random_state3(nx, ny, nz, 15)
    z = np.zeros((nz, ny, nx))
    g = O3.Grid3(nx, ny, nz, 0.1, 0.2, 0.3)
    a = O3.apply_A(g, 0.9, z, z, s)
    for f in range(4):
        assert abs(a[f].sum() - s[f].sum()) <= 1e-12 * np.abs(s[0]).sum()


def test_equilibrium_is_returned_unchanged():
    nx = ny = nz = 4
    g = O3.Grid3(nx, ny, nz, 0.25, 0.25, 0.25, ("reflect",) * 6)
    s = np.zeros(g.shape)
    s[4] = 1.7
    s[0] = 1.7 ** 4
    sa, ss = opacities((nz, ny, nx), 16)
    out, st, _ = O3.implicit_step(g, 0.5, sa, ss, s, O3.SolveParams3(lmax=2))
    assert st["cycles"] == 0 and st["status"] == 0
    np.testing.assert_array_equal(out, s)


# ---- transfers (Section 4.2, R = 2^-d P^T with d = 3) ----

def test_restriction_is_the_scaled_transpose_of_prolongation():
    g = O3.Grid3(4, 4, 4, 0.25, 0.25, 0.25)
    gc = g.coarse()
    nf, nc = 64, 8
    P = np.zeros((nf, nc))
    for q in range(nc):
        e = np.zeros(gc.shape)
        e[0].reshape(-1)[q] = 1.0
        P[:, q] = O3.prolong(g, e)[0].reshape(-1)
    R = np.zeros((nc, nf))
    for q in range(nf):
        e = np.zeros(g.shape)
        e[0].reshape(-1)[q] = 1.0
        R[:, q] = O3.restrict_state(g, e)[0].reshape(-1)
    np.testing.assert_allclose(R, P.T / 8.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(P.sum(axis=1), 1.0)           # constants are kept
    np.testing.assert_allclose(R.sum(axis=1), 1.0)


# ---- admissibility (Propositions 1 and 2 in 3D) ----

@pytest.mark.parametrize("seed", [17, 18])
def test_sweeps_and_pseudo_time_steps_stay_admissible(seed):
    nx, ny, nz = 6, 4, 4
    g = O3.Grid3(nx, ny, nz, 1.0 / nx, 1.0 / ny, 1.0 / nz, ("reflect",) * 6)
    u = random_state3(nx, ny, nz, seed, fmax=0.999)
    b = random_state3(nx, ny, nz, seed + 100, fmax=0.999)
    sa, ss = opacities((nz, ny, nx), seed + 200)

    def ok(v):
        return (np.all(v[0] > 0) and np.all(v[4] > 0)
                and np.all(np.sqrt((v[1:4] ** 2).sum(0)) <= v[0] * (1 + 1e-12)))

    for dt in (0.01, 1.0, 100.0):
        v = u
        for _ in range(3):
            v, it = O3.jacobi_sweep(g, dt, sa, ss, b, v)
            assert it >= 0 and ok(v)
        f = O3.apply_A(g, dt, sa, ss, b) - O3.apply_A(g, dt, sa, ss, u)   # any source
        w, it = O3.pseudo_time_smooth(g, dt, sa, ss, f, u, dtau=0.3)
        assert it >= 0 and ok(w)


# ---- the whole step ----

def _newton_solve3(g, dt, sa, ss, b, v0, iters=30):
    v = v0.copy()
    n = v.size
    for _ in range(iters):
        r = O3.apply_A(g, dt, sa, ss, v) - b
        if np.abs(r).max() <= 1e-15 * np.abs(b).max():
            break
        J = np.zeros((n, n))
        flat = v.reshape(-1)
        for k in range(n):
            h = 1e-7 * max(abs(flat[k]), 1e-3)
            vp, vm = flat.copy(), flat.copy()
            vp[k] += h
            vm[k] -= h
            J[:, k] = (O3.apply_A(g, dt, sa, ss, vp.reshape(v.shape))
                       - O3.apply_A(g, dt, sa, ss, vm.reshape(v.shape))).reshape(-1) / (2 * h)
        v = v - np.linalg.solve(J, r.reshape(-1)).reshape(v.shape)
    return v


def test_multigrid_step_matches_brute_force_newton_4cube():
    g = O3.Grid3(4, 4, 4, 0.25, 0.25, 0.25)
    v0 = random_state3(4, 4, 4, 19, fmax=0.7)
    sa, ss = opacities((4, 4, 4), 20, -1.0, 1.0)
    dt = 1.0
    b = v0.copy()
    mg, st, hist = O3.implicit_step(g, dt, sa, ss, v0, O3.SolveParams3(lmax=2, tol=0.0,
                                                                        max_cycles=1500))
    assert hist[-1] <= 1e-15 * hist[0]
    rng = np.random.default_rng(3)
    nw = _newton_solve3(g, dt, sa, ss, b, mg * (1 + 1e-3 * rng.standard_normal(mg.shape)))
    np.testing.assert_allclose(mg, nw, rtol=0, atol=1e-11 * np.abs(nw[0]).max())


@pytest.mark.parametrize("shape", [1, 2])
def test_w_and_f_cycles_reach_the_v_cycle_fixed_point(shape):
    g = O3.Grid3(8, 8, 8, 0.125, 0.125, 0.125, ("reflect",) * 6)
    v0 = random_state3(8, 8, 8, 21, fmax=0.6)
    sa, ss = opacities((8, 8, 8), 22, -1.0, 1.0)
    p = dict(lmax=3, tol=0.0, max_cycles=300)
    ref, _, hv = O3.implicit_step(g, 2.0, sa, ss, v0, O3.SolveParams3(**p))
    out, _, hs = O3.implicit_step(g, 2.0, sa, ss, v0, O3.SolveParams3(cycle=shape, **p))
    assert hv[-1] <= 1e-14 * hv[0] and hs[-1] <= 1e-14 * hs[0]
    assert rel(out, ref) <= 1e-12


# ---- inflow walls ----

def _inflow3(g, wall, E, F):
    """A (6, 4, F) profile array with wall `wall` set from per-face arrays."""
    out = np.zeros((6, 4, g.face))
    nf = E.size
    out[wall, 0, :nf] = E.ravel()
    for c in range(3):
        out[wall, 1 + c, :nf] = F[c].ravel()
    return out


def _beam_2d(n):
    y = (np.arange(n) + 0.5) / n
    chan = (y >= 0.4) & (y <= 0.6)
    inflow = np.zeros((4, 3, n))
    inflow[0, 0] = 1.0
    inflow[0, 1] = np.where(chan, 1.0, 0.0)
    return inflow


def test_z_uniform_inflow_operator_is_the_2d_operator():
    """An x-low inflow wall whose profile does not vary along z: the 3D operator
    of a z-uniform state equals the 2D oracle's with the same inflow wall."""
    nx = ny = 16
    nz, dt = 4, 0.3
    s2 = random_state3(nx, ny, 1, 23, fmax=0.8)[[0, 1, 2, 4], 0]
    sa2, ss2 = opacities((ny, nx), 24)
    in2 = _beam_2d(ny)
    bc2 = ("inflow", "reflect", "reflect", "neumann")
    g2 = O.Grid(2, nx, ny, 1.0 / nx, 1.0 / ny, 1.0, 1.0, 1.0, bc2, in2)
    a2 = O.apply_A(g2, dt, sa2, ss2, s2)
    g3 = O3.Grid3(nx, ny, nz, 1.0 / nx, 1.0 / ny, 0.5, bc2 + ("periodic", "periodic"))
    face_E = np.repeat(in2[0, 0][None], nz, 0)              # (nz, ny): index k*ny + j
    face_F = [np.repeat(in2[0, 1][None], nz, 0), np.repeat(in2[0, 2][None], nz, 0),
              np.zeros((nz, ny))]
    g3.inflow = _inflow3(g3, 0, face_E, face_F)
    s3 = np.zeros(g3.shape)
    s3[[0, 1, 2, 4]] = s2[:, None]
    a3 = O3.apply_A(g3, dt, np.repeat(sa2[None], nz, 0), np.repeat(ss2[None], nz, 0), s3)
    for k in range(nz):
        assert rel(a3[[0, 1, 2, 4], k], a2) <= 1e-13
    assert np.abs(a3[3]).max() == 0.0


def test_z_uniform_inflow_step_reaches_the_2d_fixed_point():
    """The whole step with an inflow wall (coarse profiles restricted along the
    wall) reaches the 2D oracle's fixed point."""
    nx = ny = 16
    s2 = random_state3(nx, ny, 1, 25, fmax=0.6)[[0, 1, 2, 4], 0]
    sa2, ss2 = opacities((ny, nx), 26, -1.0, 1.0)
    in2 = _beam_2d(ny)
    bc2 = ("inflow", "neumann", "reflect", "reflect")
    dt = 2.0 / nx
    g2 = O.Grid(2, nx, ny, 1.0 / nx, 1.0 / ny, 1.0, 1.0, 1.0, bc2, in2)
    ref, _, h2, _ = O.implicit_step(g2, dt, sa2, ss2, s2,
                                    O.SolveParams(lmax=3, tol=0.0, max_cycles=600))
    assert h2[-1] <= 1e-14 * h2[0]
    nz = 4
    g3 = O3.Grid3(nx, ny, nz, 1.0 / nx, 1.0 / ny, 0.25, bc2 + ("periodic", "periodic"))
    g3.inflow = _inflow3(g3, 0, np.repeat(in2[0, 0][None], nz, 0),
                         [np.repeat(in2[0, 1][None], nz, 0), np.repeat(in2[0, 2][None], nz, 0),
                          np.zeros((nz, ny))])
    s3 = np.zeros(g3.shape)
    s3[[0, 1, 2, 4]] = s2[:, None]
    out, _, h3 = O3.implicit_step(g3, dt, np.repeat(sa2[None], nz, 0), np.repeat(ss2[None], nz, 0),
                                  s3, O3.SolveParams3(lmax=3, tol=0.0, max_cycles=600))
    assert h3[-1] <= 1e-14 * h3[0]
    for k in range(nz):
        assert rel(out[[0, 1, 2, 4], k], ref) <= 1e-11


def test_free_streaming_front_along_z_satisfies_upwind_recurrence():
    """No matter, F = cE along z everywhere and an f = 1 beam entering through the
    z-low wall: the x and y faces cancel their diagonal terms, and the step solves
    (1 + alpha) E_k - alpha E_{k-1} = E^n_k exactly, with F = cE kept."""
    nx = ny = 4
    nz, c, cfl = 64, 1.0, 8.0
    g = O3.Grid3(nx, ny, nz, 0.25, 0.25, 1.0 / nz,
                 ("periodic",) * 4 + ("inflow", "neumann"), c=c)
    face = g.nx * g.ny
    g.inflow = _inflow3(g, 4, np.ones(face), [np.zeros(face), np.zeros(face), c * np.ones(face)])
    v = np.zeros(g.shape)
    v[0] = 1e-6
    v[3] = c * 1e-6
    v[4] = 1.0
    z = np.zeros((nz, ny, nx))
    out, st, _ = O3.implicit_step(g, cfl / nz, z, z, v, O3.SolveParams3(lmax=3, tol=1e-14,
                                                                        max_cycles=2000))
    assert st["status"] == 0
    E = np.concatenate([[1.0], out[0][:, 0, 0]])
    np.testing.assert_allclose((1 + cfl) * E[1:] - cfl * E[:-1], v[0][:, 0, 0], rtol=0,
                               atol=1e-13)
    np.testing.assert_allclose(out[3], c * out[0], rtol=1e-12)
    assert np.abs(out[1:3]).max() <= 1e-14
    assert np.ptp(out[0], axis=(1, 2)).max() <= 1e-14           # uniform across x, y


def test_multigrid_step_matches_brute_force_newton_with_inflow():
    g = O3.Grid3(4, 4, 4, 0.25, 0.25, 0.25,
                 ("inflow", "reflect", "periodic", "periodic", "neumann", "reflect"))
    rng = np.random.default_rng(27)
    E_in = 10.0 ** rng.uniform(-0.5, 0.5, 16)
    d = rng.standard_normal((3, 16))
    d /= np.linalg.norm(d, axis=0)
    F_in = 0.8 * E_in * d
    g.inflow = _inflow3(g, 0, E_in, F_in)
    v0 = random_state3(4, 4, 4, 28, fmax=0.7)
    sa, ss = opacities((4, 4, 4), 29, -1.0, 1.0)
    dt = 0.8
    mg, st, hist = O3.implicit_step(g, dt, sa, ss, v0, O3.SolveParams3(lmax=2, tol=0.0,
                                                                        max_cycles=1500))
    assert hist[-1] <= 1e-15 * hist[0]
    nw = _newton_solve3(g, dt, sa, ss, v0.copy(), mg * (1 + 1e-3 * rng.standard_normal(mg.shape)))
    np.testing.assert_allclose(mg, nw, rtol=0, atol=1e-11 * np.abs(nw[0]).max())
