"""Pins of the oracle's grid transfers (Section 4.2): the paper's printed 1D
matrices (Eqs. (19)-(20)), the printed 2D stencils (Eqs. (18), (22)), the
identity R = 2^-d P^T, constants, convexity and conservation."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.conftest import read_golden


def _matrix_P(g, kind, inflow_c=None):
    """Prolongation matrix (fine scalar E plane <- coarse E plane), built by
    applying the oracle to unit vectors."""
    gc = g.coarse()
    M = np.zeros((g.n, gc.n))
    for k in range(gc.n):
        e = np.zeros((4, gc.ny, gc.nx))
        e.reshape(4, -1)[0, k] = 1.0
        M[:, k] = O.prolong(g, e, kind, inflow_c).reshape(4, -1)[0]
    return M


def _matrix_R(g, kind):
    gc = g.coarse()
    M = np.zeros((gc.n, g.n))
    for k in range(g.n):
        e = np.zeros((4, g.ny, g.nx))
        e.reshape(4, -1)[0, k] = 1.0
        M[:, k] = O.restrict_state(g, e, kind).reshape(4, -1)[0]
    return M


def test_paper_1d_example_matrices():
    rows = read_golden("transfer_1d_paper.txt")
    P_paper = 0.5 * np.array(rows[:7], dtype=float)
    R_paper = 0.25 * np.array(rows[7:], dtype=float)
    # 8 fine / 4 coarse cells with a zero outside value (the error ghost of an
    # inflow wall); the paper's 7 x 3 example is this operator without the first
    # fine and first coarse cell (its fine cell 1 sees a zero coarse cell 0).
    L = 8
    g = O.Grid(1, 8, 1, 1 / 8, 1.0, bc=("inflow",) * 4, inflow=np.zeros((4, 3, L)))
    P = _matrix_P(g, O.KIND_DIFF)
    R = _matrix_R(g, O.KIND_DIFF)
    np.testing.assert_array_equal(P[1:, 1:], P_paper)
    np.testing.assert_array_equal(R[1:, 1:], R_paper)
    # and the defining relation R = (1/2) P^T holds for the whole operator
    np.testing.assert_array_equal(R, 0.5 * P.T)


def test_paper_2d_stencils():
    W = np.array(read_golden("restriction_2d_stencil.txt"), dtype=float)
    g = O.Grid(2, 8, 8, 1 / 8, 1 / 8, bc=("periodic",) * 4)
    R = _matrix_R(g, O.KIND_STATE)
    # coarse cell (ic, jc) = (1, 2) gathers fine cells (2ic + a, 2jc + b)
    row = R[2 * 4 + 1].reshape(8, 8)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            assert row[4 + b, 2 + a] == W[a + 1, b + 1]
    assert row.sum() == 1.0
    P = _matrix_P(g, O.KIND_STATE)
    for ipar, jpar, *w in np.array(read_golden("prolongation_2d_weights.txt"), dtype=float):
        i, j = 2 * 1 + int(ipar), 2 * 1 + int(jpar)
        col = P[j * 8 + i].reshape(4, 4)
        np.testing.assert_array_equal([col[1, 1], col[1, 2], col[2, 1], col[2, 2]], w)


@pytest.mark.parametrize("dim", [1, 2])
def test_restriction_is_scaled_transpose_of_prolongation_periodic(dim):
    g = O.Grid(dim, 8, 8, 1 / 8, 1 / 8, bc=("periodic",) * 4)
    P = _matrix_P(g, O.KIND_STATE)
    R = _matrix_R(g, O.KIND_STATE)
    np.testing.assert_array_equal(R, P.T / 2 ** dim)


@pytest.mark.parametrize("dim,bc", [(1, "periodic"), (1, "reflect"), (2, "periodic"),
                                    (2, "reflect"), (2, "neumann")])
def test_transfers_are_convex_and_keep_constants(dim, bc):
    g = O.Grid(dim, 8, 8, 1 / 8, 1 / 8, bc=(bc,) * 4)
    for M in (_matrix_P(g, O.KIND_STATE), _matrix_R(g, O.KIND_STATE)):
        assert M.min() >= 0
        np.testing.assert_allclose(M.sum(axis=1), 1.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim", [1, 2])
def test_restriction_conserves_totals_periodic(dim):
    rng = np.random.default_rng(2)
    g = O.Grid(dim, 16, 16, 1 / 16, 1 / 16, bc=("periodic",) * 4)
    f = rng.uniform(0.1, 1, (4, g.ny, g.nx))
    c = O.restrict_state(g, f)
    np.testing.assert_allclose(c.reshape(4, -1).sum(1) * 2 ** dim, f.reshape(4, -1).sum(1),
                               rtol=1e-14)


def test_transfers_keep_admissible_states_admissible():
    rng = np.random.default_rng(4)
    g = O.Grid(2, 16, 16, 1 / 16, 1 / 16, bc=("reflect",) * 4)
    E = 10 ** rng.uniform(-2, 2, (16, 16))
    th = rng.uniform(0, 2 * np.pi, (16, 16))
    f = rng.uniform(0.9, 1.0, (16, 16))
    s = np.stack([E, f * E * np.cos(th), f * E * np.sin(th), np.ones((16, 16))])
    c = O.restrict_state(g, s)
    assert np.all(c[0] > 0) and np.all(np.hypot(c[1], c[2]) <= c[0] * (1 + 1e-15))
    p = O.prolong(g, c, O.KIND_STATE)
    assert np.all(p[0] > 0) and np.all(np.hypot(p[1], p[2]) <= p[0] * (1 + 1e-15))


def test_reflect_ghost_negates_normal_flux_in_restriction():
    # a field odd in x (Fx antisymmetric about the west wall) restricted next to
    # a reflecting wall: coarse cell 0 gets 1/4*(-Fx_0) + 1/2 Fx_0 + 1/4 Fx_1
    g = O.Grid(1, 8, 1, 1 / 8, 1.0, bc=("reflect",) * 4)
    f = np.zeros((4, 1, 8))
    f[1, 0] = np.arange(1, 9, dtype=float)
    f[0] = 100.0
    c = O.restrict_state(g, f)
    assert c[1, 0, 0] == pytest.approx(-0.25 * 1 + 0.5 * 1 + 0.25 * 2)
    assert c[0, 0, 0] == pytest.approx(100.0)
