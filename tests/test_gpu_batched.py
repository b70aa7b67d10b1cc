"""Batches: independent instances of uneven sizes (1D and 2D mixed) stepped
together by one persistent launch per level and kernel.  Each instance's
result must equal, bit for bit, the same instance stepped alone (its arithmetic
and its reductions never involve another instance), and the FP64 results must
match the oracle like single grids do."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14703_gb300 import inputs

pytestmark = pytest.mark.gpu

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")


def mixed_bag():
    """Instances of uneven sizes sharing L_max = 4 (sizes divisible by 8)."""
    cases = []
    for k, n in enumerate([64, 96, 32, 128, 40, 72]):
        c = inputs.random_admissible_2d(n, n, seed=100 + k, fmax=0.9, cfl=30,
                                        bc=("reflect",) * 4, lmax=4)
        c["tol"] = 1e-8
        cases.append(c)
    for n in (256, 512):
        c = inputs.gaussian_1d(n, lmax=4)
        c["tol"] = 1e-8
        cases.append(c)
    cases.append(inputs.beam_channel_2d(64, lmax=4))
    cases.append(inputs.hot_square_2d(64, lmax=4))
    return cases


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_instances_alone(precision):
    cases = mixed_bag()
    params = m1.m1_default_params(tol=1e-8)
    b = m1.batch_from_cases(cases, precision=precision)
    stats = b.implicit_step([c["dt"] for c in cases], params)
    together = [np.stack(b.get_state(k)) for k in range(len(cases))]
    b.close()
    for k, c in enumerate(cases):
        g = m1.grid_from_case(c, precision=precision)
        st = g.implicit_step(c["dt"], params)
        alone = np.stack(g.get_state())
        g.close()
        assert st.cycles == stats[k].cycles, k
        np.testing.assert_array_equal(alone, together[k])


def test_batch_fp64_matches_oracle():
    cases = mixed_bag()[:4] + mixed_bag()[6:7]
    params = m1.m1_default_params(tol=1e-8)
    b = m1.batch_from_cases(cases)
    stats = b.implicit_step([c["dt"] for c in cases], params)
    for k, c in enumerate(cases):
        og = O.Grid.from_case(c)
        ref, ost, _, _ = O.implicit_step(og, c["dt"], c["sa"], c["ss"], c["state"],
                                         O.SolveParams(lmax=4, tol=1e-8))
        out = np.stack(b.get_state(k))
        assert stats[k].cycles == ost["cycles"], k
        nE = np.linalg.norm(ref[0])
        assert np.linalg.norm(out[0] - ref[0]) / nE <= 1e-10
        assert np.linalg.norm(out[1:3] - ref[1:3]) / nE <= 1e-10
        assert np.linalg.norm(out[3] - ref[3]) / np.linalg.norm(ref[3]) <= 1e-10
    b.close()


def test_batch_rejects_mixed_level_counts():
    a = m1.desc_from_case(inputs.gaussian_1d(64, lmax=2))
    c = m1.desc_from_case(inputs.gaussian_1d(64, lmax=3))
    with pytest.raises(m1.M1Error):
        m1.Batch([a, c])
