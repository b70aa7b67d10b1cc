"""The strip-shape table of the sweep kernels: defaults and installed entries
(host logic, no GPU needed); on the GPU, the autotuner's output, the fact that
the strip height changes no arithmetic (bitwise equal steps) and that the two
row stagings of the FP32 correction form agree to rounding."""
import numpy as np
import pytest

from paper_2208_14703_gb300 import inputs

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")


@pytest.fixture
def restore_tuning():
    yield
    m1.set_tuning([{"kind": k, "n": 1 << c, "strip_rows": 0, "staging": 0} for k in (0, 1)
                   for c in range(16)])


def test_default_strip_rows(restore_tuning):
    for kind in (0, 1):
        assert m1.strip_rows(kind, 2048, 2048) == 16
        assert m1.strip_rows(kind, 1024, 1024) == 16
        assert m1.strip_rows(kind, 512, 512) == 8
        assert m1.strip_rows(kind, 64, 64) == 1
        assert m1.strip_rows(kind, 16, 16) == 1


def test_installed_entries_and_reset(restore_tuning):
    m1.set_tuning([{"kind": 1, "n": 256, "strip_rows": 8}, {"kind": 0, "n": 32, "strip_rows": 32}])
    assert m1.strip_rows(1, 256, 256) == 8
    assert m1.strip_rows(0, 256, 256) == 4          # the other kind keeps its default
    assert m1.strip_rows(0, 32, 32) == 32
    assert m1.strip_rows(0, 32, 16) == 16           # never taller than the level
    m1.set_tuning([{"kind": 1, "n": 256, "strip_rows": 0}])
    assert m1.strip_rows(1, 256, 256) == 4
    with pytest.raises(m1.M1Error):
        m1.set_tuning([{"kind": 2, "n": 256, "strip_rows": 8}])
    with pytest.raises(m1.M1Error):
        m1.set_tuning([{"kind": 0, "n": 256, "strip_rows": 8, "staging": 1}])
    m1.set_tuning([{"kind": 1, "n": 4096, "strip_rows": 128, "staging": 1}])
    assert m1.strip_rows(1, 4096, 4096) == 128
    with pytest.raises(m1.M1Error):
        m1.set_tuning([{"kind": 1, "n": 4096, "strip_rows": 257}])


@pytest.mark.gpu
def test_autotune_entries(restore_tuning):
    ent = m1.autotune()
    assert {(e["kind"], e["n"]) for e in ent} == (
        {(0, 1 << c) for c in range(4, 12)} | {(1, 1 << c) for c in range(4, 13)})
    for e in ent:
        assert e["strip_rows"] in (1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128)
        assert e["strip_rows"] <= e["n"]
        assert e["staging"] in ((0,) if e["kind"] == 0 else (0, 1))
        assert e["ms"] > 0 and (np.isnan(e["ms_default"]) or e["ms"] <= e["ms_default"])
        assert m1.strip_rows(e["kind"], e["n"], e["n"]) == e["strip_rows"]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_strip_shape_changes_no_arithmetic(precision, restore_tuning):
    """Strip heights 1, 24 and 32 give bitwise equal steps (the same kernel,
    every cell's update the same whatever strip it falls in; 24 rows leave a
    partial strip at the top of every level).  The two row stagings of
    the FP32 correction form are two kernels whose FP32 contractions may round
    differently, so their steps agree to rounding: same cycle count, results
    within 1e-10 relative.  Checked on a square hot-square grid and on a ragged
    periodic grid."""
    cases = [inputs.hot_square_2d(128, lmax=5),
             inputs.random_admissible_2d(80, 48, seed=9, fmax=0.95, cfl=20,
                                         bc=("periodic",) * 4, lmax=3)]
    cases[1]["tol"] = 1e-8
    for case in cases:
        outs = {}
        for rows, staging in ((1, 0), (24, 0), (32, 0), (1, 1), (24, 1), (32, 1)):
            if staging and precision == 0:
                continue
            m1.set_tuning([{"kind": k, "n": 1 << c, "strip_rows": rows,
                            "staging": staging if k == 1 else 0}
                           for k in (0, 1) for c in range(16)])
            g = m1.grid_from_case(case, precision=precision)
            st = g.implicit_step(case["dt"], m1.m1_default_params(tol=case["tol"]))
            outs[rows, staging] = (st.cycles, np.stack(g.get_state()))
            g.close()
        for staging in (0, 1) if precision else (0,):
            for rows in (24, 32):
                assert outs[rows, staging][0] == outs[1, staging][0]
                np.testing.assert_array_equal(outs[rows, staging][1], outs[1, staging][1])
        if precision:
            a, b = outs[1, 0], outs[1, 1]
            assert a[0] == b[0]
            for f in range(4):
                assert np.linalg.norm(a[1][f] - b[1][f]) <= 1e-10 * np.linalg.norm(a[1][0])


@pytest.mark.gpu
def test_ring_staging_serves_1d_instances_of_a_batch(restore_tuning):
    """A batch mixing 2D and 1D instances, with every size class tuned to the
    cp.async staging: the 2D instances choose it for every level, so the 1D
    instances' strips run through that kernel's one-row path.  Their steps agree
    with the register staging to rounding."""
    cases = [inputs.hot_square_2d(64, lmax=4), inputs.random_admissible_2d(
        48, 32, seed=5, fmax=0.9, cfl=20, bc=("periodic",) * 4, lmax=4),
        inputs.gaussian_1d(64, lmax=4), inputs.gaussian_1d(128, lmax=4)]
    cases[1]["tol"] = 1e-8
    outs = {}
    for staging in (0, 1):
        m1.set_tuning([{"kind": k, "n": 1 << c, "strip_rows": 0,
                        "staging": staging if k == 1 else 0} for k in (0, 1) for c in range(16)])
        b = m1.batch_from_cases(cases, precision=m1.MIXED)
        st = b.implicit_step([c["dt"] for c in cases], m1.m1_default_params(tol=1e-10))
        outs[staging] = ([s.cycles for s in st],
                         [np.stack(b.get_state(k)) for k in range(len(cases))])
        b.close()
    assert outs[0][0] == outs[1][0]
    for a, b in zip(outs[0][1], outs[1][1]):
        for f in range(4):
            assert np.linalg.norm(a[f] - b[f]) <= 1e-10 * np.linalg.norm(a[0])
