"""The strip-height table of the sweep kernels: defaults and installed entries
(host logic, no GPU needed); on the GPU, the autotuner's output and the fact
that the strip height changes no arithmetic (bitwise equal steps)."""
import numpy as np
import pytest

from paper_2208_14703_gb300 import inputs

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")


@pytest.fixture
def restore_tuning():
    yield
    m1.set_tuning([{"kind": k, "n": 1 << c, "strip_rows": 0} for k in (0, 1) for c in range(16)])


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


@pytest.mark.gpu
def test_autotune_entries(restore_tuning):
    ent = m1.autotune()
    assert {(e["kind"], e["n"]) for e in ent} == {(k, 1 << c) for k in (0, 1) for c in range(4, 12)}
    for e in ent:
        assert e["strip_rows"] in (1, 2, 4, 8, 16, 32) and e["strip_rows"] <= e["n"]
        assert e["ms"] > 0 and (np.isnan(e["ms_default"]) or e["ms"] <= e["ms_default"])
        assert m1.strip_rows(e["kind"], e["n"], e["n"]) == e["strip_rows"]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_strip_height_changes_no_arithmetic(precision, restore_tuning):
    case = inputs.hot_square_2d(128, lmax=5)
    outs = []
    for rows in (1, 32):
        m1.set_tuning([{"kind": k, "n": 1 << c, "strip_rows": rows} for k in (0, 1)
                       for c in range(16)])
        g = m1.grid_from_case(case, precision=precision)
        st = g.implicit_step(case["dt"], m1.m1_default_params(tol=1e-8))
        outs.append((st.cycles, np.stack(g.get_state())))
        g.close()
    assert outs[0][0] == outs[1][0]
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
