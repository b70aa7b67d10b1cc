"""The synthetic workloads are the setups they claim to be (CPU only)."""
import numpy as np
import pytest

from paper_2208_14703_gb300 import inputs


def test_paper_beam_is_the_section_4_1_setup():
    c = inputs.paper_beam_2d(64)
    d = c["desc"]
    assert (d["nx"], d["ny"], d["lx"], d["ly"]) == (64, 64, 2.0, 2.0)
    assert d["bc"][0] == "inflow" and not c["sa"].any() and not c["ss"].any()
    y = -1.0 + (np.arange(64) + 0.5) * (2.0 / 64)
    beam = (y >= -0.875) & (y <= -0.75)
    assert beam.sum() == 4                            # 0.125 of the height of 2
    e = c["inflow"][0, 0]
    np.testing.assert_allclose(e[beam], (1000 / 300) ** 4)
    np.testing.assert_array_equal(e[~beam], 1.0)
    # f = 1 at 45 degrees: |F| = c E, Fx = Fy
    fx, fy = c["inflow"][0, 1], c["inflow"][0, 2]
    np.testing.assert_allclose(np.hypot(fx, fy)[beam], e[beam])
    np.testing.assert_array_equal(fx, fy)
    assert c["dt"] == pytest.approx(2000 * 2.0 / 64) and c["tol"] == 1e-2
    np.testing.assert_array_equal(c["state"][0], 1.0)
    np.testing.assert_array_equal(c["state"][1:3], 0.0)
