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


# ---- the random streams ----

def test_splitmix64_reference_outputs():
    """splitmix64 (Steele, Lea & Flood, OOPSLA 2014) started at state 0 yields
    0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f."""
    got = [int(x) for x in inputs.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_normal_moments():
    u = inputs.uniform(3, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    z = inputs.normal(4, 200_000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert abs((np.abs(z) < 1.0).mean() - 0.6827) < 0.005          # one-sigma mass


def test_opacity_field_recipe():
    """log10 sigma = 1 + 3 g, g a zero-mean unit-variance field smoothed over
    about 8 cells, clipped to [-2, 4] (one g-sigma on each side), so about 32%
    of the cells sit on a clip and sigma spans 1e-2 .. 1e4."""
    g = inputs.gaussian_field(256, 256, 1)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    lag1 = np.corrcoef(g[:, :-1].ravel(), g[:, 1:].ravel())[0, 1]
    lag64 = np.corrcoef(g[:, :-64].ravel(), g[:, 64:].ravel())[0, 1]
    assert lag1 > 0.95 and abs(lag64) < 0.15
    s = np.log10(inputs.lognormal_opacity(256, 256, 1))
    assert s.min() >= -2.0 - 1e-12 and s.max() <= 4.0 + 1e-12
    clipped = np.mean((s <= -2.0 + 1e-12) | (s >= 4.0 - 1e-12))
    assert 0.2 < clipped < 0.45


# ---- the workload recipes ----

def test_gaussian_1d_recipe():
    c = inputs.gaussian_1d(256)
    x = (np.arange(256) + 0.5) / 256
    np.testing.assert_allclose(c["state"][0, 0], 1e-2 + np.exp(-(x - 0.5) ** 2 / 0.005))
    np.testing.assert_array_equal(c["state"][[1, 2]], 0.0)
    np.testing.assert_array_equal(c["state"][3], 1.0)
    assert np.all(c["sa"] == 1.0) and np.all(c["ss"] == 1.0)
    assert c["desc"]["bc"] == ["periodic"] * 4 and c["lmax"] == 4 and c["tol"] == 1e-10
    assert c["dt"] == pytest.approx(50.0 / 256)


def test_hot_square_recipe():
    n = 256
    c = inputs.hot_square_2d(n)
    T = c["state"][3]
    assert (T == 4.0).sum() == (n // 8) ** 2 and set(np.unique(T)) == {1.0, 4.0}
    hot = np.argwhere(T == 4.0)
    assert hot.min() == n // 2 - n // 16 and hot.max() == n // 2 + n // 16 - 1
    np.testing.assert_array_equal(c["state"][0], T ** 4)
    assert c["desc"]["bc"] == ["reflect"] * 4 and c["lmax"] == 8 and c["tol"] == 1e-8
    assert c["dt"] == pytest.approx(100.0 / n)


def test_beam_channel_recipe():
    n = 256
    c = inputs.beam_channel_2d(n)
    y = (np.arange(n) + 0.5) / n
    chan = (y >= 0.45) & (y <= 0.55)
    assert np.all(c["sa"][chan] == 1e-2) and np.all(c["ss"][chan] == 1e-2)
    assert np.all(c["inflow"][0, 0] == 1.0)
    np.testing.assert_array_equal(c["inflow"][0, 1], np.where(chan, 1.0, 0.0))
    assert c["desc"]["bc"] == ["inflow", "reflect", "reflect", "reflect"] and c["lmax"] == 10
    np.testing.assert_array_equal(c["state"][0], 1.0)


def test_riemann_quadrants():
    c = inputs.riemann_2d(64)
    k = 1.0 - 1e-8
    s = c["state"]
    assert s[1, 0, 0] == k and s[2, 0, 0] == 0.0           # bottom-left: +x
    assert s[1, 0, -1] == 0.0 and s[2, 0, -1] == -k        # bottom-right: -y
    assert s[1, -1, 0] == 0.0 and s[2, -1, 0] == k         # top-left: +y
    assert s[1, -1, -1] == -k and s[2, -1, -1] == 0.0      # top-right: -x
    assert c["desc"]["bc"] == ["periodic"] * 4


def test_batched_instances_recipe():
    cases = inputs.batched_instances(70)
    sizes = [c["desc"]["nx"] for c in cases]
    allowed = (64, 96, 128, 192, 256, 512, 1024)
    assert set(sizes) == set(allowed)
    counts = np.array([sizes.count(s) for s in allowed])
    assert np.all(np.abs(counts - 10) < 4 * np.sqrt(10))
    for c in cases[:20]:
        E = c["state"][0]
        assert E.min() >= 1.0 and E.max() <= 101.0
        assert c["lmax"] == 5 and c["desc"]["bc"] == ["reflect"] * 4
        assert c["desc"]["nx"] % 32 == 0            # divisible by 2^L_max


def test_serving_stream_recipe():
    """Poisson arrivals (exponential gaps of mean 1/rate), 1D or 2D with
    probability 1/2, 10..100 steps (statistics on a stream of small grids: they
    do not depend on the sizes), sizes from the given sets."""
    reqs = inputs.serving_stream(400, rate_hz=20.0, sizes_1d=(256,), sizes_2d=(32,))
    t = np.array([r["arrival_s"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 0.05) < 0.01
    assert abs(np.std(gaps) / np.mean(gaps) - 1.0) < 0.2        # exponential: cv = 1
    dims = np.array([r["case"]["desc"]["dim"] for r in reqs])
    assert abs((dims == 1).mean() - 0.5) < 0.1
    steps = np.array([r["nsteps"] for r in reqs])
    assert steps.min() >= 10 and steps.max() <= 100 and abs(steps.mean() - 55) < 6
    for r in inputs.serving_stream(8):
        d = r["case"]["desc"]
        if d["dim"] == 1:
            assert d["nx"] in (256, 512, 1024, 2048, 4096, 8192, 16384, 32768, 65536)
        else:
            assert d["nx"] == d["ny"] and d["nx"] in (128, 256, 512, 1024, 2048)


def test_beam_window_holds_the_beam():
    # the 1024^2 window of the 4096^2 beam-in-a-channel grid, on the west wall and
    # centred on the channel: same cell size and time step as the full grid, the
    # channel rows (y in [0.45, 0.55] of the full grid) inside, the f = 1 beam on
    # exactly those rows of the west wall
    full = inputs.beam_channel_2d(4096)
    win = inputs.beam_channel_crop(1024)
    h = 1.0 / 4096
    assert win["desc"]["nx"] == win["desc"]["ny"] == 1024
    assert win["desc"]["lx"] == pytest.approx(1024 * h) and win["dt"] == full["dt"]
    rows = 1536 + np.arange(1024)
    y = (rows + 0.5) * h
    chan = (y >= 0.45) & (y <= 0.55)
    assert chan.sum() == 410
    np.testing.assert_array_equal(win["inflow"][0, 1], np.where(chan, 1.0, 0.0))
    np.testing.assert_array_equal(win["inflow"][0, 0], 1.0)
    np.testing.assert_array_equal(win["sa"], full["sa"][1536:2560, :1024])
    assert np.all(win["sa"][chan] == 1e-2)
