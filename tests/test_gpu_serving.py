"""Serving: requests of uneven sizes (1D and 2D) admitted into a running engine
in arrival order under an HBM budget, each stepped several times with its own
step length and tolerance while others join and leave.  A served request's
result must equal, bit for bit, the same steps run on its grid alone (the
instances never share arithmetic), whatever it was batched with."""
import time

import numpy as np
import pytest

from paper_2208_14703_gb300 import inputs

pytestmark = pytest.mark.gpu

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")


def requests(lmax=4):
    out = []
    for k, n in enumerate([64, 32, 96, 48]):
        c = inputs.random_admissible_2d(n, n, seed=300 + k, fmax=0.9, cfl=20,
                                        bc=("reflect",) * 4, lmax=lmax)
        out.append((c, 3 + k % 2, 1e-8))
    out.append((inputs.gaussian_1d(256, lmax=lmax), 4, 1e-9))
    out.append((inputs.beam_channel_2d(64, lmax=lmax), 1, 1e-8))
    out.append((inputs.hot_square_2d(64, lmax=lmax), 3, 1e-7))
    return out


def run_alone(case, nsteps, tol, precision):
    g = m1.grid_from_case(case, precision=precision)
    p = m1.m1_default_params(tol=tol)
    cycles = []
    for _ in range(nsteps):
        cycles.append(g.implicit_step(case["dt"], p).cycles)
    out = np.stack(g.get_state())
    g.close()
    return out, cycles


def serve(reqs, precision, budget, max_slots, stagger=False, small_cells=m1.SMALL_CELLS):
    srv = m1.Server(budget, max_slots, reqs[0][0]["lmax"], precision, small_cells=small_cells)
    grids, tickets = [], []
    for k, (c, nsteps, tol) in enumerate(reqs):
        g = m1.grid_from_case(c, precision=precision)
        grids.append(g)
        tickets.append(srv.submit(g, nsteps, c["dt"], m1.m1_default_params(tol=tol)))
        if stagger and k % 2 == 1:
            time.sleep(0.01)
    for t in tickets:
        assert srv.wait(t, 300.0) == m1.OK
    stats = srv.stats()
    lasts = [srv.poll(t) for t in tickets]
    srv.close()
    outs = [np.stack(g.get_state()) for g in grids]
    for g in grids:
        g.close()
    return outs, lasts, stats


@pytest.mark.parametrize("precision", [0, 1])
def test_served_equals_alone(precision):
    reqs = requests()
    outs, lasts, stats = serve(reqs, precision, budget=1 << 34, max_slots=8, stagger=True)
    for k, (c, nsteps, tol) in enumerate(reqs):
        alone, cycles = run_alone(c, nsteps, tol, precision)
        st, done, last = lasts[k]
        assert st == m1.OK and done == nsteps
        assert last.cycles == cycles[-1], k
        np.testing.assert_array_equal(alone, outs[k])
    assert stats.requests_done == len(reqs)
    assert stats.steps_done == sum(n for _, n, _ in reqs)
    assert 0 < stats.p50_ms <= stats.p99_ms
    assert stats.active == 0 and stats.queued == 0 and stats.bytes_in_use == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_small_and_large_lanes_equal_alone(precision):
    """A 384^2 request (147456 cells) runs in the large lane, beside small
    requests in the small lane (their own engine, stream and scheduler thread):
    every result equals the same steps run alone, and so does a one-lane server
    (small_cells 0) on the same mix."""
    big = inputs.hot_square_2d(384, lmax=4, tol=1e-7)
    reqs = [(big, 2, 1e-7)] + requests()[:3] + requests()[4:5]
    alone = [run_alone(c, n, tol, precision) for c, n, tol in reqs]
    for small in (m1.SMALL_CELLS, 0):
        outs, lasts, stats = serve(reqs, precision, budget=1 << 34, max_slots=4, small_cells=small)
        for k, (c, nsteps, tol) in enumerate(reqs):
            st, done, last = lasts[k]
            assert st == m1.OK and done == nsteps
            assert last.cycles == alone[k][1][-1], (small, k)
            np.testing.assert_array_equal(alone[k][0], outs[k])
        assert stats.requests_done == len(reqs) and stats.bytes_in_use == 0


def test_budget_bounds_resident_bytes():
    """A budget (2.5 MB) below the three hierarchies' sum (about 3.3 MB in FP64):
    the later request waits for memory, the device bytes in use never pass the
    budget, and the results are unchanged."""
    reqs = requests()[:3]
    budget = 5 << 19
    outs, lasts, stats = serve(reqs, 0, budget=budget, max_slots=4)
    for k, (c, nsteps, tol) in enumerate(reqs):
        alone, _ = run_alone(c, nsteps, tol, 0)
        np.testing.assert_array_equal(alone, outs[k])
    assert stats.requests_done == 3
    assert 0 < stats.bytes_peak <= budget


def test_over_budget_rejected_and_bad_requests():
    c = inputs.random_admissible_2d(64, 64, seed=1, fmax=0.5, cfl=5, bc=("reflect",) * 4, lmax=3)
    g = m1.grid_from_case(c)
    srv = m1.Server(1 << 16, 2, 3)          # 64 KB: smaller than the grid's hierarchy
    with pytest.raises(m1.M1Error) as e:
        srv.submit(g, 1, c["dt"])
    assert e.value.status == m1.ERR_REJECTED
    srv.close()
    srv = m1.Server(1 << 30, 2, 4)           # level count differs from the grid's
    with pytest.raises(m1.M1Error):
        srv.submit(g, 1, c["dt"])
    with pytest.raises(m1.M1Error):
        srv.submit(g, 0, c["dt"])
    srv.close()
    g.close()


def test_not_converged_request_stops_alone():
    """The beam channel (64^2, CFL 100) takes 358 cycles for its first step and
    does not converge on its second (the oracle's residual grows there too).
    With max_cycles 400 the request ends after its second step with
    NOT_CONVERGED and the last iterate, while a request batched with it is
    unaffected."""
    beam = inputs.beam_channel_2d(64, lmax=4)
    other = requests()[1][0]
    p_beam = m1.m1_default_params(tol=1e-8, max_cycles=400)
    p_other = m1.m1_default_params(tol=1e-8)
    srv = m1.Server(1 << 34, 4, 4)
    gb, go = m1.grid_from_case(beam), m1.grid_from_case(other)
    tb = srv.submit(gb, 3, beam["dt"], p_beam)
    to = srv.submit(go, 3, other["dt"], p_other)
    assert srv.wait(tb, 300.0) == m1.ERR_NOT_CONVERGED
    assert srv.wait(to, 300.0) == m1.OK
    st, done, last = srv.poll(tb)
    assert st == m1.ERR_NOT_CONVERGED and done == 2 and last.cycles == 400
    srv.close()
    served_b, served_o = np.stack(gb.get_state()), np.stack(go.get_state())
    gb.close()
    go.close()
    g = m1.grid_from_case(beam)
    assert g.implicit_step(beam["dt"], p_beam).cycles == 358
    g.implicit_step(beam["dt"], p_beam, allow_not_converged=True)
    np.testing.assert_array_equal(np.stack(g.get_state()), served_b)
    g.close()
    alone_o, _ = run_alone(other, 3, 1e-8, 0)
    np.testing.assert_array_equal(alone_o, served_o)


def test_poll_reports_progress_and_queue():
    reqs = requests()[:2]
    srv = m1.Server(1 << 34, 1, 4)             # one slot: the second request queues
    grids = [m1.grid_from_case(c) for c, _, _ in reqs]
    ts = [srv.submit(g, n, c["dt"], m1.m1_default_params(tol=tol))
          for g, (c, n, tol) in zip(grids, reqs)]
    st, done, _ = srv.poll(ts[1])
    assert st in (m1.PENDING, m1.OK)
    for t in ts:
        assert srv.wait(t, 300.0) == m1.OK
    for t, (_, n, _) in zip(ts, reqs):
        st, done, last = srv.poll(t)
        assert st == m1.OK and done == n and last.res <= last.res0
    s = srv.stats()
    assert s.requests_done == 2 and s.cycles > 0 and s.solves_per_s > 0
    srv.close()
    for g in grids:
        g.close()


def test_destroy_finishes_submitted_requests():
    """Destroying a server right after submitting finishes every request first:
    each grid then holds the result of its steps, the same as run alone."""
    reqs = requests()[:3]
    srv = m1.Server(1 << 34, 2, 4)                # two slots: the third request queues
    grids = [m1.grid_from_case(c) for c, _, _ in reqs]
    for g, (c, n, tol) in zip(grids, reqs):
        srv.submit(g, n, c["dt"], m1.m1_default_params(tol=tol))
    srv.close()
    for g, (c, n, tol) in zip(grids, reqs):
        alone, _ = run_alone(c, n, tol, 0)
        np.testing.assert_array_equal(alone, np.stack(g.get_state()))
        g.close()


def test_w_cycle_server_equals_alone():
    """A server whose structure is the W-cycle (every request must take it) runs
    the same steps as the grids alone, bit for bit; a V-cycle request is refused.
    The steps use the worded dtau rule: under the printed one the 32^2 request's
    fourth W-cycle step does not converge (the oracle's neither)."""
    reqs = requests()[:3] + requests()[4:5]
    structure = m1.m1_default_params(cycle=m1.CYCLE_W)
    rule = m1.DTAU_SIGNED
    srv = m1.Server(1 << 34, 4, reqs[0][0]["lmax"], m1.FP64, structure=structure)
    grids, tickets = [], []
    for c, n, tol in reqs:
        g = m1.grid_from_case(c)
        grids.append(g)
        tickets.append(srv.submit(g, n, c["dt"], m1.m1_default_params(tol=tol, cycle=m1.CYCLE_W,
                                                                      dtau_rule=rule)))
    g_v = m1.grid_from_case(reqs[0][0])
    with pytest.raises(m1.M1Error):
        srv.submit(g_v, 1, reqs[0][0]["dt"], m1.m1_default_params())
    g_v.close()
    for t in tickets:
        assert srv.wait(t, 300.0) == m1.OK
    srv.close()
    for g, (c, n, tol) in zip(grids, reqs):
        alone = m1.grid_from_case(c)
        p = m1.m1_default_params(tol=tol, cycle=m1.CYCLE_W, dtau_rule=rule)
        for _ in range(n):
            alone.implicit_step(c["dt"], p)
        np.testing.assert_array_equal(np.stack(alone.get_state()), np.stack(g.get_state()))
        alone.close()
        g.close()
