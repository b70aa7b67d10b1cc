"""Benchmark of the implicit M1 multigrid step on GB300.

Workload (one "step" = one implicit time step v^n -> v^{n+1}, Algorithm 4, of
the 2D plain-FP64 case): 1024 x 1024 cells on [0,1]^2, seeded lognormal
sigma_a, sigma_s spanning 1e-2 .. 1e4, T_g = 1 with a hot square T_g = 4,
E = a_r T^4, F = 0, reflecting walls, dt = 100 h / c, L_max = 8, V-cycles until
||r|| <= 1e-8 ||r_0||.  Every timed step solves the same v^n (the state is reset
on the device before each step, inside the timed region).

metric: fine-level smoother cell-updates per second over the whole step
        (fine cells x fine Jacobi sweeps / step time), summed over ranks.
roofline: the dominant kernel (the fine Jacobi sweep, FP64), timed with CUDA
        events on the grid's stream.
e2e:    the same metric through the C ABI with host buffers: set_state from
        pinned host arrays, the step, get_state back to host, per step.
cpu_baseline / --impl reference: the FP64 CPU oracle on a bounded sample of the
        same workload (a fixed number of V-cycles), on this host's cores.

Multi-GPU: instances are independent, so N ranks run N replicas of the step
(weak scaling, no collective on the data path); value = all ranks' cell-updates
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M1 smoother cell-updates/s"
UNIT = "cell-updates/s"
WORKLOAD = "m1-implicit-step-2d-fp64-1024x1024-lmax8-tol1e-8"
N = 1024


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "_fallback": True}


# Algorithmic work of one fine FP64 Jacobi sweep (2D), per cell-update.
# Bytes: read the iterate u, the right-hand side b and (sigma_a, sigma_s); write u'.
SWEEP_BYTES = 4 * 8 + 4 * 8 + 2 * 8 + 4 * 8
# DRAM bytes per cell of the FP64 sweep kernel measured by ncu on one 2048^2
# launch (dram__bytes_read.sum + dram__bytes_write.sum = 458.3 MB / 4,194,304 cells)
SWEEP64_TRAFFIC_PER_CELL = 458.3e6 / (2048 * 2048)
# FP64 work of one fine Jacobi update (2D), counted in FP64-pipe operations
# (each DFMA, DMUL, DADD, FP64 compare or FP32<->FP64 conversion is one issue
# slot; a reciprocal = hardware estimate + 3 DFMA of third-order refinement = 4;
# a square root = estimate + 5) on the arithmetic as written, with one closure
# per cell (halo re-evaluations are not algorithmic work):
#   closure 29 (reciprocal of E 4, F/E 2, 4 - 3 f^2 3 and its clamp 1, square
#     root 6, E (s - 1)/3 2, 3/(c^2 (2 + s)) 6, q F/E 2, P 3)
#   neighbour operators 26 (x faces 13, y faces 13)
#   opacity products and right-hand sides 6
#   local solve 42 (one reciprocal for both denominators 9, flux 2, quartic
#     setup and conversions 8, one FP64 Halley step after the FP32 Newton
#     iteration 18, E 5)
SWEEP_OPS = 29 + 26 + 6 + 42
# GB300 FP64 pipe: 2 operations per clock per SM (nominal 1.25 TFLOP/s counts a
# DFMA as 2 flops): 152 SMs x 2 x 2.07 GHz.
FP64_PEAK_TOPS = 152 * 2 * 2.07e9 / 1e12
# FP32 fine sweep of the mixed path (correction form), per cell-update: read the
# correction e, the base state w and the source g (3 x 16 B), (sigma_a, sigma_s)
# (8 B); write e' (16 B).
SWEEP32_BYTES = 3 * 16 + 8 + 16
# The plain FP32 sweep (no correction form) would move 4 x 4 (state) + 4 x 4 (rhs)
# + 2 x 4 (opacities) read + 4 x 4 written = 56 B per cell-update.
SWEEP32_PLAN_BYTES = 16 + 16 + 8 + 16
# DRAM bytes per cell of that kernel (cp.async staging, the tuned choice), ncu on
# one 2048^2 launch (307.1 MB)
SWEEP32_TRAFFIC_PER_CELL = 307.1e6 / (2048 * 2048)


class ClockSampler:
    """nvidia-smi clock / throttle samples (every 200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_sample(case, cycles, all_cores=False):
    """The FP64 oracle, as it stands, on `cycles` V-cycles of the workload, on
    one host core or on all of them (the OpenMP build of the same source, bit
    for bit the same results).  Returns (cell-updates/s, seconds, fine sweeps,
    threads)."""
    from oracle import oracle as O
    threads = O.use_all_cores(all_cores and O.have_all_cores())
    try:
        g = O.Grid.from_case(case)
        p = O.SolveParams(lmax=case["lmax"], tol=0.0, max_cycles=cycles)
        t = time.perf_counter()
        _, st, _, _ = O.implicit_step(g, case["dt"], case["sa"], case["ss"], case["state"], p)
        dt = time.perf_counter() - t
    finally:
        O.use_all_cores(False)
    cells = case["desc"]["nx"] * case["desc"]["ny"]
    return cells * st["fine_sweeps"] / dt, dt, st["fine_sweeps"], threads


def oracle_step_worker(path, threads):
    """Child process (spawned): the oracle's full step of the FP64 workload on
    `threads` host threads, saved to `path` (state, cycles, seconds)."""
    os.environ["OMP_NUM_THREADS"] = str(threads)
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2208_14703_gb300 import inputs
    case = inputs.hot_square_2d(N)
    nthr = O.use_all_cores(O.have_all_cores())
    g = O.Grid.from_case(case)
    t = time.perf_counter()
    v, st, _, _ = O.implicit_step(g, case["dt"], case["sa"], case["ss"], case["state"],
                                  O.SolveParams(lmax=case["lmax"], tol=case["tol"]))
    np.savez(path, state=v, cycles=st["cycles"], status=st["status"],
             seconds=time.perf_counter() - t, threads=nthr)


def start_oracle_step():
    """Starts the oracle's full step of the FP64 workload in a spawned process
    on all but two host cores (the GPU's host threads keep two).  Returns
    (process, path)."""
    import multiprocessing as mp
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    threads = max(1, (os.cpu_count() or 1) - 2)
    proc = mp.get_context("spawn").Process(target=oracle_step_worker, args=(path, threads))
    proc.start()
    return proc, path


def finish_oracle_step(proc, path, results, timeout_s=3600.0):
    """Waits for the oracle's step and returns the relative L2 error per field of
    each GPU result in `results` (name -> (4, ny, nx) state) against it."""
    proc.join(timeout_s)
    if proc.is_alive():
        proc.terminate()
        proc.join()
        return {"error": f"the oracle step did not finish within {timeout_s:.0f} s"}
    try:
        d = np.load(path)
        ref = d["state"]
        out = {"oracle_cycles": int(d["cycles"]), "oracle_status": int(d["status"]),
               "oracle_seconds": float(d["seconds"]), "oracle_threads": int(d["threads"])}
    except (OSError, KeyError, ValueError) as e:
        return {"error": f"the oracle step failed: {e}"}
    finally:
        if os.path.exists(path):
            os.unlink(path)
    for name, got in results.items():
        out[name] = field_errors(got, ref)
    return out


def rounded(x, sig=4):
    """A copy of a JSON-able structure with floats kept to `sig` significant
    digits (keeps the printed line short)."""
    if isinstance(x, float):
        return float(f"{x:.{sig}g}")
    if isinstance(x, dict):
        return {k: rounded(v, sig) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [rounded(v, sig) for v in x]
    return x


def sweep_ms(grid, dt, stream, flush, reset, reps=20):
    """Median time of one fine sweep: 0.5 x (m1_jacobi with 2 sweeps - with 0
    sweeps), each launch sequence timed with CUDA events on the grid's stream
    after an L2 flush (state reset before each call, untimed)."""
    import torch

    def timed(nsw):
        out = []
        for _ in range(reps):
            reset()
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            grid.jacobi(dt, nsw)
            b.record(stream)
            out.append((a, b))
        torch.cuda.synchronize()
        return float(np.median([x.elapsed_time(y) for x, y in out]))

    return 0.5 * (timed(2) - timed(0))


def field_errors(got, ref):
    """Relative L2 errors per field (E and the flux against ||E||, T against ||T||)."""
    nE = np.linalg.norm(ref[0])
    return {"E": float(np.linalg.norm(got[0] - ref[0]) / nE),
            "Fx": float(np.linalg.norm(got[1] - ref[1]) / nE),
            "Fy": float(np.linalg.norm(got[2] - ref[2]) / nE),
            "T": float(np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(ref[3]))}


def bench_mixed(m1, case, stream, s0, flush, ref64, steps, hbm_peak):
    """The same workload through the mixed-precision path (FP32 V-cycles in
    correction form inside FP64 defect correction)."""
    import torch
    grid = m1.grid_from_case(case, precision=m1.MIXED, stream=stream.cuda_stream)
    params = m1.m1_default_params(tol=case["tol"])
    dt = case["dt"]
    cells = case["desc"]["nx"] * case["desc"]["ny"]

    def one():
        grid.set_state(*s0, on_device=True)
        return grid.implicit_step(dt, params)

    one()
    torch.cuda.synchronize()
    ev, st = [], []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.append(one())
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    got = np.stack(grid.get_state())
    sms = sweep_ms(grid, dt, stream, flush, lambda: grid.set_state(*s0, on_device=True))
    grid.close()
    gbs = SWEEP32_BYTES * cells / (sms * 1e-3) / 1e9
    units = cells * sum(x.sweeps for x in st)
    bench_mixed.state = got
    return {"workload": WORKLOAD.replace("fp64", "mixed"), "value": units / (sum(ms) * 1e-3),
            "unit": UNIT, "ms_per_step": float(np.mean(ms)),
            "cycles_per_step": [x.cycles for x in st],
            "err_vs_fp64_gpu": field_errors(got, ref64),
            "roofline_fp32_sweep": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                                    "unit": "GB/s", "frac": gbs / hbm_peak, "kernel_ms": sms,
                                    "traffic": SWEEP32_TRAFFIC_PER_CELL * cells,
                                    "bytes_per_cell": SWEEP32_BYTES,
                                    "kernel": "k_sweep<float, correction form>"}}


def bench_fp32_sweep_large(m1, stream, flush, hbm_peak, n=4096):
    """The FP32 correction-form sweep at the mixed-precision configuration's size
    (the 4096^2 beam-in-a-channel grid): one fine sweep timed as in `sweep_ms`
    (state reset on the device before each call), 72 algorithmic bytes per
    cell against the measured HBM peak."""
    import torch
    from paper_2208_14703_gb300 import inputs
    case = inputs.beam_channel_2d(n)
    grid = m1.grid_from_case(case, precision=m1.MIXED, stream=stream.cuda_stream)
    s0 = [torch.from_numpy(np.ascontiguousarray(case["state"][k])).to("cuda") for k in range(4)]
    torch.cuda.synchronize()
    ms = sweep_ms(grid, case["dt"], stream, flush, lambda: grid.set_state(*s0, on_device=True))
    grid.close()
    cells = n * n
    gbs = SWEEP32_BYTES * cells / (ms * 1e-3) / 1e9
    gbs56 = SWEEP32_PLAN_BYTES * cells / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
            "frac": gbs / hbm_peak, "kernel_ms": ms, "cells": cells, "bytes_per_cell": SWEEP32_BYTES,
            "frac_at_56_bytes": gbs56 / hbm_peak,
            "note_56_bytes": "the plain FP32 sweep's 56 B/cell (state, rhs, opacities read, "
                             "state written); the correction form also reads the base state w",
            "traffic": SWEEP32_TRAFFIC_PER_CELL * cells,
            "traffic_source": "ncu DRAM bytes of the 2048^2 cp.async launch (307.1 MB), scaled "
                              "by cells (both working sets exceed L2)",
            "strip_rows": m1.strip_rows(1, n, n),
            "kernel": "k_sweep FP32 correction form at the 4096^2 mixed configuration"}


def bench_mixed_beam(m1, stream, flush, n=4096):
    """The mixed-precision configuration: an f = 1 beam entering a thin channel
    at the west wall of a 4096^2 lognormal medium (L_max = 10, tol 1e-8).  One
    step through each path, timed after a two-cycle warm-up that builds the
    captured cycle, and the per-field difference of the two results (the
    element-wise comparison with the oracle runs on the 1024^2 window of this
    grid that holds the beam, tests/test_gpu_full_size.py)."""
    import torch
    from paper_2208_14703_gb300 import inputs
    case = inputs.beam_channel_2d(n)
    s0 = [torch.from_numpy(np.ascontiguousarray(case["state"][k])).to("cuda") for k in range(4)]
    cells = n * n
    out = {"workload": f"m1-implicit-step-2d-beam-channel-{n}x{n}-lmax{case['lmax']}-tol1e-8",
           "l2": "flushed before each timed step"}
    states = {}
    for name, prec in (("mixed", m1.MIXED), ("fp64", m1.FP64)):
        g = m1.grid_from_case(case, precision=prec, stream=stream.cuda_stream)
        g.set_state(*s0, on_device=True)
        g.implicit_step(case["dt"], m1.m1_default_params(tol=case["tol"], max_cycles=2),
                        allow_not_converged=True)
        g.set_state(*s0, on_device=True)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = g.implicit_step(case["dt"], m1.m1_default_params(tol=case["tol"]))
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        states[name] = np.stack(g.get_state())
        g.close()
        out[name] = {"ms_per_step": ms, "cycles": st.cycles,
                     "cell_updates_per_s": cells * st.sweeps / (ms * 1e-3)}
    out["fp64_over_mixed_time"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["mixed_err_vs_fp64_gpu"] = field_errors(states["mixed"], states["fp64"])
    return out


# FP64 work of one 3D Jacobi update, counted as SWEEP_OPS is: the closure pass
# (reciprocal 4, F/E 3, 4 - 3 f^2 and its clamp 5, square root 6, E (s - 1)/3 2,
# 3/(c^2 (2 + s)) 6, q F/E 3, the six tensor entries 6) and the operator pass
# (six face neighbours of 9 each: the energy term c E + s F_d scaled and summed
# in 3, each flux component's F_a + s c P_da scaled and summed in 2; opacity
# products 3, right-hand sides 4, local solve 43: one reciprocal for both
# denominators 9, flux 3, quartic setup and conversions 8, one Halley step 18,
# E 5).  ncu counts about 35 + 116 issued FP64 operations per cell for the two
# passes at 128^3.
SWEEP3D_OPS = 35 + 6 * 9 + 3 + 4 + 43


def bench_sweep3d(m1, stream, n=256, sweeps=2):
    """The 3D single-level Jacobi sweep (closure pass + operator pass) on an n^3
    grid with reflecting walls, inputs generated on the device (admissible random
    states, lognormal opacities, seeded): device time of `sweeps` sweeps from
    the operator's own events."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    shape = (n, n, n)
    u = lambda: torch.rand(shape, generator=gen, device="cuda", dtype=torch.float64)

    def state():
        E = 10.0 ** (2.0 * u() - 1.0)
        d = torch.randn((3,) + shape, generator=gen, device="cuda", dtype=torch.float64)
        d = d / d.norm(dim=0)
        F = 0.9 * u() * E * d
        T = 10.0 ** (0.6 * u() - 0.3)
        return torch.cat([E[None], F, T[None]]).contiguous()

    s, b = state(), state()
    sig = (10.0 ** (4.0 * torch.rand((2,) + shape, generator=gen, device="cuda",
                                     dtype=torch.float64) - 2.0)).contiguous()
    out = torch.empty_like(s)
    d = m1.make_desc3(n, n, n, 1.0, 1.0, 1.0, ("reflect",) * 6)
    torch.cuda.synchronize()
    m1.m1_op_level3(d, 100.0 / n, sig, s, rhs=b, mode=m1.OP3_JACOBI, sweeps=1, out=out,
                    on_device=True, stream=stream.cuda_stream)
    best = None
    for _ in range(3):
        _, ms = m1.m1_op_level3(d, 100.0 / n, sig, s, rhs=b, mode=m1.OP3_JACOBI, sweeps=sweeps,
                                out=out, on_device=True, stream=stream.cuda_stream)
        best = ms if best is None else min(best, ms)
    per = best / sweeps
    cells = n ** 3
    tops = SWEEP3D_OPS * cells / (per * 1e-3) / 1e12
    return {"workload": f"3d-jacobi-sweep-{n}^3-reflect-fp64", "cells": cells,
            "ms_per_sweep": per, "cell_updates_per_s": cells / (per * 1e-3),
            "roofline": {"bound": "alu", "achieved": tops, "peak": FP64_PEAK_TOPS, "unit": "Top/s",
                         "frac": tops / FP64_PEAK_TOPS, "ops_per_cell": SWEEP3D_OPS}}


def bench_step3d(m1, stream, n=128, lmax=5, fp64_peak=None):
    """One implicit step in 3D (Algorithm 4 on a 3D hierarchy): the n^3 hot cube
    (lognormal opacities, reflecting walls, CFL 100, L_max = 5, tol 1e-8),
    one untimed then one timed step (the state reset in between), and the fine
    Jacobi sweep of that grid (closure pass + operator pass) against the FP64
    pipe's ceiling (SWEEP3D_OPS per cell-update)."""
    import torch
    from paper_2208_14703_gb300 import inputs
    case = inputs.hot_cube_3d(n, lmax=lmax)
    g = m1.grid3_from_case(case, stream=stream.cuda_stream)
    params = m1.m1_default_params(tol=case["tol"])
    sig = np.stack([case["sa"], case["ss"]])
    g.implicit_step(case["dt"], params)
    g.set_state(case["state"], sig)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    st = g.implicit_step(case["dt"], params)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    out = g.get_state()
    g.close()
    cells = n ** 3
    sweep = bench_sweep3d(m1, stream, n=n)
    peak = fp64_peak or FP64_PEAK_TOPS
    tops = SWEEP3D_OPS * cells / (sweep["ms_per_sweep"] * 1e-3) / 1e12
    return {"workload": f"m1-implicit-step-3d-fp64-{n}^3-lmax{lmax}-tol1e-8", "cells": cells,
            "cycles": st.cycles, "ms_per_step": ms, "ms_per_cycle": ms / max(st.cycles, 1),
            "cell_updates_per_s": cells * st.sweeps / (ms * 1e-3),
            "launches_per_cycle": (st.launches - 5) / max(st.cycles, 1),
            "admissible": bool(np.all(out[0] > 0) and np.all(out[4] > 0)),
            "fine_sweep": {"ms": sweep["ms_per_sweep"], "bound": "alu", "achieved": tops,
                           "peak": peak, "unit": "Top/s", "frac": tops / peak,
                           "ops_per_cell": SWEEP3D_OPS}}


def bench_cycle_shapes(m1, case, stream, s0, flush):
    """Cycles to tolerance and step time of the same workload with V-, W- and
    F-cycles (Section 6.3 names W and F as the alternatives), FP64 and mixed:
    one untimed step, then one timed step per shape and precision."""
    import torch
    out = {}
    for pname, prec in (("fp64", m1.FP64), ("mixed", m1.MIXED)):
        grid = m1.grid_from_case(case, precision=prec, stream=stream.cuda_stream)
        for sname, shape in (("V", m1.CYCLE_V), ("W", m1.CYCLE_W), ("F", m1.CYCLE_F)):
            params = m1.m1_default_params(tol=case["tol"], cycle=shape)
            grid.set_state(*s0, on_device=True)
            grid.implicit_step(case["dt"], params)
            grid.set_state(*s0, on_device=True)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = grid.implicit_step(case["dt"], params)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            out[f"{pname}_{sname}"] = {"cycles": st.cycles, "ms_per_step": ms,
                                       "ms_per_cycle": ms / max(st.cycles, 1),
                                       "launches_per_cycle": (st.launches - 4) / max(st.cycles, 1)}
        grid.close()
    return out


def bench_paper_beam(m1, stream, sizes=(256, 512), levels=(1, 2, 3, 4)):
    """The paper's beam (Section 4.1, run in Section 5.1) in nondimensional form
    at 2^k stand-ins for its 257^2 and 513^2 grids, CFL 2000, tolerance 1e-2:
    V-cycles to tolerance, step time and time per cycle (normalised to L_max = 1,
    as the paper's per-cycle cost table) for L_max = 1..4, and the largest E on
    the horizontal cut at mid height against the beam's inflow E (the paper
    compares that cut's maximum across solvers), and the W- and F-cycles at the
    deepest hierarchy.  FP64, one untimed step then one timed step per
    configuration."""
    import torch
    from paper_2208_14703_gb300 import inputs
    out = {}
    for n in sizes:
        rows = {}
        for lmax in levels:
            case = inputs.paper_beam_2d(n, lmax=lmax)
            grid = m1.grid_from_case(case, stream=stream.cuda_stream)
            params = m1.m1_default_params(tol=case["tol"])
            state = [np.ascontiguousarray(case["state"][k]) for k in range(4)]
            grid.implicit_step(case["dt"], params)
            grid.set_state(*state)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = grid.implicit_step(case["dt"], params)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            E = grid.get_state()[0]
            grid.close()
            e_beam = case["inflow"][0, 0].max()
            rows[f"L{lmax}"] = {"cycles": st.cycles, "ms_per_step": ms,
                                "ms_per_cycle": ms / max(st.cycles, 1),
                                "cut_max_over_beam_E": float(E[n // 2].max() / e_beam)}
        base = rows[f"L{levels[0]}"]["ms_per_cycle"]
        for r in rows.values():
            r["cost_per_cycle_normalised"] = r["ms_per_cycle"] / base
        # the W- and F-cycle at the deepest hierarchy (the coarse correction is
        # the bottleneck here, unlike the diffusive hot square)
        case = inputs.paper_beam_2d(n, lmax=levels[-1])
        grid = m1.grid_from_case(case, stream=stream.cuda_stream)
        state = [np.ascontiguousarray(case["state"][k]) for k in range(4)]
        for name, shape in (("W", m1.CYCLE_W), ("F", m1.CYCLE_F)):
            params = m1.m1_default_params(tol=case["tol"], cycle=shape)
            grid.set_state(*state)
            grid.implicit_step(case["dt"], params)
            grid.set_state(*state)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = grid.implicit_step(case["dt"], params)
            b.record(stream)
            torch.cuda.synchronize()
            rows[f"L{levels[-1]}_{name}"] = {"cycles": st.cycles, "ms_per_step": a.elapsed_time(b)}
        grid.close()
        out[f"{n}x{n}"] = rows
    return out


def bench_paper_riemann(m1, stream, n=256, steps=10, cfl=150.0, levels=(1, 2, 4)):
    """The periodic 2D Riemann problem of Section 5.2 in nondimensional form: no
    energy enters or leaves the box, so the relative change of the total
    radiative energy after each step measures the solver's conservation at the
    paper's residual 5e-3 (the paper: below 1e-12 with Jacobi, about 1e-8 with
    the multigrid).  FP64; the largest relative error over the steps, the mean
    cycles per step and the time per step for each L_max."""
    import torch
    from paper_2208_14703_gb300 import inputs
    out = {}
    for lmax in levels:
        case = inputs.riemann_2d(n, cfl=cfl, lmax=lmax, tol=5e-3)
        grid = m1.grid_from_case(case, stream=stream.cuda_stream)
        params = m1.m1_default_params(tol=case["tol"])
        e0 = float(case["state"][0].sum())
        worst, cycles = 0.0, []
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            st = grid.implicit_step(case["dt"], params)
            cycles.append(st.cycles)
            worst = max(worst, abs(float(grid.get_state()[0].sum()) - e0) / e0)
        b.record(stream)
        torch.cuda.synchronize()
        grid.close()
        out[f"L{lmax}"] = {"max_rel_energy_error": worst, "mean_cycles": float(np.mean(cycles)),
                           "ms_per_step": a.elapsed_time(b) / steps}
    return {"workload": f"riemann-2d-periodic-{n}x{n}-cfl{cfl:g}-tol5e-3-{steps}-steps", **out}


def bench_batched(m1, count, stream):
    """Independent 2D instances of uneven sizes stepped together, mixed and FP64."""
    import torch
    from paper_2208_14703_gb300 import inputs
    cases = inputs.batched_instances(count)
    cells = sum(c["desc"]["nx"] * c["desc"]["ny"] for c in cases)
    out = {"workload": f"m1-batched-2d-{count}-instances-64..1024-lmax5-tol1e-8",
           "instances": count, "cells": cells}
    for name, prec in (("mixed", m1.MIXED), ("fp64", m1.FP64)):
        b = m1.batch_from_cases(cases, precision=prec, stream=stream.cuda_stream)
        params = m1.m1_default_params(tol=1e-8)
        dts = [c["dt"] for c in cases]
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        st = b.implicit_step(dts, params, allow_not_converged=True)
        e.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(e)
        b.close()
        units = sum(c["desc"]["nx"] * c["desc"]["ny"] * x.sweeps for c, x in zip(cases, st))
        out[name] = {"ms_per_step": ms, "solves_per_s": count / (ms * 1e-3),
                     "cell_updates_per_s": units / (ms * 1e-3),
                     "not_converged": sum(1 for x in st if x.status != 0),
                     "max_cycles": max(x.cycles for x in st)}
    out["mixed_over_fp64_solves"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


def bench_serving(m1, reqs, stream, budget, paths=("mixed", "fp64"), small_cells=None):
    """A Poisson arrival stream of simulations served with continuous batching,
    mixed precision against the plain FP64 path (the same stream through an FP64
    server); `paths` selects which of the two run, `small_cells` the size up to
    which requests take the server's small lane (0: one lane)."""
    if small_cells is None:
        small_cells = m1.SMALL_CELLS
    out = {"requests": len(reqs), "steps": sum(r["nsteps"] for r in reqs),
           "sizes": sorted({(r["case"]["desc"]["dim"], r["case"]["desc"]["nx"]) for r in reqs}),
           "arrival_span_s": reqs[-1]["arrival_s"], "budget_bytes": budget,
           "dtau_rule": "signed (decrease of the residual norm)", "small_lane_cells": small_cells}
    for name, prec in (("mixed", m1.MIXED), ("fp64", m1.FP64)):
        if name not in paths:
            continue
        grids = [m1.grid_from_case(r["case"], precision=prec) for r in reqs]
        srv = m1.Server(budget, 64, reqs[0]["case"]["lmax"], prec, stream=stream.cuda_stream,
                        small_cells=small_cells)
        t0 = time.perf_counter()
        tickets = []
        for r, g in zip(reqs, grids):
            delay = r["arrival_s"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(g, r["nsteps"], r["case"]["dt"],
                                      m1.m1_default_params(tol=r["case"]["tol"],
                                                           dtau_rule=m1.DTAU_SIGNED)))
        status = [srv.wait(t, 3600.0) for t in tickets]
        wall = time.perf_counter() - t0
        s = srv.stats()
        srv.close()
        for g in grids:
            g.close()
        out[name] = {"solves_per_s": s.steps_done / wall, "busy_solves_per_s": s.solves_per_s,
                     "p50_ms": s.p50_ms, "p99_ms": s.p99_ms, "mean_ms": s.mean_ms,
                     "wall_s": wall, "cycles": s.cycles, "bytes_peak": s.bytes_peak,
                     "failed": sum(1 for x in status if x != m1.OK)}
    if "mixed" in out and "fp64" in out:
        out["mixed_over_fp64_solves"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


def reduce_over_ranks(ms, units, device, world):
    """Whole-job throughput of replicas: the slowest rank's time and the units
    of all ranks (MAX and SUM all-reduces when world > 1).  Returns
    (ms_max, units_sum, units_sum / seconds)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.item(), u.item(), u.item() / (t.item() * 1e-3)


def run_reference(args, case):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    cyc = 2
    threads = 1
    for _ in range(args.warmup):
        cpu_sample(case, cyc, all_cores=True)
    vals, secs = [], []
    for _ in range(args.steps):
        v, s, _, threads = cpu_sample(case, cyc, all_cores=True)
        vals.append(v)
        secs.append(s)
    value = float(np.mean(vals))
    sample = (f"{cyc} V-cycles of the workload per step (fine sweeps x 1024^2 cells / time), "
              f"the oracle's OpenMP build on {threads} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mixed, batched and serving measurements")
    ap.add_argument("--batch-count", type=int, default=512,
                    help="instances of the batched configuration (default: all 512)")
    ap.add_argument("--serve-full", action="store_true",
                    help="serve 64 requests of the serving recipe instead of the 10-request sample")
    ap.add_argument("--no-oracle-errors", action="store_true",
                    help="skip the oracle's full step (per-field errors of the GPU results)")
    args = ap.parse_args()

    from paper_2208_14703_gb300 import inputs
    case = inputs.hot_square_2d(N)
    if args.impl == "reference":
        run_reference(args, case)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    from paper_2208_14703_gb300 import build
    build.build()
    from paper_2208_14703_gb300 import m1

    # a dedicated (non-default) stream shared by the grid and the CUDA events
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    # strip heights of the sweep kernels, tuned on this GPU (untimed)
    tuning = m1.autotune(stream.cuda_stream)
    grid = m1.grid_from_case(case, stream=stream.cuda_stream)
    dev = torch.device("cuda", local)
    s0 = [torch.from_numpy(np.ascontiguousarray(case["state"][k])).to(dev) for k in range(4)]
    params = m1.m1_default_params(tol=case["tol"])
    dt = case["dt"]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    cells = N * N

    def one_step():
        grid.set_state(*s0, on_device=True)
        return grid.implicit_step(dt, params)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    stats = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                       # L2 flushed between timed steps (not timed)
        ev[k][0].record(stream)
        stats.append(one_step())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    ms_total = sum(ms_steps)

    # dominant kernel: the fine FP64 Jacobi sweep, timed with CUDA events on the
    # grid's stream (each m1_jacobi call = rhs build + the sweeps; an even count
    # ends in the state buffer, so 0.5 x (2 sweeps - 0 sweeps) is one sweep)
    ref64 = np.stack(grid.get_state())
    sweep64_ms = sweep_ms(grid, dt, stream, flush, lambda: grid.set_state(*s0, on_device=True))
    sampler_out = sampler.stop()

    sweeps = [s.sweeps for s in stats]
    cycles = [s.cycles for s in stats]
    units = cells * sum(sweeps)
    ms_max, _, value = reduce_over_ranks(ms_total, units, dev, world)

    # end to end through the C ABI with host buffers, over as many steps as the
    # timed region: set_state from pinned host arrays, the step, get_state back
    pin = [torch.from_numpy(np.ascontiguousarray(case["state"][k])).pin_memory() for k in range(4)]
    outp = [torch.empty((N, N), dtype=torch.float64).pin_memory() for _ in range(4)]
    e2e_steps = max(1, args.steps)
    torch.cuda.synchronize()
    te = time.perf_counter()
    e2e_units = 0
    for _ in range(e2e_steps):
        grid.set_state(*[p.numpy() for p in pin])
        st = grid.implicit_step(dt, params)
        grid.get_state([o.numpy() for o in outp])
        e2e_units += cells * st.sweeps
    te = time.perf_counter() - te
    _, _, e2e_val = reduce_over_ranks(1e3 * te, e2e_units, dev, world)

    # the FP64 pipe's ceiling on this GPU (the fine sweep's roof), measured
    pk = peaks()
    try:
        fp64_peak = m1.probe_fma_peak(m1.FP64, stream.cuda_stream, reps=5) / 1e12
        peak_source = ("measured: m1_probe_fma_peak, DFMA instructions per second over lanes "
                       "(independent chains, median of 5 launches), this GPU, this run")
    except m1.M1Error as e:
        fp64_peak = FP64_PEAK_TOPS
        peak_source = f"derived 152 SMs x 2 FP64 ops/clk x 2.07 GHz (the probe failed: {e})"
    tops = SWEEP_OPS * cells / (sweep64_ms * 1e-3) / 1e12
    gbs = SWEEP_BYTES * cells / (sweep64_ms * 1e-3) / 1e9
    roof = {"bound": "alu", "achieved": tops, "peak": fp64_peak, "unit": "Top/s",
            "frac": tops / fp64_peak, "traffic": SWEEP64_TRAFFIC_PER_CELL * cells,
            "kernel": "k_sweep<double> (fine Jacobi sweep, FP64)", "kernel_ms": sweep64_ms,
            "peak_source": peak_source, "peak_derived": FP64_PEAK_TOPS,
            "frac_of_derived": tops / FP64_PEAK_TOPS,
            "ops_per_cell": SWEEP_OPS, "op": "FP64-pipe operation (DFMA, DMUL, DADD, FP64 compare or conversion)",
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                              "2048^2 launch (458.3 MB), scaled to 1024^2 by cells",
            "hbm": {"achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / pk["hbm_gbs"], "bytes_per_cell": SWEEP_BYTES}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        v, secs, fs, thr = cpu_sample(case, 4, all_cores=True)
        v1, secs1, fs1, _ = cpu_sample(case, 4, all_cores=False)
        cpu = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"4 V-cycles of the same 1024^2 workload ({fs} fine sweeps, {secs:.1f} s), "
                         f"the oracle's OpenMP build on {thr} host threads (of {os.cpu_count()})",
               "one_core": {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"the same 4 V-cycles, one-core build ({secs1:.1f} s)"}}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        from paper_2208_14703_gb300 import inputs
        ora = None if args.no_oracle_errors else start_oracle_step()
        extras["cycle_shapes"] = bench_cycle_shapes(m1, case, stream, s0, flush)
        extras["sweep3d"] = bench_sweep3d(m1, stream)
        extras["step3d"] = bench_step3d(m1, stream, fp64_peak=fp64_peak)
        extras["paper_beam"] = bench_paper_beam(m1, stream)
        extras["paper_riemann"] = bench_paper_riemann(m1, stream)
        mixed = bench_mixed(m1, case, stream, s0, flush, ref64, args.steps, pk["hbm_gbs"])
        mixed["roofline_fp32_sweep_4096"] = bench_fp32_sweep_large(m1, stream, flush,
                                                                   pk["hbm_gbs"])
        extras["mixed_beam"] = bench_mixed_beam(m1, stream, flush)
        extras["batched"] = bench_batched(m1, args.batch_count, stream)
        if args.serve_full:
            reqs = inputs.serving_stream(64)
            sample = "64 requests of the serving recipe (seed 11)"
        else:
            reqs = inputs.serving_stream(10, seed=133)
            sample = ("10 requests of the serving recipe (seed 133: 1D 256..65536, 2D "
                      "128..2048, 10-100 steps each, 432 steps)")
        extras["serving"] = bench_serving(m1, reqs, stream, 32 << 30)
        extras["serving"]["workload"] = (
            f"poisson-stream: {sample}, against the recipe's 2000 requests at 4 offered loads")
        if ora is not None:
            mixed["err_vs_oracle"] = finish_oracle_step(*ora, {"fp64": ref64,
                                                               "mixed": bench_mixed.state})
        extras["mixed"] = mixed
        extras = {k: rounded(v) for k, v in extras.items()}
        # the large blocks last: a reader of the line's tail sees them
        for k in ("mixed_beam", "mixed", "batched", "serving"):
            extras[k] = extras.pop(k)

    launches = sum(s.launches for s in stats) + 2 * args.steps
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": cells, "lmax": case["lmax"],
                       "tol": case["tol"], "cfl": 100, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MB write)",
                       "reset": "v^n restored on the device before every step (timed)",
                       "strip_rows": {f"{'fp64' if t['kind'] == 0 else 'fp32'}-{t['n']}": t["strip_rows"]
                                      for t in tuning},
                       "fp32_cp_async_staging": sorted(t["n"] for t in tuning
                                                       if t["kind"] == 1 and t["staging"] == 1)},
            "cycles_per_step": cycles, "fine_sweeps_per_step": sweeps,
            "steps_cells_per_s": cells * args.steps / (ms_max * 1e-3) * world,
            "wall_s": wall,
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 4 * 8 * cells,
                    "d2h_bytes_per_step": 4 * 8 * cells, "steps": e2e_steps},
            "gpu_launches": launches, "clocks": sampler_out, **extras,
        }))
    grid.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
