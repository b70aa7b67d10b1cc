"""Small fixed workloads for kernel profiles (run under ncu by the caller).

    python -m paper_2208_14703_gb300.profile_kernels --case sweep32 --n 2048

Cases (2D hot-square workload: lognormal opacities, hot square, reflecting walls,
CFL 100, at n x n cells):
  sweep64   FP64 grid: the right-hand side kernel, then 2 fine Jacobi sweeps
            (k_sweep<double>)
  sweep32   MIXED grid: rhs, FP64 defect, 2 FP32 correction-form sweeps
            (k_sweep<float> in correction form), FP64 accumulation
  step64    one implicit step on an FP64 grid with L_max = --lmax
  stepmixed one implicit step on a MIXED grid with L_max = --lmax
            (step64 and stepmixed: --workload beam takes the beam-in-a-channel
            grid of the mixed-precision configuration instead of the hot square)
  sweep3d   3D: one Jacobi sweep (closure pass + operator pass) of an n^3 grid with
            reflecting walls, admissible random states and lognormal opacities
            generated on the device
  step3d    3D: one implicit step of the n^3 hot cube (lognormal opacities,
            reflecting walls, CFL 100) with L_max = --lmax
  steptime  not a profile: the full step (tol 1e-8) on an FP64 and on a MIXED
            grid with L_max = --lmax, each timed three times with CUDA events
            after an L2 flush; prints the faster of the last two and the cycle
            counts as one JSON line (the before / after timings of kernel
            changes quoted in the design notes come from this case at
            --n 1024 --lmax 8)
The state and opacities are set once; each case runs its launches once after one
untimed warm-up of the same launches, so `ncu -s` skips the warm-up.

--tune-file PATH: the strip shapes of the sweep kernels.  If PATH exists its
table is installed (no tuning launches, so a profiled run sees only the case's
kernels); otherwise the autotuner runs and its table is written to PATH (run the
command once without ncu first).  tune_gb300.json beside this file is the table
the autotuner wrote on a GB300; the committed profiles use it.
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", required=True,
                    choices=["sweep64", "sweep32", "step64", "stepmixed", "sweep3d", "step3d",
                             "steptime"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--lmax", type=int, default=6)
    ap.add_argument("--cycles", type=int, default=50, help="max_cycles of the step cases")
    ap.add_argument("--tune-file", default=None)
    ap.add_argument("--workload", choices=["hot", "beam"], default="hot",
                    help="2D step cases: the hot square, or the beam entering a channel "
                         "(the mixed-precision configuration's generator)")
    args = ap.parse_args()

    from paper_2208_14703_gb300 import inputs, m1
    if args.case == "sweep3d":
        sweep3d(m1, args.n)
        return
    if args.case == "step3d":
        step3d(m1, inputs, args.n, args.lmax, args.cycles)
        return
    if args.tune_file:
        import json
        import os
        if os.path.exists(args.tune_file):
            with open(args.tune_file) as fh:
                m1.set_tuning(json.load(fh))
        else:
            with open(args.tune_file, "w") as fh:
                json.dump(m1.autotune(), fh)
    if args.case == "steptime":
        steptime(m1, inputs, args.n, args.lmax)
        return
    mixed = args.case in ("sweep32", "stepmixed")
    lmax = 1 if args.case.startswith("sweep") else args.lmax
    if args.workload == "beam" and not args.case.startswith("sweep"):
        case = inputs.beam_channel_2d(args.n, lmax=lmax)
    else:
        case = inputs.hot_square_2d(args.n, lmax=lmax)
    g = m1.grid_from_case(case, precision=m1.MIXED if mixed else m1.FP64)
    state = [np.ascontiguousarray(case["state"][k]) for k in range(4)]
    dt = case["dt"]
    params = m1.m1_default_params(tol=case["tol"], max_cycles=args.cycles)
    for _ in range(2):                       # warm-up, then the profiled pass
        g.set_state(*state)
        if args.case.startswith("sweep"):
            g.jacobi(dt, 2)
            g.get_state()                    # synchronises the grid's stream
        else:
            st = g.implicit_step(dt, params, allow_not_converged=True)
    if not args.case.startswith("sweep"):
        print(f"cycles {st.cycles} sweeps {st.sweeps} ms {st.ms:.3f}")
    g.close()


def step3d(m1, inputs, n, lmax, cycles):
    case = inputs.hot_cube_3d(n, lmax=lmax)
    g = m1.grid3_from_case(case)
    sig = np.stack([case["sa"], case["ss"]])
    params = m1.m1_default_params(tol=case["tol"], max_cycles=cycles)
    for _ in range(2):                       # warm-up, then the profiled pass
        g.set_state(case["state"], sig)
        st = g.implicit_step(case["dt"], params, allow_not_converged=True)
    print(f"cycles {st.cycles} sweeps {st.sweeps} ms {st.ms:.3f}")
    g.close()


def sweep3d(m1, n):
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    shape = (n, n, n)

    def u():
        return torch.rand(shape, generator=gen, device="cuda", dtype=torch.float64)

    def state():
        E = 10.0 ** (2.0 * u() - 1.0)
        d = torch.randn((3,) + shape, generator=gen, device="cuda", dtype=torch.float64)
        F = 0.9 * u() * E * d / d.norm(dim=0)
        return torch.cat([E[None], F, (10.0 ** (0.6 * u() - 0.3))[None]]).contiguous()

    s, b = state(), state()
    sig = (10.0 ** (4.0 * torch.rand((2,) + shape, generator=gen, device="cuda",
                                     dtype=torch.float64) - 2.0)).contiguous()
    out = torch.empty_like(s)
    d = m1.make_desc3(n, n, n, 1.0, 1.0, 1.0, ("reflect",) * 6)
    torch.cuda.synchronize()
    for _ in range(2):                       # warm-up, then the profiled pass
        _, ms = m1.m1_op_level3(d, 100.0 / n, sig, s, rhs=b, mode=m1.OP3_JACOBI, sweeps=1,
                                out=out, on_device=True)
    print(f"sweep3d n {n} ms {ms:.3f}")



def steptime(m1, inputs, n, lmax):
    """Full-step timings of both precisions (see the module docstring)."""
    import json
    import torch
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    case = inputs.hot_square_2d(n, lmax=lmax)
    s0 = [torch.from_numpy(np.ascontiguousarray(case["state"][k])).cuda() for k in range(4)]
    out = {"n": n, "lmax": lmax}
    for name, prec in (("fp64", m1.FP64), ("mixed", m1.MIXED)):
        g = m1.grid_from_case(case, precision=prec, stream=stream.cuda_stream)
        params = m1.m1_default_params(tol=case["tol"])
        ms = []
        for _ in range(3):
            g.set_state(*s0, on_device=True)
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = g.implicit_step(case["dt"], params)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        g.close()
        out[name] = {"ms": round(min(ms[1:]), 2), "cycles": st.cycles}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
