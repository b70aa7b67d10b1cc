"""m1_residual_norm_noalloc: the residual norm for callers that cannot allocate
device memory (a framework whose own pool owns all of it, or a latency-critical
loop where cudaMalloc's device-wide synchronisation is not allowed).

Called through the C ABI on caller-owned device buffers, its result must match
the allocating entry point (m1_op_level, residual mode) and the oracle's norm of
the oracle's residual within the 1e-12 relative tolerance of the other kernel
checks, on calls in a row: a larger 2D grid first, then a smaller one, then a
1D grid with an inflow wall (256-cell tiles on one axis), so a stale partial sum
left in the shared scratch by an earlier call would show in a later one."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14703_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
m1 = pytest.importorskip("paper_2208_14703_gb300.m1")


def _device(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _noalloc_norm(desc, dt, state, rhs, sig, inflow, stream):
    n = desc.nx * desc.ny
    st_d = _device(np.reshape(state, (4, n)))
    b_d = _device(np.reshape(rhs, (4, n)))
    sg_d = _device(np.reshape(sig, (2, n)))
    in_d = _device(inflow) if inflow is not None else None
    out_d = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    status = m1._lib.m1_residual_norm_noalloc(
        ctypes.byref(desc), dt, st_d.data_ptr(), b_d.data_ptr(), sg_d.data_ptr(),
        in_d.data_ptr() if in_d is not None else None, out_d.data_ptr(), stream.cuda_stream)
    assert status == m1.OK, m1._lib.m1_last_error()
    stream.synchronize()
    return out_d.item()


def test_noalloc_norm_matches_allocating_entry_point_twice():
    stream = torch.cuda.Stream()
    cases = [inputs.random_admissible_2d(200, 120, seed=31, fmax=0.99, cfl=80,
                                         bc=("reflect", "inflow", "periodic", "periodic")),
             inputs.random_admissible_2d(48, 24, seed=32, fmax=0.9, cfl=20,
                                         bc=("neumann",) * 4),
             inputs.random_admissible_2d(700, 1, seed=33, fmax=0.99, cfl=40,
                                         bc=("inflow", "reflect", "periodic", "periodic"), dim=1)]
    for case in cases:
        g = O.Grid.from_case(case)
        desc = m1.desc_from_case(case, lmax=1)
        sig = np.stack([case["sa"], case["ss"]])
        b = O.rhs_of(g, case["state"]) * 1.01
        _, ref = m1.m1_op_level(desc, case["dt"], sig, case["state"], b, mode=m1.OP_RESIDUAL,
                                inflow=case["inflow"])
        ora = O.norm(g, O.residual(g, case["dt"], case["sa"], case["ss"], b, case["state"]))
        got = _noalloc_norm(desc, case["dt"], case["state"], b, sig, case["inflow"], stream)
        assert got == pytest.approx(ref, rel=1e-12)
        assert got == pytest.approx(ora, rel=1e-12)


def test_noalloc_rejects_grids_beyond_the_fixed_scratch():
    # 8192 x 4096 cells need 131072 tile partials; the scratch holds 65536.  The
    # check happens before any device access, so tiny buffers suffice.
    desc = m1.make_desc(2, 8192, 4096, 2.0, 1.0, ["reflect"] * 4, lmax=1)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    status = m1._lib.m1_residual_norm_noalloc(ctypes.byref(desc), 0.01, p, p, p, None, p, None)
    assert status == m1.ERR_INVALID_ARG
    assert b"scratch" in m1._lib.m1_last_error()
    # sizes whose cell or tile counts overflow 32-bit arithmetic are rejected the
    # same way (the counts are formed in 64 bits before the check)
    for dim, nx, ny in ((2, 65536, 65536), (1, 2**31 - 1, 1), (2, 2**31 - 1, 2**31 - 1)):
        desc = m1.make_desc(dim, nx, ny, 1.0, 1.0, ["reflect"] * 4, lmax=1)
        status = m1._lib.m1_residual_norm_noalloc(ctypes.byref(desc), 0.01, p, p, p, None, p, None)
        assert status == m1.ERR_INVALID_ARG
