"""The 3D single-level operators (m1_op_level3) against the 3D FP64 oracle:
A(u), b - A(u) and Jacobi sweeps on grids with periodic, reflecting and Neumann
walls, element by element within 1e-12 of each field's scale; the device-array
path gives the host path's result bit for bit."""
import numpy as np
import pytest

from oracle import oracle3d as O3
from tests.test_oracle3d import opacities, random_state3

pytestmark = pytest.mark.gpu

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")

GRIDS = [
    ("periodic-8x6x4", (8, 6, 4), ("periodic",) * 6),
    ("reflect-12x10x6", (12, 10, 6), ("reflect",) * 6),
    ("mixed-31x7x5", (31, 7, 5), ("reflect", "neumann", "periodic", "periodic", "neumann",
                                  "reflect")),
    ("cube-24", (24, 24, 24), ("reflect", "reflect", "periodic", "periodic", "neumann",
                               "neumann")),
]


def _case(dims, bc, seed, dt=0.05):
    nx, ny, nz = dims
    g = O3.Grid3(nx, ny, nz, 1.0 / nx, 0.8 / ny, 0.6 / nz, bc)
    d = m1.make_desc3(nx, ny, nz, 1.0, 0.8, 0.6, bc)
    s = random_state3(nx, ny, nz, seed, fmax=0.95)
    b = random_state3(nx, ny, nz, seed + 1, fmax=0.95)
    sa, ss = opacities((nz, ny, nx), seed + 2)
    return g, d, s, b, sa, ss, dt


def _close(got, ref, tol):
    scale = np.maximum(np.abs(ref).reshape(5, -1).max(axis=1), 1e-300)[:, None, None, None]
    err = np.abs(got - ref) / scale
    assert err.max() <= tol, (err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("name,dims,bc", GRIDS)
def test_apply_and_residual_match_oracle(name, dims, bc):
    g, d, s, b, sa, ss, dt = _case(dims, bc, 30)
    sig = np.stack([sa, ss])
    got, _ = m1.m1_op_level3(d, dt, sig, s, mode=m1.OP3_APPLY)
    _close(got, O3.apply_A(g, dt, sa, ss, s), 1e-12)
    got, _ = m1.m1_op_level3(d, dt, sig, s, rhs=b, mode=m1.OP3_RESIDUAL)
    ref = O3.residual(g, dt, sa, ss, b, s)
    scale = np.maximum(np.abs(b).reshape(5, -1).max(1), 1e-300)[:, None, None, None]
    assert (np.abs(got - ref) / scale).max() <= 1e-12


@pytest.mark.parametrize("name,dims,bc", GRIDS)
@pytest.mark.parametrize("sweeps", [1, 3])
def test_jacobi_sweeps_match_oracle(name, dims, bc, sweeps):
    for dt in (0.05, 5.0):
        g, d, s, b, sa, ss, _ = _case(dims, bc, 40)
        got, _ = m1.m1_op_level3(d, dt, np.stack([sa, ss]), s, rhs=b, mode=m1.OP3_JACOBI,
                                 sweeps=sweeps)
        ref = s
        for _ in range(sweeps):
            ref, it = O3.jacobi_sweep(g, dt, sa, ss, b, ref)
            assert it >= 0
        _close(got, ref, 1e-12 * sweeps)
        assert np.all(got[0] > 0) and np.all(got[4] > 0)
        assert np.all(np.sqrt((got[1:4] ** 2).sum(0)) <= got[0] * (1 + 1e-12))


def test_no_matter_jacobi_is_the_transport_update():
    """Without matter the local solve is the division by the transport diagonal
    (the k_a = 0 branch)."""
    g, d, s, b, sa, ss, dt = _case((8, 8, 8), ("periodic",) * 6, 50)
    z = np.zeros_like(sa)
    got, _ = m1.m1_op_level3(d, dt, np.stack([z, z]), s, rhs=b, mode=m1.OP3_JACOBI, sweeps=2)
    ref = s
    for _ in range(2):
        ref, _ = O3.jacobi_sweep(g, dt, z, z, b, ref)
    _close(got, ref, 1e-12)


def test_device_arrays_give_the_host_result():
    torch = pytest.importorskip("torch")
    g, d, s, b, sa, ss, dt = _case((16, 12, 10), ("reflect",) * 6, 60)
    sig = np.stack([sa, ss])
    host, _ = m1.m1_op_level3(d, dt, sig, s, rhs=b, mode=m1.OP3_JACOBI, sweeps=2)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ts, tb, tg = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (s, b, sig))
        out = torch.empty_like(ts)
        st.synchronize()
        _, ms = m1.m1_op_level3(d, dt, tg, ts, rhs=tb, mode=m1.OP3_JACOBI, sweeps=2, out=out,
                                on_device=True, stream=st.cuda_stream)
    np.testing.assert_array_equal(out.cpu().numpy(), host)
    assert ms > 0
