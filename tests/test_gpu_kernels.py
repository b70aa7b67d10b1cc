"""Kernel-by-kernel parity of the CUDA path (through the C ABI) with the FP64
oracle, element by element, on seeded inputs spanning several tiles with
ragged edges, every boundary kind, 1D and 2D.

Tolerances: the FP64 kernels evaluate the same formulas in a different but
algebraically equal form (closure without the unit vector, FP32-seeded Newton
with FP64 polish), so they differ from the oracle by rounding only: 1e-12
relative to the field scale.  FP32 kernels: 2e-5 relative (a few FP32 ulps
amplified by the transport diagonal)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14703_gb300 import inputs

pytestmark = pytest.mark.gpu

m1 = pytest.importorskip("paper_2208_14703_gb300.m1")

CASES = [
    ("2d-periodic-ragged", dict(nx=80, ny=48, dim=2, bc=("periodic",) * 4, fmax=0.99, cfl=30)),
    ("2d-reflect", dict(nx=64, ny=40, dim=2, bc=("reflect",) * 4, fmax=0.999, cfl=100)),
    ("2d-neumann-f1", dict(nx=36, ny=20, dim=2, bc=("neumann",) * 4, fmax=1.0, cfl=7)),
    ("2d-inflow", dict(nx=48, ny=24, dim=2, bc=("inflow", "reflect", "inflow", "neumann"),
                       fmax=0.9, cfl=50)),
    ("1d-periodic-ragged", dict(nx=600, ny=1, dim=1, bc=("periodic",) * 4, fmax=0.99, cfl=50)),
    ("1d-inflow", dict(nx=300, ny=1, dim=1, bc=("inflow", "neumann", "periodic", "periodic"),
                       fmax=1.0, cfl=20)),
]


def _case(kw, seed=3):
    kw = dict(kw)
    return inputs.random_admissible_2d(kw.pop("nx"), kw.pop("ny"), seed=seed, **kw)


def _scale(ref):
    return np.maximum(np.abs(ref).max(axis=(1, 2), keepdims=True), 1e-300)


def _close(got, ref, rtol):
    err = np.abs(got - ref) / _scale(ref)
    assert err.max() <= rtol, (err.max(), np.unravel_index(err.argmax(), err.shape))


def _setup(kw, seed=3, precision=m1.FP64):
    case = _case(kw, seed)
    g = O.Grid.from_case(case)
    desc = m1.desc_from_case(case, lmax=1, precision=precision)
    sig = np.stack([case["sa"], case["ss"]])
    return case, g, desc, sig


@pytest.mark.parametrize("name,kw", CASES)
def test_apply_operator(name, kw):
    case, g, desc, sig = _setup(kw)
    got, _ = m1.m1_op_level(desc, case["dt"], sig, case["state"], mode=m1.OP_APPLY,
                            inflow=case["inflow"])
    ref = O.apply_A(g, case["dt"], case["sa"], case["ss"], case["state"])
    _close(got, ref, 1e-12)


@pytest.mark.parametrize("name,kw", CASES)
def test_residual_and_norm(name, kw):
    case, g, desc, sig = _setup(kw)
    b = O.rhs_of(g, case["state"]) * 1.01
    got, nrm = m1.m1_op_level(desc, case["dt"], sig, case["state"], b, mode=m1.OP_RESIDUAL,
                              inflow=case["inflow"])
    ref = O.residual(g, case["dt"], case["sa"], case["ss"], b, case["state"])
    _close(got, ref, 1e-12)
    assert nrm == pytest.approx(O.norm(g, ref), rel=1e-12)


@pytest.mark.parametrize("name,kw", CASES[:3])
def test_fas_rhs(name, kw):
    case, g, desc, sig = _setup(kw)
    rng = np.random.default_rng(5)
    r = rng.normal(0, 1, case["state"].shape)
    got, _ = m1.m1_op_level(desc, case["dt"], sig, case["state"], r, mode=m1.OP_FAS_RHS,
                            inflow=case["inflow"])
    ref = O.apply_A(g, case["dt"], case["sa"], case["ss"], case["state"]) + r
    _close(got, ref, 1e-12)


@pytest.mark.parametrize("name,kw", CASES)
def test_jacobi_sweep(name, kw):
    case, g, desc, sig = _setup(kw)
    b = O.rhs_of(g, case["state"])
    v1, _ = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, case["state"])
    # sweep from a perturbed iterate so neighbours and centre differ
    got, _ = m1.m1_op_level(desc, case["dt"], sig, v1, b, mode=m1.OP_JACOBI,
                            inflow=case["inflow"])
    ref, it = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, v1)
    assert it >= 0
    _close(got, ref, 1e-12)


@pytest.mark.parametrize("name,kw", CASES)
@pytest.mark.parametrize("dtau", [1e-3, 0.7, 50.0])
def test_pseudo_time_step(name, kw, dtau):
    case, g, desc, sig = _setup(kw)
    rng = np.random.default_rng(9)
    f = rng.normal(0, 1, case["state"].shape) * case["state"][0] + O.rhs_of(g, case["state"])
    got, _ = m1.m1_op_level(desc, case["dt"], sig, case["state"], f, mode=m1.OP_PSEUDO,
                            dtau=dtau, theta=0.5, inflow=case["inflow"])
    ref, it = O.pseudo_time_smooth(g, case["dt"], case["sa"], case["ss"], f, case["state"], dtau,
                                   m=1, nu=1, theta=0.5)
    assert it >= 0
    _close(got, ref, 1e-12)
    assert np.all(got[0] > 0) and np.all(np.hypot(got[1], got[2]) <= got[0] * (1 + 1e-12))


@pytest.mark.parametrize("name,kw", CASES)
def test_restriction(name, kw):
    case, g, desc, sig = _setup(kw)
    rng = np.random.default_rng(2)
    r = rng.normal(0, 1, case["state"].shape)
    cs, cr = m1.m1_op_restrict(m1.desc_from_case(case, lmax=2), case["state"], r,
                               inflow=case["inflow"])
    _close(cs, O.restrict_state(g, case["state"], O.KIND_STATE), 1e-15)
    _close(cr, O.restrict_state(g, r, O.KIND_DIFF), 1e-15)


@pytest.mark.parametrize("name,kw", CASES)
def test_prolong_correct_and_damping(name, kw):
    case, g, desc, sig = _setup(kw)
    rng = np.random.default_rng(4)
    vc = O.restrict_state(g, case["state"])
    uc = vc + rng.normal(0, 0.6, vc.shape) * vc[0]
    got, nd = m1.m1_op_prolong_correct(m1.desc_from_case(case, lmax=2), uc, vc, case["state"])
    ref, nd_ref = O.prolong_correct(g, uc, vc, case["state"])
    assert nd == nd_ref and nd > 0      # the same cells are damped
    _close(got, ref, 1e-13)


@pytest.mark.parametrize("name,kw", CASES[:2] + CASES[4:5])
def test_fp32_kernels_close_to_fp64_oracle(name, kw):
    case, g, desc, sig = _setup(kw, precision=m1.MIXED)
    b = O.rhs_of(g, case["state"])
    got, _ = m1.m1_op_level(desc, case["dt"], sig, case["state"], b, mode=m1.OP_JACOBI,
                            inflow=case["inflow"])
    ref, _ = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, case["state"])
    _close(got, ref, 2e-5)
    got, _ = m1.m1_op_level(desc, case["dt"], sig, case["state"], mode=m1.OP_APPLY,
                            inflow=case["inflow"])
    ref = O.apply_A(g, case["dt"], case["sa"], case["ss"], case["state"])
    _close(got, ref, 2e-5)


@pytest.mark.parametrize("name,kw", CASES[:2] + CASES[4:5])
def test_mixed_grid_jacobi_close_to_fp64_oracle(name, kw):
    """Two Jacobi sweeps on a MIXED grid (FP32 sweeps of the correction equation
    around the FP64 state, accumulated in FP64) against two FP64 oracle sweeps."""
    case, g, desc, sig = _setup(kw, precision=m1.MIXED)
    b = O.rhs_of(g, case["state"])
    v1, _ = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, case["state"])
    ref, _ = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, v1)
    grid = m1.grid_from_case(case, lmax=1, precision=m1.MIXED)
    grid.jacobi(case["dt"], 2)
    got = np.stack(grid.get_state())
    grid.close()
    _close(got, ref, 5e-5)      # two sweeps, each within the 2e-5 of one FP32 sweep


def test_full_size_sweep_matches_oracle():
    # the 1024^2 workload (lognormal opacities, hot square, reflecting walls):
    # one Jacobi sweep and one operator application over the whole grid
    case = inputs.hot_square_2d(1024)
    g = O.Grid.from_case(case)
    desc = m1.desc_from_case(case, lmax=1)
    sig = np.stack([case["sa"], case["ss"]])
    b = O.rhs_of(g, case["state"])
    v1, _ = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, case["state"])
    got, _ = m1.m1_op_level(desc, case["dt"], sig, v1, b, mode=m1.OP_JACOBI)
    ref, _ = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, v1)
    _close(got, ref, 1e-12)


def _extreme_case(kind, nx=40, ny=24, seed=17):
    """Admissible states far outside the nondimensional range: a hot gas (T up
    to 1e9, E = a_r T^4 up to 1e36, opacities up to 1e4: K T^3 and g'^2 of the
    local quartic overflow FP32) or a cold one (T from 1e-44 to 1e-39, E from
    1e-120 to 1e-100: the quartic's right-hand side and root are below FP32's
    normal range; E stays where |F|^2 is an FP64 normal number, which the
    oracle's closure needs)."""
    rng = np.random.default_rng(seed)
    if kind == "hot":
        T = 10.0 ** rng.uniform(5.0, 9.0, (ny, nx))
        E = T ** 4 * rng.uniform(0.5, 2.0, (ny, nx))
    else:
        T = 10.0 ** rng.uniform(-44.0, -39.0, (ny, nx))
        E = 10.0 ** rng.uniform(-120.0, -100.0, (ny, nx))
    th = rng.uniform(0, 2 * np.pi, (ny, nx))
    f = rng.uniform(0, 0.9, (ny, nx))
    state = np.stack([E, f * E * np.cos(th), f * E * np.sin(th), T * rng.uniform(0.8, 1.2, (ny, nx))])
    sa = 10.0 ** rng.uniform(0.0, 4.0, (ny, nx))
    ss = 10.0 ** rng.uniform(-2.0, 2.0, (ny, nx))
    desc = dict(dim=2, nx=nx, ny=ny, lx=1.0, ly=ny / nx, bc=["reflect"] * 4, c=1.0, a_r=1.0,
                c_v=1.0)
    return dict(desc=desc, dt=10.0 / nx, state=state, sa=sa, ss=ss, inflow=None, lmax=1, tol=1e-8)


@pytest.mark.parametrize("kind", ["hot", "cold"])
def test_local_solve_outside_fp32_range(kind):
    """The FP64 local solve seeds Newton in FP32 only where FP32 can represent the
    quartic; elsewhere it solves in FP64.  One Jacobi sweep matches the oracle
    cell by cell and no local solve is reported as failed."""
    case = _extreme_case(kind)
    g = O.Grid.from_case(case)
    desc = m1.desc_from_case(case, lmax=1)
    sig = np.stack([case["sa"], case["ss"]])
    b = O.rhs_of(g, case["state"])
    v1, it = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, case["state"])
    assert it >= 0
    ref, it = O.jacobi_sweep(g, case["dt"], case["sa"], case["ss"], b, v1)
    assert it >= 0
    got, fails = m1.m1_op_level(desc, case["dt"], sig, v1, b, mode=m1.OP_JACOBI)
    assert fails == 0
    assert np.all(np.isfinite(got))
    # per cell: E and T relative to themselves, the flux relative to E
    errE = np.abs(got[0] - ref[0]) / ref[0]
    errF = np.hypot(got[1] - ref[1], got[2] - ref[2]) / ref[0]
    errT = np.abs(got[3] - ref[3]) / ref[3]
    assert max(errE.max(), errF.max(), errT.max()) <= 1e-12, (errE.max(), errF.max(), errT.max())


def test_fma_peak_probe():
    """The FP64 FMA probe measures a rate below the nominal pipe ceiling (152 SMs
    x 2 DFMA per clock x the maximum SM clock, 2.07 GHz on GB300) and well above a
    tenth of it; the FP32 rate is many times the FP64 one."""
    f64 = m1.probe_fma_peak(m1.FP64, reps=3)
    f32 = m1.probe_fma_peak(m1.MIXED, reps=3)
    nominal = 152 * 2 * 2.07e9
    assert 0.1 * nominal < f64 <= 1.02 * nominal, f64
    assert f32 > 20 * f64, (f32, f64)


@pytest.mark.parametrize("name,kw", CASES)
def test_double_word_residual(name, kw):
    """The residual in double-word FP32 (the mixed path's defect arithmetic)
    against the oracle: about 48 bits per operation (relative error a few
    2^-48 per step, Joldes, Muller & Popescu 2017) through the closure and the
    neighbour sums, so within 1e-11 of each field's scale (the FP64 kernel's
    1e-12 with a margin for the shorter significand) and the norm within 1e-11."""
    case, g, desc, sig = _setup(kw)
    b = O.rhs_of(g, case["state"]) * 1.01
    got, nrm = m1.m1_op_level(desc, case["dt"], sig, case["state"], b, mode=m1.OP_RESIDUAL_DW,
                              inflow=case["inflow"])
    ref = O.residual(g, case["dt"], case["sa"], case["ss"], b, case["state"])
    err = np.abs(got - ref) / _scale(ref)
    print(name, "double-word residual max rel error", err.max())
    _close(got, ref, 1e-11)
    assert nrm == pytest.approx(O.norm(g, ref), rel=1e-11)
