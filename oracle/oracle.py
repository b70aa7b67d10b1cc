"""Python handle on the FP64 CPU oracle (``m1_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
``bench.py`` may import this module; the product path never does.  It shares no
code with the CUDA implementation; both take their inputs from
``paper_2208_14703_gb300.inputs``.

Arrays: a state is a float64 array of shape (4, ny, nx) holding the planes
E, Fx, Fy, T (1D: ny = 1, Fy = 0).  Opacities are (ny, nx).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "m1_oracle.c")
LIB = os.path.join(HERE, "liboracle_m1.so")

BC = {"periodic": 0, "reflect": 1, "neumann": 2, "inflow": 3}
KIND_STATE, KIND_DIFF = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


LIB_OMP = os.path.join(HERE, "liboracle_m1_omp.so")
_FLAGS = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no contraction so x86 and Arm
    agree): the one-core build, and the all-core build of the same source with
    OpenMP when the compiler supports it (else only the one-core build)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.run(_FLAGS + ["-o", LIB, SRC, "-lm"], check=True)
    if force or not os.path.exists(LIB_OMP) or os.path.getmtime(LIB_OMP) < os.path.getmtime(SRC):
        subprocess.run(_FLAGS + ["-fopenmp", "-o", LIB_OMP, SRC, "-lm"], check=False,
                       stderr=subprocess.DEVNULL)
    return LIB


_LIB = None
_LIBS = {}


def _load(path):
    if path not in _LIBS:
        L = bind(ctypes.CDLL(path))
        L.ora_threads.restype = ctypes.c_int
        _LIBS[path] = L
    return _LIBS[path]


def lib():
    global _LIB
    if _LIB is None:
        build()
        _LIB = _load(LIB)
    return _LIB


def have_all_cores() -> bool:
    build()
    return os.path.exists(LIB_OMP)


def use_all_cores(on: bool = True) -> int:
    """Route every call of this module to the all-core (OpenMP) build of the
    same source (on) or the one-core build (off).  Returns the thread count."""
    global _LIB
    build()
    _LIB = _load(LIB_OMP if on else LIB)
    return threads()


def threads() -> int:
    """Host threads the oracle's cell loops run on (1 for the one-core build)."""
    return int(lib().ora_threads())


def bind(L):
    """Declare the argument and result types of the oracle's exported functions
    on a loaded copy of the library (the tests also bind copies built with a
    planted mistake, to show that the pins catch it)."""
    L.ora_closure.argtypes = [ctypes.c_double] * 4 + [_dp]
    L.ora_eddington_factor.argtypes = [ctypes.c_double]
    L.ora_eddington_factor.restype = ctypes.c_double
    L.ora_apply_A.argtypes = [_ip, _dp, _dp, ctypes.c_double, _dp, _dp, _dp, _dp]
    L.ora_residual.argtypes = [_ip, _dp, _dp, ctypes.c_double, _dp, _dp, _dp, _dp, _dp]
    L.ora_norm.argtypes = [_ip, _dp, _dp]
    L.ora_norm.restype = ctypes.c_double
    L.ora_jacobi_sweep.argtypes = [_ip, _dp, _dp, ctypes.c_double, _dp, _dp, _dp, _dp, _dp,
                                   ctypes.c_double, ctypes.c_double]
    L.ora_jacobi_sweep.restype = ctypes.c_int
    L.ora_local_solve.argtypes = [ctypes.c_double] * 7 + [_dp, _dp]
    L.ora_local_solve.restype = ctypes.c_int
    L.ora_max_admissible_step.argtypes = [ctypes.c_double] * 9
    L.ora_max_admissible_step.restype = ctypes.c_double
    L.ora_admissible.argtypes = [ctypes.c_double] * 5
    L.ora_admissible.restype = ctypes.c_int
    L.ora_pseudo_time_smooth.argtypes = [_ip, _dp, _dp, ctypes.c_double, _dp, _dp, _dp, _dp,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double]
    L.ora_pseudo_time_smooth.restype = ctypes.c_int
    L.ora_restrict_state.argtypes = [_ip, _dp, _dp, ctypes.c_int, _dp, _dp]
    L.ora_restrict_scalar.argtypes = [_ip, _dp, _dp, _dp]
    L.ora_prolong.argtypes = [_ip, _dp, _dp, ctypes.c_int, _dp, _dp]
    L.ora_prolong_correct.argtypes = [_ip, _dp, _dp, _dp, _dp, ctypes.c_double]
    L.ora_prolong_correct.restype = ctypes.c_int
    L.ora_implicit_step.argtypes = [_ip, _dp, _dp, ctypes.c_double, _dp, _dp, _ip, _dp, _dp,
                                    _dp, _dp, _dp]
    L.ora_implicit_step.restype = ctypes.c_int
    return L


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Grid:
    """A uniform Cartesian grid: dim 1 or 2, nx x ny cells of size hx x hy."""
    dim: int
    nx: int
    ny: int
    hx: float
    hy: float
    c: float = 1.0
    a_r: float = 1.0
    c_v: float = 1.0
    bc: tuple = ("periodic",) * 4          # west, east, south, north
    inflow: np.ndarray | None = None       # (4 walls, 3 fields E/Fx/Fy, max(nx, ny))
    _i: np.ndarray = field(init=False, repr=False)
    _dd: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        if self.dim == 1:
            self.ny = 1
        self._i = np.array([self.dim, self.nx, self.ny] + [BC[b] for b in self.bc], dtype=np.int32)
        self._dd = np.array([self.hx, self.hy, self.c, self.a_r, self.c_v], dtype=np.float64)
        if self.inflow is not None:
            self.inflow = _f64(self.inflow)

    @property
    def n(self):
        return self.nx * self.ny

    def ip(self):
        return self._i.ctypes.data_as(_ip)

    def dp(self):
        return self._dd.ctypes.data_as(_dp)

    def coarse(self, inflow_c=None) -> "Grid":
        return Grid(self.dim, self.nx // 2, self.ny // 2 if self.dim == 2 else 1, 2 * self.hx,
                    2 * self.hy if self.dim == 2 else self.hy, self.c, self.a_r, self.c_v,
                    self.bc, inflow_c)

    @classmethod
    def from_case(cls, case: dict) -> "Grid":
        d = case["desc"]
        return cls(d["dim"], d["nx"], d["ny"], d["lx"] / d["nx"],
                   d["ly"] / d["ny"] if d["dim"] == 2 else d["ly"], d["c"], d["a_r"], d["c_v"],
                   tuple(d["bc"]), case.get("inflow"))


def closure(E, Fx, Fy, c=1.0):
    P = np.zeros(3)
    lib().ora_closure(E, Fx, Fy, c, _d(P))
    return P


def eddington_factor(f):
    return lib().ora_eddington_factor(f)


def apply_A(g: Grid, dt, sa, ss, v):
    v, sa, ss = _f64(v), _f64(sa), _f64(ss)
    out = np.zeros_like(v)
    lib().ora_apply_A(g.ip(), g.dp(), _d(g.inflow), dt, _d(sa), _d(ss), _d(v), _d(out))
    return out


def residual(g: Grid, dt, sa, ss, b, v):
    v, b, sa, ss = _f64(v), _f64(b), _f64(sa), _f64(ss)
    r = np.zeros_like(v)
    lib().ora_residual(g.ip(), g.dp(), _d(g.inflow), dt, _d(sa), _d(ss), _d(b), _d(v), _d(r))
    return r


def norm(g: Grid, r):
    r = _f64(r)
    return lib().ora_norm(g.ip(), g.dp(), _d(r))


def jacobi_sweep(g: Grid, dt, sa, ss, rhs, v, w0=0.0, w1=1.0):
    v, rhs, sa, ss = _f64(v), _f64(rhs), _f64(sa), _f64(ss)
    out = np.zeros_like(v)
    it = lib().ora_jacobi_sweep(g.ip(), g.dp(), _d(g.inflow), dt, _d(sa), _d(ss), _d(rhs), _d(v),
                                _d(out), w0, w1)
    return out, it


def local_solve(w0, w1, diag, ka, kt, c_v, a_r, beta):
    beta = _f64(beta)
    out = np.zeros(4)
    it = lib().ora_local_solve(w0, w1, diag, ka, kt, c_v, a_r, _d(beta), _d(out))
    return out, it


def max_admissible_step(u, d, c=1.0):
    return lib().ora_max_admissible_step(*[float(x) for x in u], *[float(x) for x in d], c)


def admissible(u, c=1.0):
    return bool(lib().ora_admissible(*[float(x) for x in u], c))


def pseudo_time_smooth(g: Grid, dt, sa, ss, f, u, dtau, m=3, nu=1, theta=0.5):
    u = _f64(u).copy()
    f, sa, ss = _f64(f), _f64(sa), _f64(ss)
    it = lib().ora_pseudo_time_smooth(g.ip(), g.dp(), _d(g.inflow), dt, _d(sa), _d(ss), _d(f),
                                      _d(u), dtau, m, nu, theta)
    return u, it


def restrict_state(g: Grid, fine, kind=KIND_STATE):
    fine = _f64(fine)
    gc = g.coarse()
    out = np.zeros((4, gc.ny, gc.nx))
    lib().ora_restrict_state(g.ip(), g.dp(), _d(g.inflow), kind, _d(fine), _d(out))
    return out


def restrict_scalar(g: Grid, fine):
    fine = _f64(fine)
    gc = g.coarse()
    out = np.zeros((gc.ny, gc.nx))
    lib().ora_restrict_scalar(g.ip(), g.dp(), _d(fine), _d(out))
    return out


def prolong(g: Grid, coarse, kind=KIND_DIFF, inflow_c=None):
    coarse = _f64(coarse)
    out = np.zeros((4, g.ny, g.nx))
    inflow_c = _f64(inflow_c) if inflow_c is not None else None
    lib().ora_prolong(g.ip(), g.dp(), _d(inflow_c), kind, _d(coarse), _d(out))
    return out


def prolong_correct(g: Grid, uc, vc, uf, theta=0.5):
    uc, vc = _f64(uc), _f64(vc)
    uf = _f64(uf).copy()
    nd = lib().ora_prolong_correct(g.ip(), g.dp(), _d(uc), _d(vc), _d(uf), theta)
    return uf, nd


@dataclass
class SolveParams:
    """Section 5 defaults: nu0 = 3, nu_l = 1, m = 3, dtau_im^0 = 1e-3; the rest are
    the stated readings (eps_i, eps_d, clamps, theta's, max_cycles)."""
    lmax: int = 4
    nu0: int = 3
    nu_l: int = 1
    m: int = 3
    m_coarse: int = 3
    max_cycles: int = 20000
    literal_fas: int = 0
    dtau_rule: int = 0
    cycle: int = 0              # 0 V, 1 W, 2 F (Section 6.3; shapes in m1_oracle.c)
    dtau0: float = 1e-3
    grow: float = 1.1
    shrink: float = 0.5
    eps_i: float = 1e-2
    eps_d: float = 1e-4
    tol: float = 1e-10
    dtau_min: float = 1e-12
    dtau_max: float = 1e6
    theta_ex: float = 0.5
    theta_c: float = 0.5

    def arrays(self):
        ip = np.array([self.lmax, self.nu0, self.nu_l, self.m, self.m_coarse, self.max_cycles,
                       self.literal_fas, self.dtau_rule, self.cycle], dtype=np.int32)
        dp = np.array([self.dtau0, self.grow, self.shrink, self.eps_i, self.eps_d, self.tol,
                       self.dtau_min, self.dtau_max, self.theta_ex, self.theta_c])
        return ip, dp


STATUS = {0: "ok", -1: "invalid_parameters", -2: "nonadmissible_input", -4: "not_converged"}


def implicit_step(g: Grid, dt, sa, ss, v, params: SolveParams):
    """Algorithm 4: one implicit step.  Returns (v_new, stats, res_hist, dtau_hist)."""
    v = _f64(v).copy()
    sa, ss = _f64(sa), _f64(ss)
    ip, dp = params.arrays()
    stats = np.zeros(8 + params.lmax)
    res_hist = np.zeros(params.max_cycles + 1)
    dtau_hist = np.zeros(max(params.max_cycles, 1))
    lib().ora_implicit_step(g.ip(), g.dp(), _d(g.inflow), dt, _d(sa), _d(ss),
                            ip.ctypes.data_as(_ip), _d(dp), _d(v), _d(stats), _d(res_hist),
                            _d(dtau_hist))
    cyc = int(stats[0])
    st = dict(cycles=cyc, res0=stats[1], res=stats[2], dtau=stats[3], fine_sweeps=int(stats[4]),
              status=int(stats[5]), newton_fail=int(stats[6]), damped=int(stats[7]),
              visits=[int(x) for x in stats[8:]])
    return v, st, res_hist[:cyc + 1].copy(), dtau_hist[:cyc].copy()


def rhs_of(g: Grid, v):
    """b = (E^n, F^n, C_v T^n), the right-hand side of Algorithm 4."""
    b = _f64(v).copy()
    b[3] *= g.c_v
    return b
