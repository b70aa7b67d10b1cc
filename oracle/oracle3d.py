"""ctypes wrapper of the 3D FP64 CPU oracle (oracle/m1_oracle3d.c).

TEST INFRASTRUCTURE ONLY: the tests use it; the product path never imports,
links or runs anything under oracle/.  States are float64 arrays of shape
(5, nz, ny, nx): planes E, Fx, Fy, Fz, T.  Walls (W, E, S, N, B, T) are
"periodic", "reflect", "neumann" or "inflow"; inflow profiles are an array
(6 walls, 4 fields E/Fx/Fy/Fz, F) with F the largest face, a wall's face indexed
q_b * n_a + q_a over its two other axes a < b.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "m1_oracle3d.c")
LIB = os.path.join(HERE, "liboracle3d.so")
BC = {"periodic": 0, "reflect": 1, "neumann": 2, "inflow": 3}
KIND_STATE, KIND_DIFF = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


LIB_OMP = os.path.join(HERE, "liboracle3d_omp.so")
_FLAGS = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the 3D oracle with gcc (plain C99, no contraction so x86 and Arm
    agree), and its all-core OpenMP build when the compiler supports it."""
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
        L = ctypes.CDLL(path)
        L.ora3_norm.restype = ctypes.c_double
        L.ora3_threads.restype = ctypes.c_int
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
    _LIB = _load(LIB_OMP if on and os.path.exists(LIB_OMP) else LIB)
    return int(_LIB.ora3_threads())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _d(a):
    return None if a is None else a.ctypes.data_as(_dp)


@dataclass
class Grid3:
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    bc: tuple = ("periodic",) * 6
    c: float = 1.0
    a_r: float = 1.0
    c_v: float = 1.0
    inflow: np.ndarray | None = None

    @property
    def face(self):
        """Doubles per field of an inflow profile: the largest face."""
        return max(self.ny * self.nz, self.nx * self.nz, self.nx * self.ny)

    def inflow_ptr(self):
        if self.inflow is None:
            return None
        self.inflow = _f64(self.inflow)
        assert self.inflow.shape == (6, 4, self.face)
        return _d(self.inflow)

    def ip(self):
        self._ip = np.array([self.nx, self.ny, self.nz, *[BC[b] for b in self.bc]], dtype=np.int32)
        return self._ip.ctypes.data_as(_ip)

    def dp(self):
        self._dp = np.array([self.hx, self.hy, self.hz, self.c, self.a_r, self.c_v])
        return _d(self._dp)

    @property
    def shape(self):
        return (5, self.nz, self.ny, self.nx)

    def coarse(self, inflow_c=None) -> "Grid3":
        return Grid3(self.nx // 2, self.ny // 2, self.nz // 2, 2 * self.hx, 2 * self.hy,
                     2 * self.hz, self.bc, self.c, self.a_r, self.c_v, inflow_c)


def closure(E, F, c=1.0):
    """The 3x3 pressure tensor of Eq. (5) for one cell."""
    P = np.zeros(9)
    lib().ora3_closure(ctypes.c_double(E), _d(_f64(F)), ctypes.c_double(c), _d(P))
    return P.reshape(3, 3)


def apply_A(g: Grid3, dt, sa, ss, v):
    v, sa, ss = _f64(v), _f64(sa), _f64(ss)
    out = np.zeros(g.shape)
    lib().ora3_apply_A(g.ip(), g.dp(), g.inflow_ptr(), ctypes.c_double(dt), _d(sa), _d(ss), _d(v),
                       _d(out))
    return out


def residual(g: Grid3, dt, sa, ss, b, v):
    b, v, sa, ss = _f64(b), _f64(v), _f64(sa), _f64(ss)
    r = np.zeros(g.shape)
    lib().ora3_residual(g.ip(), g.dp(), g.inflow_ptr(), ctypes.c_double(dt), _d(sa), _d(ss), _d(b),
                        _d(v), _d(r))
    return r


def norm(g: Grid3, r):
    return lib().ora3_norm(g.ip(), g.dp(), _d(_f64(r)))


def jacobi_sweep(g: Grid3, dt, sa, ss, rhs, v, w0=0.0, w1=1.0):
    rhs, v, sa, ss = _f64(rhs), _f64(v), _f64(sa), _f64(ss)
    out = np.zeros(g.shape)
    it = lib().ora3_jacobi_sweep(g.ip(), g.dp(), g.inflow_ptr(), ctypes.c_double(dt), _d(sa),
                                 _d(ss), _d(rhs), _d(v), _d(out), ctypes.c_double(w0),
                                 ctypes.c_double(w1))
    return out, it


def pseudo_time_smooth(g: Grid3, dt, sa, ss, f, u, dtau, m=3, nu=1, theta=0.5):
    f, sa, ss = _f64(f), _f64(sa), _f64(ss)
    u = _f64(u).copy()
    it = lib().ora3_pseudo_time_smooth(g.ip(), g.dp(), g.inflow_ptr(), ctypes.c_double(dt), _d(sa),
                                       _d(ss), _d(f), _d(u), ctypes.c_double(dtau), m, nu,
                                       ctypes.c_double(theta))
    return u, it


def restrict_state(g: Grid3, fine, kind=KIND_STATE):
    gc = g.coarse()
    out = np.zeros(gc.shape)
    lib().ora3_restrict_state(g.ip(), g.dp(), g.inflow_ptr(), kind, _d(_f64(fine)), _d(out))
    return out


def prolong(g: Grid3, coarse, kind=KIND_STATE, inflow_c=None):
    """Plain prolongation of a coarse state onto the fine grid g (coarse ghosts
    of kind `kind`; inflow_c: the coarse grid's profiles)."""
    out = np.zeros(g.shape)
    lib().ora3_prolong(g.ip(), g.dp(), _d(None if inflow_c is None else _f64(inflow_c)), kind,
                       _d(_f64(coarse)), _d(out))
    return out


@dataclass
class SolveParams3:
    lmax: int = 2
    nu0: int = 3
    nu_l: int = 1
    m: int = 3
    m_coarse: int = 3
    max_cycles: int = 20000
    dtau_rule: int = 0
    cycle: int = 0
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


def implicit_step(g: Grid3, dt, sa, ss, v, p: SolveParams3):
    """Algorithm 4 in 3D.  Returns (v_new, stats, res_hist)."""
    v = _f64(v).copy()
    sa, ss = _f64(sa), _f64(ss)
    ip = np.array([p.lmax, p.nu0, p.nu_l, p.m, p.m_coarse, p.max_cycles, p.dtau_rule, p.cycle],
                  dtype=np.int32)
    dp = np.array([p.dtau0, p.grow, p.shrink, p.eps_i, p.eps_d, p.tol, p.dtau_min, p.dtau_max,
                   p.theta_ex, p.theta_c])
    stats = np.zeros(8)
    hist = np.zeros(p.max_cycles + 1)
    lib().ora3_implicit_step(g.ip(), g.dp(), g.inflow_ptr(), ctypes.c_double(dt), _d(sa), _d(ss),
                             ip.ctypes.data_as(_ip), _d(dp), _d(v), _d(stats), _d(hist))
    cyc = int(stats[0])
    st = dict(cycles=cyc, res0=stats[1], res=stats[2], dtau=stats[3], fine_sweeps=int(stats[4]),
              status=int(stats[5]), newton_fail=int(stats[6]), damped=int(stats[7]))
    return v, st, hist[:cyc + 1].copy()
