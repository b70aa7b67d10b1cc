"""Python binding of libm1 (include/m1.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all the
arithmetic of the implicit M1 step runs in the CUDA kernels of libm1.so.  The
module raises at import time if libm1.so has not been built, so nothing can
silently run without the CUDA library.

Arrays: numpy float64 (host) or torch CUDA float64 tensors (device).  States
are passed per field (E, Fx, Fy, T), each of shape (ny, nx) or (nx,) in 1D.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libm1.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libm1.so is not built ({_LIB_PATH}); run "
                      "`python -m paper_2208_14703_gb300.build` (needs nvcc)")
_lib = ctypes.CDLL(_LIB_PATH)

OK, PENDING, ERR_INVALID_ARG, ERR_NONADMISSIBLE_INPUT, ERR_OOM, ERR_NOT_CONVERGED, ERR_CUDA, \
    ERR_TIMEOUT, ERR_REJECTED = 0, 1, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "OK", 1: "PENDING", -1: "INVALID_ARG", -2: "NONADMISSIBLE_INPUT", -3: "OOM",
                -4: "NOT_CONVERGED", -5: "CUDA", -6: "TIMEOUT", -7: "REJECTED"}
BC = {"periodic": 0, "reflect": 1, "neumann": 2, "inflow": 3}
FP64, MIXED = 0, 1
DTAU_ABS, DTAU_SIGNED = 0, 1
CYCLE_V, CYCLE_W, CYCLE_F = 0, 1, 2
OP3_APPLY, OP3_RESIDUAL, OP3_JACOBI = 0, 1, 2
SMALL_CELLS = 65536          # servers: requests of at most this many cells take the small lane
OP_APPLY, OP_RESIDUAL, OP_FAS_RHS, OP_JACOBI, OP_PSEUDO, OP_RESIDUAL_DW = 0, 1, 2, 3, 4, 5

EXPORTS = ["m1_default_params", "m1_create_grid", "m1_destroy_grid", "m1_set_state",
           "m1_set_inflow", "m1_get_state", "m1_implicit_step", "m1_residual_norm",
           "m1_step_history", "m1_jacobi", "m1_op_level", "m1_op_restrict", "m1_op_prolong_correct",
           "m1_residual_norm_noalloc", "m1_last_error", "m1_create_batch", "m1_destroy_batch",
           "m1_batch_set_state", "m1_batch_set_inflow", "m1_batch_get_state",
           "m1_batch_implicit_step", "m1_server_create", "m1_serve_submit", "m1_serve_poll",
           "m1_serve_wait", "m1_server_get_stats", "m1_server_destroy", "m1_autotune",
           "m1_set_tuning", "m1_strip_rows", "m1_op_level3", "m1_probe_fma_peak",
           "m1_op_elementwise", "m1_dw_split", "m1_f32_widen",
           "m1_create_grid3", "m1_destroy_grid3", "m1_grid3_set_state", "m1_grid3_set_inflow",
           "m1_grid3_get_state", "m1_grid3_implicit_step", "m1_grid3_step_history"]


class M1Error(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = f"{what}: {STATUS_NAMES.get(status, status)}"
        err = _lib.m1_last_error().decode()
        if status == ERR_CUDA and err:
            msg += f" ({err})"
        super().__init__(msg)


class GridDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("bc", ctypes.c_int * 4),
                ("lmax", ctypes.c_int), ("c", ctypes.c_double), ("a_r", ctypes.c_double),
                ("c_v", ctypes.c_double), ("precision", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("nu0", ctypes.c_int), ("nu_l", ctypes.c_int), ("m_pseudo", ctypes.c_int),
                ("m_coarse", ctypes.c_int), ("dtau0", ctypes.c_double),
                ("grow", ctypes.c_double), ("shrink", ctypes.c_double),
                ("eps_i", ctypes.c_double), ("eps_d", ctypes.c_double),
                ("tol", ctypes.c_double), ("dtau_min", ctypes.c_double),
                ("dtau_max", ctypes.c_double), ("theta_ex", ctypes.c_double),
                ("theta_c", ctypes.c_double), ("max_cycles", ctypes.c_int),
                ("dtau_rule", ctypes.c_int), ("cycle", ctypes.c_int)]


class StepStats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("res0", ctypes.c_double), ("res", ctypes.c_double),
                ("dtau_final", ctypes.c_double), ("sweeps", ctypes.c_longlong),
                ("ms", ctypes.c_double), ("status", ctypes.c_int),
                ("newton_fail", ctypes.c_uint), ("damped", ctypes.c_uint),
                ("launches", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_longlong), ("steps_done", ctypes.c_longlong),
                ("cycles", ctypes.c_longlong), ("wall_s", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("active", ctypes.c_int), ("queued", ctypes.c_int),
                ("bytes_in_use", ctypes.c_longlong), ("bytes_peak", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneEntry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("strip_rows", ctypes.c_int),
                ("staging", ctypes.c_int), ("ms", ctypes.c_double),
                ("ms_default", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_lib.m1_last_error.restype = ctypes.c_char_p
_lib.m1_default_params.argtypes = [ctypes.POINTER(SolveParams)]
_lib.m1_create_grid.argtypes = [ctypes.POINTER(GridDesc), _vp, ctypes.POINTER(_vp)]
_lib.m1_destroy_grid.argtypes = [_vp]
_lib.m1_set_state.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int]
_lib.m1_set_inflow.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
_lib.m1_get_state.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]
_lib.m1_implicit_step.argtypes = [_vp, ctypes.c_double, ctypes.POINTER(SolveParams),
                                  ctypes.POINTER(StepStats)]
_lib.m1_residual_norm.argtypes = [_vp, ctypes.c_double, _dp]
_lib.m1_step_history.argtypes = [_vp, _vp, _vp, ctypes.c_int]
_lib.m1_jacobi.argtypes = [_vp, ctypes.c_double, ctypes.c_int]
_lib.m1_op_level.argtypes = [ctypes.POINTER(GridDesc), _vp, ctypes.c_double, _vp, _vp, _vp,
                             ctypes.c_int, ctypes.c_double, ctypes.c_double, _vp, _dp]
_lib.m1_residual_norm_noalloc.argtypes = [ctypes.POINTER(GridDesc), ctypes.c_double, _vp, _vp,
                                          _vp, _vp, _vp, _vp]
_lib.m1_create_batch.argtypes = [ctypes.POINTER(GridDesc), ctypes.c_int, _vp, ctypes.POINTER(_vp)]
_lib.m1_destroy_batch.argtypes = [_vp]
_lib.m1_batch_set_state.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int]
_lib.m1_batch_set_inflow.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
_lib.m1_batch_get_state.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int]
_lib.m1_batch_implicit_step.argtypes = [_vp, _dp, ctypes.POINTER(SolveParams),
                                        ctypes.POINTER(StepStats)]
_lib.m1_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(SolveParams), ctypes.c_longlong, _vp,
                                  ctypes.POINTER(_vp)]
_lib.m1_serve_submit.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_double,
                                 ctypes.POINTER(SolveParams), ctypes.POINTER(ctypes.c_ulonglong)]
_lib.m1_serve_poll.argtypes = [_vp, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(StepStats)]
_lib.m1_serve_wait.argtypes = [_vp, ctypes.c_ulonglong, ctypes.c_double]
_lib.m1_server_get_stats.argtypes = [_vp, ctypes.POINTER(ServerStats)]
_lib.m1_server_destroy.argtypes = [_vp]
_lib.m1_autotune.argtypes = [_vp, ctypes.POINTER(TuneEntry), ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int)]
_lib.m1_set_tuning.argtypes = [ctypes.POINTER(TuneEntry), ctypes.c_int]
_lib.m1_strip_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int)]
_lib.m1_probe_fma_peak.argtypes = [ctypes.c_int, _vp, ctypes.c_int, _dp]
_lib.m1_op_elementwise.argtypes = [ctypes.c_int, _vp, ctypes.c_longlong, _vp, _vp]
_lib.m1_dw_split.argtypes = [_vp, ctypes.c_longlong, _vp, _vp]
_lib.m1_f32_widen.argtypes = [_vp, ctypes.c_longlong, _vp]
_lib.m1_op_restrict.argtypes = [ctypes.POINTER(GridDesc), _vp, _vp, _vp, _vp, _vp]
_lib.m1_op_prolong_correct.argtypes = [ctypes.POINTER(GridDesc), _vp, _vp, _vp, ctypes.c_double,
                                       _vp, ctypes.POINTER(ctypes.c_int)]


def _check(status, what, allow=()):
    if status != OK and status not in allow:
        raise M1Error(status, what)
    return status


def _ptr(a):
    """Data pointer of a numpy array (host) or a torch tensor (device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data
    return a.data_ptr()


def _host(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_desc(dim, nx, ny, lx, ly, bc, lmax, c=1.0, a_r=1.0, c_v=1.0, precision=FP64):
    d = GridDesc()
    d.dim, d.nx, d.ny = dim, nx, ny if dim == 2 else 1
    d.lx, d.ly = lx, ly
    for k, b in enumerate(bc):
        d.bc[k] = BC[b] if isinstance(b, str) else int(b)
    d.lmax, d.c, d.a_r, d.c_v, d.precision = lmax, c, a_r, c_v, precision
    return d


def desc_from_case(case, lmax=None, precision=FP64):
    s = case["desc"]
    return make_desc(s["dim"], s["nx"], s["ny"], s["lx"], s["ly"], s["bc"],
                     case["lmax"] if lmax is None else lmax, s["c"], s["a_r"], s["c_v"], precision)


def m1_default_params(**overrides) -> SolveParams:
    p = SolveParams()
    _check(_lib.m1_default_params(ctypes.byref(p)), "m1_default_params")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Grid:
    """Owner of one m1_grid_t (m1_create_grid / m1_destroy_grid)."""

    def __init__(self, desc: GridDesc, stream=None):
        h = _vp()
        _check(_lib.m1_create_grid(ctypes.byref(desc), stream, ctypes.byref(h)), "m1_create_grid")
        self.h = h
        self.desc = desc

    def close(self):
        if getattr(self, "h", None):
            _lib.m1_destroy_grid(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def shape(self):
        return (self.desc.ny, self.desc.nx)

    def set_state(self, E, Fx, Fy, T, sig_a=None, sig_s=None, on_device=False):
        if not on_device:
            E, Fx, Fy, T, sig_a, sig_s = map(_host, (E, Fx, Fy, T, sig_a, sig_s))
        st = _lib.m1_set_state(self.h, _ptr(E), _ptr(Fx), _ptr(Fy), _ptr(T), _ptr(sig_a),
                               _ptr(sig_s), int(on_device))
        return _check(st, "m1_set_state")

    def set_inflow(self, side, E, Fx, Fy):
        E, Fx, Fy = map(_host, (E, Fx, Fy))
        return _check(_lib.m1_set_inflow(self.h, side, _ptr(E), _ptr(Fx), _ptr(Fy)),
                      "m1_set_inflow")

    def get_state(self, out=None, on_device=False):
        """Returns (E, Fx, Fy, T) as host arrays, or fills `out` (4 arrays/tensors)."""
        if out is None:
            out = [np.zeros(self.shape) for _ in range(4)]
        st = _lib.m1_get_state(self.h, *[_ptr(a) for a in out], int(on_device))
        _check(st, "m1_get_state")
        return out

    def implicit_step(self, dt, params: SolveParams | None = None, allow_not_converged=False):
        stats = StepStats()
        st = _lib.m1_implicit_step(self.h, dt, ctypes.byref(params) if params else None,
                                   ctypes.byref(stats))
        _check(st, "m1_implicit_step", allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return stats

    def jacobi(self, dt, sweeps):
        """Queue `sweeps` Jacobi sweeps (Algorithm 1) on the grid's stream."""
        return _check(_lib.m1_jacobi(self.h, dt, sweeps), "m1_jacobi")

    def residual_norm(self, dt):
        out = ctypes.c_double()
        _check(_lib.m1_residual_norm(self.h, dt, ctypes.byref(out)), "m1_residual_norm")
        return out.value

    def step_history(self, length):
        hist = np.zeros(length)
        dtau = np.zeros(length)
        _check(_lib.m1_step_history(self.h, _ptr(hist), _ptr(dtau), length), "m1_step_history")
        return hist, dtau


class Batch:
    """Owner of one m1_batch_t: independent instances stepped together."""

    def __init__(self, descs, stream=None):
        arr = (GridDesc * len(descs))(*descs)
        h = _vp()
        _check(_lib.m1_create_batch(arr, len(descs), stream, ctypes.byref(h)), "m1_create_batch")
        self.h = h
        self.descs = list(descs)

    def close(self):
        if getattr(self, "h", None):
            _lib.m1_destroy_batch(self.h)
            self.h = None

    __del__ = close

    def __len__(self):
        return len(self.descs)

    def set_state(self, k, E, Fx, Fy, T, sig_a=None, sig_s=None, on_device=False):
        if not on_device:
            E, Fx, Fy, T, sig_a, sig_s = map(_host, (E, Fx, Fy, T, sig_a, sig_s))
        st = _lib.m1_batch_set_state(self.h, k, _ptr(E), _ptr(Fx), _ptr(Fy), _ptr(T), _ptr(sig_a),
                                     _ptr(sig_s), int(on_device))
        return _check(st, "m1_batch_set_state")

    def set_inflow(self, k, side, E, Fx, Fy):
        E, Fx, Fy = map(_host, (E, Fx, Fy))
        return _check(_lib.m1_batch_set_inflow(self.h, k, side, _ptr(E), _ptr(Fx), _ptr(Fy)),
                      "m1_batch_set_inflow")

    def get_state(self, k):
        d = self.descs[k]
        out = [np.zeros((d.ny, d.nx)) for _ in range(4)]
        _check(_lib.m1_batch_get_state(self.h, k, *[_ptr(a) for a in out], 0),
               "m1_batch_get_state")
        return out

    def implicit_step(self, dts, params: SolveParams | None = None, allow_not_converged=False):
        dts = np.ascontiguousarray(dts, dtype=np.float64)
        stats = (StepStats * len(self.descs))()
        st = _lib.m1_batch_implicit_step(self.h, dts.ctypes.data_as(_dp),
                                         ctypes.byref(params) if params else None, stats)
        _check(st, "m1_batch_implicit_step",
               allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return list(stats)


class Server:
    """Owner of one m1_server_t (continuous-batching request loop)."""

    def __init__(self, budget_bytes, max_slots, lmax, precision=FP64, structure=None,
                 stream=None, small_cells=SMALL_CELLS):
        h = _vp()
        st = _lib.m1_server_create(int(budget_bytes), max_slots, lmax, precision,
                                   ctypes.byref(structure) if structure else None,
                                   int(small_cells), stream, ctypes.byref(h))
        _check(st, "m1_server_create")
        self.h = h
        self._held = {}   # grids in flight, kept alive until their tickets complete

    def submit(self, grid: Grid, nsteps, dt, params: SolveParams | None = None):
        t = ctypes.c_ulonglong()
        st = _lib.m1_serve_submit(self.h, grid.h, nsteps, dt,
                                  ctypes.byref(params) if params else None, ctypes.byref(t))
        _check(st, "m1_serve_submit")
        self._held[t.value] = grid
        return t.value

    def poll(self, ticket):
        """(status, steps done, last step's StepStats); status PENDING while running."""
        n = ctypes.c_int()
        last = StepStats()
        st = _lib.m1_serve_poll(self.h, ticket, ctypes.byref(n), ctypes.byref(last))
        if st != PENDING:
            self._held.pop(ticket, None)
        return st, n.value, last

    def wait(self, ticket, timeout_s=600.0):
        st = _lib.m1_serve_wait(self.h, ticket, timeout_s)
        if st != ERR_TIMEOUT:
            self._held.pop(ticket, None)
        return st

    def stats(self):
        out = ServerStats()
        _check(_lib.m1_server_get_stats(self.h, ctypes.byref(out)), "m1_server_get_stats")
        return out

    def close(self):
        if getattr(self, "h", None):
            st = _lib.m1_server_destroy(self.h)
            self.h = None
            _check(st, "m1_server_destroy")

    def __del__(self):
        if getattr(self, "h", None):
            _lib.m1_server_destroy(self.h)
            self.h = None


def autotune(stream=None):
    """Run the strip-height autotuner; returns its entries as dicts."""
    buf = (TuneEntry * 64)()
    n = ctypes.c_int()
    _check(_lib.m1_autotune(stream, buf, 64, ctypes.byref(n)), "m1_autotune")
    return [buf[k].as_dict() for k in range(min(n.value, 64))]


def set_tuning(entries):
    """Install tuner entries (dicts with kind, n, strip_rows)."""
    arr = (TuneEntry * max(1, len(entries)))()
    for k, e in enumerate(entries):
        arr[k] = TuneEntry(e["kind"], e["n"], e["strip_rows"], e.get("staging", 0),
                           e.get("ms", 0.0), e.get("ms_default", 0.0))
    _check(_lib.m1_set_tuning(arr, len(entries)), "m1_set_tuning")


def strip_rows(kind, nx, ny):
    r = ctypes.c_int()
    _check(_lib.m1_strip_rows(kind, nx, ny, ctypes.byref(r)), "m1_strip_rows")
    return r.value


def load_case(target, case, index=None):
    """Set the state, opacities and inflow of an input case on a Grid or a
    Batch slot."""
    s = case["state"]
    args = (s[0], s[1], s[2], s[3], case["sa"], case["ss"])
    if index is None:
        target.set_state(*args)
    else:
        target.set_state(index, *args)
    if case.get("inflow") is not None:
        d = case["desc"]
        for w in range(4):
            if d["bc"][w] == "inflow":
                n = d["ny"] if w < 2 else d["nx"]
                prof = [case["inflow"][w, f, :n] for f in range(3)]
                if index is None:
                    target.set_inflow(w, *prof)
                else:
                    target.set_inflow(index, w, *prof)


def batch_from_cases(cases, lmax=None, precision=FP64, stream=None) -> Batch:
    b = Batch([desc_from_case(c, lmax, precision) for c in cases], stream)
    for k, c in enumerate(cases):
        load_case(b, c, k)
    return b


def grid_from_case(case, lmax=None, precision=FP64, stream=None) -> Grid:
    """A grid holding the state, opacities and inflow of an input case."""
    g = Grid(desc_from_case(case, lmax, precision), stream)
    load_case(g, case)
    return g


def m1_op_level(desc, dt, sig, state, rhs=None, mode=OP_APPLY, dtau=0.0, theta=0.5, inflow=None):
    n = desc.nx * desc.ny
    state = _host(state).reshape(4, n)
    sig = _host(sig).reshape(2, n)
    rhs = None if rhs is None else _host(rhs).reshape(4, n)
    inflow = _host(inflow)
    out = np.zeros((4, n))
    nrm = ctypes.c_double()
    st = _lib.m1_op_level(ctypes.byref(desc), _ptr(inflow), dt, _ptr(sig), _ptr(state), _ptr(rhs),
                          mode, dtau, theta, _ptr(out), ctypes.byref(nrm))
    _check(st, "m1_op_level")
    return out.reshape(4, desc.ny, desc.nx), nrm.value


def probe_fma_peak(precision=FP64, stream=None, reps=5):
    """FMA instructions per second summed over lanes (median of `reps` timed
    launches): the FP64 (DFMA) or FP32 (FFMA) pipe ceiling of this GPU."""
    out = ctypes.c_double()
    _check(_lib.m1_probe_fma_peak(precision, stream, reps, ctypes.byref(out)), "m1_probe_fma_peak")
    return out.value


FN_RCP64, FN_SQRT64, FN_RCP32, FN_SQRT32, FN_DW_SPLIT, FN_WIDEN = range(6)


def op_elementwise(fn, x, stream=None):
    """The kernels' per-element arithmetic applied on the device to a contiguous
    CUDA tensor x by m1_op_elementwise: float64 in and out for RCP64 / SQRT64,
    float32 for RCP32 / SQRT32, float64 in and float32 pairs [n, 2] out for
    DW_SPLIT, float32 in and float64 out for WIDEN."""
    import torch
    want = torch.float32 if fn in (FN_RCP32, FN_SQRT32, FN_WIDEN) else torch.float64
    if x.dtype != want or not x.is_cuda or not x.is_contiguous():
        raise ValueError(f"m1_op_elementwise fn {fn}: x must be a contiguous {want} CUDA tensor")
    n = x.numel()
    if fn == FN_DW_SPLIT:
        y = torch.empty((n, 2), dtype=torch.float32, device=x.device)
    elif fn in (FN_RCP32, FN_SQRT32):
        y = torch.empty(n, dtype=torch.float32, device=x.device)
    else:
        y = torch.empty(n, dtype=torch.float64, device=x.device)
    _check(_lib.m1_op_elementwise(fn, x.data_ptr(), n, y.data_ptr(), stream), "m1_op_elementwise")
    return y


def dw_split(x):
    """(hi, lo) float32 arrays of the double-word split the kernels apply to
    FP64 values, computed on the host by the same code (m1_dw_split)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    hi, lo = np.empty(x.shape, np.float32), np.empty(x.shape, np.float32)
    _check(_lib.m1_dw_split(x.ctypes.data, x.size, hi.ctypes.data, lo.ctypes.data), "m1_dw_split")
    return hi, lo


def f32_widen(x):
    """float64 copy of a float32 array by the kernels' widening (m1_f32_widen)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty(x.shape, np.float64)
    _check(_lib.m1_f32_widen(x.ctypes.data, x.size, y.ctypes.data), "m1_f32_widen")
    return y


class GridDesc3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("bc", ctypes.c_int * 6), ("c", ctypes.c_double), ("a_r", ctypes.c_double),
                ("c_v", ctypes.c_double)]


def make_desc3(nx, ny, nz, lx, ly, lz, bc=("periodic",) * 6, c=1.0, a_r=1.0, c_v=1.0):
    d = GridDesc3()
    d.nx, d.ny, d.nz, d.lx, d.ly, d.lz = nx, ny, nz, lx, ly, lz
    for k, b in enumerate(bc):
        d.bc[k] = BC[b]
    d.c, d.a_r, d.c_v = c, a_r, c_v
    return d


_lib.m1_op_level3.argtypes = [ctypes.POINTER(GridDesc3), ctypes.c_double, _vp, _vp, _vp,
                              ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _dp]
_lib.m1_create_grid3.argtypes = [ctypes.POINTER(GridDesc3), ctypes.c_int, _vp, ctypes.POINTER(_vp)]
_lib.m1_destroy_grid3.argtypes = [_vp]
_lib.m1_grid3_set_state.argtypes = [_vp, _vp, _vp, ctypes.c_int]
_lib.m1_grid3_set_inflow.argtypes = [_vp, _vp]
_lib.m1_grid3_get_state.argtypes = [_vp, _vp, ctypes.c_int]
_lib.m1_grid3_implicit_step.argtypes = [_vp, ctypes.c_double, ctypes.POINTER(SolveParams),
                                        ctypes.POINTER(StepStats)]
_lib.m1_grid3_step_history.argtypes = [_vp, _vp, _vp, ctypes.c_int]


def m1_op_level3(desc, dt, sig, state, rhs=None, mode=OP3_APPLY, sweeps=1, out=None,
                 on_device=False, stream=None):
    """3D single-level operators on planar [5][nz, ny, nx] states (host numpy
    arrays, or device tensors with on_device=True).  Returns (out, ms)."""
    n = desc.nx * desc.ny * desc.nz
    if not on_device:
        state = _host(state).reshape(5, n)
        sig = _host(sig).reshape(2, n)
        rhs = None if rhs is None else _host(rhs).reshape(5, n)
        out = np.zeros((5, n))
    ms = ctypes.c_double()
    st = _lib.m1_op_level3(ctypes.byref(desc), dt, _ptr(sig), _ptr(state), _ptr(rhs), mode, sweeps,
                           _ptr(out), int(on_device), stream, ctypes.byref(ms))
    _check(st, "m1_op_level3")
    if not on_device:
        out = out.reshape(5, desc.nz, desc.ny, desc.nx)
    return out, ms.value


class Grid3:
    """Owner of one m1_grid3_t: the implicit step in 3D (m1_create_grid3 ...)."""

    def __init__(self, desc: GridDesc3, lmax: int, stream=None):
        h = _vp()
        _check(_lib.m1_create_grid3(ctypes.byref(desc), lmax, stream, ctypes.byref(h)),
               "m1_create_grid3")
        self.h = h
        self.desc = desc
        self.lmax = lmax

    def close(self):
        if getattr(self, "h", None):
            _lib.m1_destroy_grid3(self.h)
            self.h = None

    __del__ = close

    @property
    def shape(self):
        return (5, self.desc.nz, self.desc.ny, self.desc.nx)

    def set_state(self, state, sig, on_device=False):
        """state: planar (5, nz, ny, nx) E, Fx, Fy, Fz, T; sig: (2, nz, ny, nx)."""
        if not on_device:
            state, sig = _host(state), _host(sig)
        return _check(_lib.m1_grid3_set_state(self.h, _ptr(state), _ptr(sig), int(on_device)),
                      "m1_grid3_set_state")

    def set_inflow(self, faces):
        """faces: (6 walls, 4 fields E, Fx, Fy, Fz, largest face) host array."""
        return _check(_lib.m1_grid3_set_inflow(self.h, _ptr(_host(faces))), "m1_grid3_set_inflow")

    def get_state(self, out=None, on_device=False):
        if out is None:
            out = np.zeros(self.shape)
        _check(_lib.m1_grid3_get_state(self.h, _ptr(out), int(on_device)), "m1_grid3_get_state")
        return out

    def implicit_step(self, dt, params: SolveParams | None = None, allow_not_converged=False):
        stats = StepStats()
        st = _lib.m1_grid3_implicit_step(self.h, dt, ctypes.byref(params) if params else None,
                                         ctypes.byref(stats))
        _check(st, "m1_grid3_implicit_step",
               allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return stats

    def step_history(self, length):
        hist = np.zeros(length)
        dtau = np.zeros(length)
        _check(_lib.m1_grid3_step_history(self.h, _ptr(hist), _ptr(dtau), length),
               "m1_grid3_step_history")
        return hist, dtau


def grid3_from_case(case, lmax=None, stream=None):
    """A Grid3 holding a 3D case of inputs.py (state, opacities and inflow set)."""
    d = case["desc"]
    g = Grid3(make_desc3(d["nx"], d["ny"], d["nz"], d["lx"], d["ly"], d["lz"], tuple(d["bc"]),
                         d["c"], d["a_r"], d["c_v"]),
              case["lmax"] if lmax is None else lmax, stream)
    g.set_state(case["state"], np.stack([case["sa"], case["ss"]]))
    if case.get("inflow") is not None:
        g.set_inflow(case["inflow"])
    return g


def m1_op_restrict(desc, state, resid, inflow=None):
    n = desc.nx * desc.ny
    nc = (desc.nx // 2) * (desc.ny // 2 if desc.dim == 2 else 1)
    state, resid = _host(state).reshape(4, n), _host(resid).reshape(4, n)
    cs, cr = np.zeros((4, nc)), np.zeros((4, nc))
    st = _lib.m1_op_restrict(ctypes.byref(desc), _ptr(_host(inflow)), _ptr(state), _ptr(resid),
                             _ptr(cs), _ptr(cr))
    _check(st, "m1_op_restrict")
    shp = (4, desc.ny // 2 if desc.dim == 2 else 1, desc.nx // 2)
    return cs.reshape(shp), cr.reshape(shp)


def m1_op_prolong_correct(desc, uc, vc, uf, theta=0.5):
    n = desc.nx * desc.ny
    uc, vc, uf = _host(uc).reshape(4, -1), _host(vc).reshape(4, -1), _host(uf).reshape(4, n)
    out = np.zeros((4, n))
    damped = ctypes.c_int()
    st = _lib.m1_op_prolong_correct(ctypes.byref(desc), _ptr(uc), _ptr(vc), _ptr(uf), theta,
                                    _ptr(out), ctypes.byref(damped))
    _check(st, "m1_op_prolong_correct")
    return out.reshape(4, desc.ny, desc.nx), damped.value
