"""FP64 CPU oracle for the 4D HJ reachability scheme of arxiv 2012.04011.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never imports it, links it or calls it, and the two share no code:
the oracle builds its own grid, tables and time loop from the paper
(Eq. central_diff, Algorithms 1-2 of Sec. II-B, the car of Sec. IV-A).

The arithmetic lives in ``hj_oracle.c`` (plain scalar C, FP64, no FMA
contraction, optional OpenMP over the slowest axis with bit-identical
results).  This module only compiles it with gcc and marshals numpy arrays
through ctypes.

Parity status of each entry point (how it is pinned) is listed in the tests
``tests/test_oracle_pins.py`` (FP64 scheme) and
``tests/test_oracle_q527_pins.py`` (Q5.27 fixed-point variant of Sec. III-C /
Sec. IV-B); every function here is pinned by at least one closed form,
invariant, textbook special case or paper number.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hj_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libhj_oracle.so")

DYN_CAR4D = 0  # params (a_max, w_max): x'=v cos th, y'=v sin th, v'=a, th'=w
DYN_CONST = 1  # params (c1, c2, c3, c4): xdot = c, no control
DYN_CAR4D_STEER = 2  # params (a_max, delta_max, L): th' = v tan(delta) / L (Eq. car_dynamics)

_lock = threading.Lock()
_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 4),
        ("lo", ctypes.c_double * 4),
        ("hi", ctypes.c_double * 4),
        ("periodic", ctypes.c_uint32),
        ("dyn", ctypes.c_int32),
        ("p", ctypes.c_double * 4),
    ]


def build(force: bool = False) -> str:
    """Compile hj_oracle.c into a shared library (gcc, -O2, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.hjo_spacing.argtypes = [P, ctypes.c_int]
        lib.hjo_spacing.restype = ctypes.c_double
        lib.hjo_coord.argtypes = [P, ctypes.c_int, ctypes.c_int]
        lib.hjo_coord.restype = ctypes.c_double
        lib.hjo_cfl_dt.argtypes = [P, dp, ctypes.c_double]
        lib.hjo_cfl_dt.restype = ctypes.c_double
        lib.hjo_rate.argtypes = [P, dp, dp, dp, ctypes.c_int]
        lib.hjo_rate.restype = ctypes.c_int
        lib.hjo_step_cells.argtypes = [P, dp, dp, ctypes.c_double, i64p, ctypes.c_int64, dp]
        lib.hjo_step_cells.restype = ctypes.c_int
        lib.hjo_advance.argtypes = [P, dp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                    dp, ctypes.c_int]
        lib.hjo_advance.restype = ctypes.c_int64
        lib.hjo_advance_converged.argtypes = [P, dp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int64, dp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int)]
        lib.hjo_advance_converged.restype = ctypes.c_int64
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.hjo_to_q527.argtypes = [dp, ctypes.c_int64, i32p]
        lib.hjo_to_q527.restype = ctypes.c_int
        lib.hjo_from_q527.argtypes = [i32p, ctypes.c_int64, dp]
        lib.hjo_from_q527.restype = None
        lib.hjo_advance_q527.argtypes = [P, i32p, i32p, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                         dp, ctypes.c_int]
        lib.hjo_advance_q527.restype = ctypes.c_int64
        lib.hjo_advance_converged_q527.argtypes = [P, i32p, i32p, dp, ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_double, ctypes.c_int64, dp, ctypes.c_int, dp,
                                                   ctypes.POINTER(ctypes.c_int)]
        lib.hjo_advance_converged_q527.restype = ctypes.c_int64
        lib.hjo_step_cells_q527.argtypes = [P, i32p, i32p, ctypes.c_double, i64p, ctypes.c_int64, i32p]
        lib.hjo_step_cells_q527.restype = ctypes.c_int
        lib.hjo_query.argtypes = [P, dp, dp, ctypes.c_int64, dp, dp, dp]
        lib.hjo_query.restype = ctypes.c_int
        lib.hjo_max_threads.argtypes = []
        lib.hjo_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


class Problem:
    """Grid + dynamics description handed to the oracle.

    n: points per axis (x, y, v, theta), theta fastest in memory.
    lo, hi: axis bounds.  periodic: bit d set for a periodic axis.
    dyn: DYN_CAR4D with params (a_max, w_max) or DYN_CONST with (c1..c4).
    """

    def __init__(self, n, lo, hi, periodic=0b1000, dyn=DYN_CAR4D, params=(1.5, 1.0)):
        self.n = tuple(int(x) for x in n)
        self.lo = tuple(float(x) for x in lo)
        self.hi = tuple(float(x) for x in hi)
        self.periodic = int(periodic)
        self.dyn = int(dyn)
        p = list(float(x) for x in params) + [0.0] * (4 - len(params))
        self.params = tuple(p[:4])
        s = _Problem()
        for d in range(4):
            s.n[d] = self.n[d]
            s.lo[d] = self.lo[d]
            s.hi[d] = self.hi[d]
            s.p[d] = self.params[d]
        s.periodic = self.periodic
        s.dyn = self.dyn
        self._s = s

    @property
    def shape(self):
        return self.n

    @property
    def ncell(self):
        return int(np.prod(self.n))

    def spacing(self, d: int) -> float:
        return _load().hjo_spacing(ctypes.byref(self._s), d)

    def coord(self, d: int, i: int) -> float:
        return _load().hjo_coord(ctypes.byref(self._s), d, i)

    def coords(self, d: int) -> np.ndarray:
        return np.array([self.coord(d, i) for i in range(self.n[d])])


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_grid(P: Problem, a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.size != P.ncell:
        raise ValueError(f"array has {a.size} values, grid has {P.ncell}")
    return a.reshape(P.n)


def max_threads() -> int:
    return int(_load().hjo_max_threads())


def rate(P: Problem, V, nthreads: int = 1):
    """L = H + dissipation per cell and alpha_d^max (Alg. 1 sweeps 1-2)."""
    V = _as_grid(P, V)
    L = np.empty_like(V)
    am = np.zeros(4)
    rc = _load().hjo_rate(ctypes.byref(P._s), _dptr(V), _dptr(L), _dptr(am), int(nthreads))
    if rc:
        raise MemoryError("oracle allocation failed")
    return L, am


def cfl_dt(P: Problem, alpha_max, cfl: float) -> float:
    """dt = CFL / sum_d alpha_d^max / dx_d (0.0 when nothing moves)."""
    am = np.ascontiguousarray(np.asarray(alpha_max, dtype=np.float64))
    return float(_load().hjo_cfl_dt(ctypes.byref(P._s), _dptr(am), float(cfl)))


def step_cells(P: Problem, V, V0, dt: float, cells) -> np.ndarray:
    """One Euler step + BRT min of size dt, evaluated only at flat cell indices."""
    V = _as_grid(P, V)
    V0 = _as_grid(P, V0)
    cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
    out = np.empty(cells.size)
    rc = _load().hjo_step_cells(ctypes.byref(P._s), _dptr(V), _dptr(V0), float(dt),
                                cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                cells.size, _dptr(out))
    if rc:
        raise MemoryError("oracle allocation failed")
    return out


def advance(P: Problem, V0, V, t: float, T: float, cfl: float = 0.8, max_steps: int = 1 << 40,
            nthreads: int = 1):
    """Advance V from time t toward T (at most max_steps steps).

    Returns (V_new, t_new, dts) with dts the step sizes taken.
    """
    V0 = _as_grid(P, V0)
    Vw = _as_grid(P, V).copy()
    cap = int(min(max_steps, 1 << 20))
    dts = np.zeros(cap)
    tt = ctypes.c_double(float(t))
    steps = _load().hjo_advance(ctypes.byref(P._s), _dptr(V0), _dptr(Vw), ctypes.byref(tt), float(T),
                                float(cfl), cap, _dptr(dts), int(nthreads))
    if steps < 0:
        raise MemoryError("oracle allocation failed")
    return Vw, float(tt.value), dts[:steps].copy()


def advance_converged(P: Problem, V0, V, t: float, threshold: float, T: float, cfl: float = 0.8,
                      max_steps: int = 1 << 40, nthreads: int = 1):
    """Step from (V, t) until a step changes V by less than threshold in the
    max norm (Algorithm 2's convergence test), or t reaches T, or max_steps.
    Returns (V_new, t_new, dts, eps_last, converged)."""
    V0 = _as_grid(P, V0)
    Vw = _as_grid(P, V).copy()
    cap = int(min(max_steps, 1 << 20))
    dts = np.zeros(cap)
    tt = ctypes.c_double(float(t))
    eps = ctypes.c_double(0.0)
    conv = ctypes.c_int(0)
    steps = _load().hjo_advance_converged(ctypes.byref(P._s), _dptr(V0), _dptr(Vw), ctypes.byref(tt), float(T),
                                          float(cfl), float(threshold), cap, _dptr(dts), int(nthreads),
                                          ctypes.byref(eps), ctypes.byref(conv))
    if steps < 0:
        raise MemoryError("oracle allocation failed")
    return Vw, float(tt.value), dts[:steps].copy(), float(eps.value), bool(conv.value)


def query(P: Problem, V, states):
    """V, grad V (4 per state) and u_opt (2 per state: a and the heading
    control) at states (m x 4: x, y, v, theta) by multilinear interpolation
    (Eq. uopt_max; the readings are listed in hj_oracle.c)."""
    V = _as_grid(P, V)
    st = np.ascontiguousarray(np.asarray(states, dtype=np.float64).reshape(-1, 4))
    m = st.shape[0]
    val = np.empty(m)
    grad = np.empty((m, 4))
    ctl = np.empty((m, 2))
    _load().hjo_query(ctypes.byref(P._s), _dptr(V), _dptr(st), m, _dptr(val), _dptr(grad), _dptr(ctl))
    return val, grad, ctl


def solve(P: Problem, V0, T: float, cfl: float = 0.8, nthreads: int = 1, max_steps: int = 1 << 40):
    """Whole BRT solve from t = 0 to T.  Returns (V(T), dts)."""
    V, _, dts = advance(P, V0, V0, 0.0, T, cfl, max_steps, nthreads)
    return V, dts


# ---------------------------------------------------------------- Q5.27 fixed point
# Sec. III-C / Sec. IV-B: V as 32-bit fixed point, 5 integer bits (sign
# included) and 27 fractional bits.  The readings of the arithmetic are listed
# in hj_oracle.c ("Q5.27 fixed-point variant").

Q527_ULP = 2.0 ** -27


def _ipt(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def to_q527(x) -> np.ndarray:
    """int32 codes of x: nearest (ties to even), saturated to the int32 range."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    q = np.empty(x.shape, dtype=np.int32)
    if _load().hjo_to_q527(_dptr(x), x.size, _ipt(q)):
        raise ValueError("NaN or Inf cannot be converted to Q5.27")
    return q


def from_q527(q) -> np.ndarray:
    """Exact FP64 values q * 2^-27."""
    q = np.ascontiguousarray(np.asarray(q, dtype=np.int32))
    x = np.empty(q.shape, dtype=np.float64)
    _load().hjo_from_q527(_ipt(q), q.size, _dptr(x))
    return x


def _as_qgrid(P: Problem, a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    if a.size != P.ncell:
        raise ValueError(f"array has {a.size} values, grid has {P.ncell}")
    return a.reshape(P.n)


def advance_q527(P: Problem, Q0, Q, t: float, T: float, cfl: float = 0.8, max_steps: int = 1 << 40,
                 nthreads: int = 1):
    """Fixed-point advance of the int32 grid Q from t toward T.  Returns
    (Q_new, t_new, dts)."""
    Q0 = _as_qgrid(P, Q0)
    Qw = _as_qgrid(P, Q).copy()
    cap = int(min(max_steps, 1 << 20))
    dts = np.zeros(cap)
    tt = ctypes.c_double(float(t))
    steps = _load().hjo_advance_q527(ctypes.byref(P._s), _ipt(Q0), _ipt(Qw), ctypes.byref(tt), float(T),
                                     float(cfl), cap, _dptr(dts), int(nthreads))
    if steps < 0:
        raise MemoryError("oracle allocation failed")
    return Qw, float(tt.value), dts[:steps].copy()


def solve_q527(P: Problem, V0, T: float, cfl: float = 0.8, nthreads: int = 1, max_steps: int = 1 << 40):
    """Fixed-point BRT solve from the FP64 V0 (converted to Q5.27) to T.
    Returns (Q(T) as int32 codes, dts)."""
    Q0 = to_q527(V0)
    Q, _, dts = advance_q527(P, Q0, Q0, 0.0, T, cfl, max_steps, nthreads)
    return Q, dts


def step_cells_q527(P: Problem, Q, Q0, dt: float, cells) -> np.ndarray:
    """One fixed-point step of size dt at flat cell indices."""
    Q = _as_qgrid(P, Q)
    Q0 = _as_qgrid(P, Q0)
    cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
    out = np.empty(cells.size, dtype=np.int32)
    rc = _load().hjo_step_cells_q527(ctypes.byref(P._s), _ipt(Q), _ipt(Q0), float(dt),
                                     cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cells.size, _ipt(out))
    if rc:
        raise MemoryError("oracle allocation failed")
    return out


def advance_converged_q527(P: Problem, Q0, Q, t: float, threshold: float, T: float, cfl: float = 0.8,
                           max_steps: int = 1 << 40, nthreads: int = 1):
    """advance_converged on the Q5.27 grid.  Returns (Q_new, t_new, dts,
    eps_last, converged)."""
    Q0 = _as_qgrid(P, Q0)
    Qw = _as_qgrid(P, Q).copy()
    cap = int(min(max_steps, 1 << 20))
    dts = np.zeros(cap)
    tt = ctypes.c_double(float(t))
    eps = ctypes.c_double(0.0)
    conv = ctypes.c_int(0)
    steps = _load().hjo_advance_converged_q527(ctypes.byref(P._s), _ipt(Q0), _ipt(Qw), ctypes.byref(tt), float(T),
                                               float(cfl), float(threshold), cap, _dptr(dts), int(nthreads),
                                               ctypes.byref(eps), ctypes.byref(conv))
    if steps < 0:
        raise MemoryError("oracle allocation failed")
    return Qw, float(tt.value), dts[:steps].copy(), float(eps.value), bool(conv.value)
