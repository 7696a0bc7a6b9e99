"""Thin ctypes binding of libhj (include/hj.h): argument marshalling only.

Every function keeps the C name and returns what the C call writes to its
out-parameters; a status other than HJ_OK raises HjError with the library's
message.  All computation happens in the CUDA library; there is no Python
or CPU fallback: if libhj.so cannot be loaded, importing the binding raises.

Device arrays may be passed as PyTorch CUDA tensors (PyTorch is used only for
device memory and streams) or as raw integer device pointers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

HJ_OK, HJ_ERR_INVALID_ARG, HJ_ERR_STATE, HJ_ERR_OOM, HJ_ERR_CUDA, HJ_ERR_UNSTABLE, HJ_ERR_TIMEOUT, \
    HJ_ERR_UNSUPPORTED = range(8)
HJ_FP64, HJ_FP32, HJ_Q527 = 0, 1, 2  # HJ_Q527: int32 codes, value = code * 2^-27
HJ_DYN_CAR4D, HJ_DYN_CONST, HJ_DYN_CAR4D_STEER = 0, 1, 2
HJ_KERNEL_AUTO, HJ_KERNEL_GENERIC, HJ_KERNEL_TILED, HJ_KERNEL_RESIDENT = 0, 1, 2, 3
PERIODIC_THETA = 0b1000


class HjError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


class hj_solve_stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("total_steps", ctypes.c_int64),
        ("t_final", ctypes.c_double),
        ("dt_first", ctypes.c_double),
        ("dt_last", ctypes.c_double),
        ("alpha_max", ctypes.c_double * 4),
        ("device_ms", ctypes.c_double),
        ("loop_ms", ctypes.c_double),
        ("kernel", ctypes.c_int32),
        ("launches", ctypes.c_int32),
        ("last_change", ctypes.c_double),
        ("converged", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["alpha_max"] = list(self.alpha_max)
        return d


class hj_tile_result(ctypes.Structure):
    _fields_ = [
        ("shape", ctypes.c_int32 * 4),
        ("threads", ctypes.c_int32),
        ("ctas", ctypes.c_int32),
        ("ms_per_step", ctypes.c_double),
        ("ms_retimed", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {"shape": list(self.shape), "threads": self.threads, "ctas": self.ctas,
                "ms_per_step": self.ms_per_step, "ms_retimed": self.ms_retimed}


class hj_grid_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 4),
        ("pitch4", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("lo", ctypes.c_double * 4),
        ("hi", ctypes.c_double * 4),
        ("dx", ctypes.c_double * 4),
        ("periodic_mask", ctypes.c_uint32),
        ("has_value", ctypes.c_int32),
        ("total_steps", ctypes.c_int64),
        ("t", ctypes.c_double),
        ("device_bytes", ctypes.c_size_t),
        ("tile", ctypes.c_int32 * 4),
        ("tile_ctas", ctypes.c_int32),
        ("v0_broadcast", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        for k in ("n", "lo", "hi", "dx", "tile"):
            d[k] = list(d[k])
        return d


class hj_batch_stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("launches", ctypes.c_int64),
        ("active", ctypes.c_int32),
        ("finished", ctypes.c_int32),
        ("device_ms", ctypes.c_double),
        ("nconsumer", ctypes.c_int32),
        ("ctas", ctypes.c_int32),
        ("items", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class hj_batch_slot_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 4),
        ("steps", ctypes.c_int64),
        ("t", ctypes.c_double),
        ("T", ctypes.c_double),
        ("dt_last", ctypes.c_double),
        ("done", ctypes.c_int32),
        ("has_value", ctypes.c_int32),
        ("tile", ctypes.c_int32 * 3),
        ("device_bytes", ctypes.c_size_t),
    ]


class hj_request_info(ctypes.Structure):
    _fields_ = [
        ("state", ctypes.c_int32),
        ("slot", ctypes.c_int32),
        ("steps", ctypes.c_int64),
        ("t_submit", ctypes.c_double),
        ("t_admit", ctypes.c_double),
        ("t_done", ctypes.c_double),
    ]


# symbol -> (restype, argtypes); the exported C ABI
_VP = ctypes.c_void_p
_SIGS = {
    "hj_create_grid": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_uint32, ctypes.c_int, _VP,
                                      ctypes.POINTER(_VP)]),
    "hj_set_dynamics": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int32]),
    "hj_set_initial_value": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]),
    "hj_set_initial_value_device": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_size_t]),
    "hj_set_initial_value_xy_device": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_size_t]),
    "hj_set_initial_value_xy": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]),
    "hj_batch_set_initial_value_xy": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                                     ctypes.c_size_t]),
    "hj_server_submit_xy": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_int64)]),
    "hj_solve_brt": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.POINTER(hj_solve_stats)]),
    "hj_advance_brt": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                      ctypes.POINTER(hj_solve_stats)]),
    "hj_solve_converged": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                          ctypes.POINTER(hj_solve_stats)]),
    "hj_query": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP]),
    "hj_query_device": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP]),
    "hj_wait_selftest": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "hj_barrier_selftest": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "hj_fp64_fma_probe": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, _VP, ctypes.POINTER(ctypes.c_int64)]),
    "hj_read_value": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]),
    "hj_read_value_device": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_size_t]),
    "hj_set_kernel": (ctypes.c_int, [_VP, ctypes.c_int]),
    "hj_set_tile_shape": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32)]),
    "hj_autotune": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(hj_tile_result), ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_int32)]),
    "hj_step_noalloc": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_int32, _VP, _VP, _VP,
                                       ctypes.c_size_t, ctypes.c_double, _VP, ctypes.POINTER(ctypes.c_double)]),
    "hj_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(hj_grid_info)]),
    "hj_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "hj_batch_slot_bytes": (ctypes.c_size_t, [ctypes.POINTER(ctypes.c_int32)]),
    "hj_batch_add": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int32)]),
    "hj_batch_remove": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "hj_batch_set_initial_value": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                                  ctypes.c_size_t]),
    "hj_batch_set_initial_value_device": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int, ctypes.c_size_t]),
    "hj_batch_set_horizons": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "hj_batch_set_initial_values_device": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                                          ctypes.POINTER(_VP), ctypes.c_int,
                                                          ctypes.POINTER(ctypes.c_size_t)]),
    "hj_batch_set_horizon": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_double, ctypes.c_double]),
    "hj_batch_advance": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(hj_batch_stats)]),
    "hj_batch_get_slot_info": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(hj_batch_slot_info)]),
    "hj_batch_read_value": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]),
    "hj_batch_read_value_device": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int, ctypes.c_size_t]),
    "hj_batch_set_shape": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32]),
    "hj_batch_autotune": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]),
    "hj_batch_destroy": (None, [_VP]),
    "hj_server_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_size_t, ctypes.c_int32, _VP, ctypes.POINTER(_VP)]),
    "hj_server_submit": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_int64)]),
    "hj_server_tick": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "hj_server_request_info": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(hj_request_info)]),
    "hj_server_fetch": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]),
    "hj_server_fetch_device": (ctypes.c_int, [_VP, ctypes.c_int64, _VP, ctypes.c_int, ctypes.c_size_t]),
    "hj_server_clock": (ctypes.c_double, [_VP]),
    "hj_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "hj_server_destroy": (None, [_VP]),
    "hj_destroy_grid": (None, [_VP]),
    "hj_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "hj_last_error": (ctypes.c_char_p, []),
    "hj_version": (ctypes.c_int32, []),
}
SYMBOLS = tuple(_SIGS)


def _load() -> ctypes.CDLL:
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libhj.so is not built ({path}); run __graft_entry__.build() or "
                          f"python -m paper_2012_04011_gb300._build")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def status_name(s: int) -> str:
    return lib.hj_status_string(int(s)).decode()


def _check(status: int):
    if status != HJ_OK:
        raise HjError(status, lib.hj_last_error().decode())


def _dptr(x) -> int:
    """Device pointer of a torch CUDA tensor (or an int pointer)."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return int(x.data_ptr())
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _dtype_code(x) -> int:
    name = str(getattr(x, "dtype", ""))
    if name.endswith("float64"):
        return HJ_FP64
    if name.endswith("float32"):
        return HJ_FP32
    if name.endswith("int32"):
        return HJ_Q527
    raise TypeError(f"unsupported dtype {name}")


# ------------------------------------------------------------- C-named calls

def hj_version() -> int:
    return int(lib.hj_version())


def hj_create_grid(n, lo, hi, periodic_mask: int = PERIODIC_THETA, prec: int = HJ_FP32, cuda_stream=None):
    """Returns the opaque grid handle (an int)."""
    cn = (ctypes.c_int32 * 4)(*[int(v) for v in n])
    clo = (ctypes.c_double * 4)(*[float(v) for v in lo])
    chi = (ctypes.c_double * 4)(*[float(v) for v in hi])
    out = _VP()
    stream = None if cuda_stream is None else ctypes.c_void_p(int(cuda_stream))
    _check(lib.hj_create_grid(cn, clo, chi, int(periodic_mask), int(prec), stream, ctypes.byref(out)))
    return out.value


def hj_set_dynamics(g, kind: int, params):
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    _check(lib.hj_set_dynamics(g, int(kind), p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(p.size)))


def hj_set_initial_value(g, v0: np.ndarray):
    a = np.ascontiguousarray(v0, dtype=np.float64)
    _check(lib.hj_set_initial_value(g, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.size))


def hj_set_initial_value_xy(g, v0_xy: np.ndarray):
    a = np.ascontiguousarray(v0_xy, dtype=np.float64)
    _check(lib.hj_set_initial_value_xy(g, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.size))


def hj_set_initial_value_xy_device(g, v0_xy_device, count: int | None = None, dtype: int | None = None):
    cnt = int(v0_xy_device.numel()) if count is None else int(count)
    code = _dtype_code(v0_xy_device) if dtype is None else int(dtype)
    _check(lib.hj_set_initial_value_xy_device(g, ctypes.c_void_p(_dptr(v0_xy_device)), code, cnt))


def hj_set_initial_value_device(g, v0_device, count: int | None = None, dtype: int | None = None):
    cnt = int(v0_device.numel()) if count is None else int(count)
    code = _dtype_code(v0_device) if dtype is None else int(dtype)
    _check(lib.hj_set_initial_value_device(g, ctypes.c_void_p(_dptr(v0_device)), code, cnt))


def hj_solve_brt(g, T: float, cfl: float = 0.8) -> hj_solve_stats:
    st = hj_solve_stats()
    _check(lib.hj_solve_brt(g, float(T), float(cfl), ctypes.byref(st)))
    return st


def hj_advance_brt(g, T: float, cfl: float, max_steps: int) -> hj_solve_stats:
    st = hj_solve_stats()
    _check(lib.hj_advance_brt(g, float(T), float(cfl), int(max_steps), ctypes.byref(st)))
    return st


def hj_solve_converged(g, threshold: float, T_max: float, cfl: float = 0.8,
                       max_steps: int = (1 << 63) - 1) -> hj_solve_stats:
    st = hj_solve_stats()
    _check(lib.hj_solve_converged(g, float(threshold), float(T_max), float(cfl), int(max_steps), ctypes.byref(st)))
    return st


def hj_query(g, states, want_grad: bool = True, want_control: bool = True):
    """(value, grad or None, control or None) at host states (m x 4)."""
    st = np.ascontiguousarray(np.asarray(states, dtype=np.float64).reshape(-1, 4))
    m = st.shape[0]
    val = np.empty(m)
    grad = np.empty((m, 4)) if want_grad else None
    ctl = np.empty((m, 2)) if want_control else None
    p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    _check(lib.hj_query(g, p(st), m, p(val), p(grad), p(ctl)))
    return val, grad, ctl


def hj_query_device(g, states_device, value_device, grad_device=None, control_device=None):
    """Device arrays (float64 tensors or pointers): states m x 4, value m,
    grad m x 4, control m x 2."""
    m = int(states_device.numel()) // 4 if hasattr(states_device, "numel") else int(value_device.numel())
    q = lambda a: None if a is None else ctypes.c_void_p(_dptr(a))
    _check(lib.hj_query_device(g, q(states_device), m, q(value_device), q(grad_device), q(control_device)))


def hj_wait_selftest(limit_ns: int):
    """(status, waited_ns) of the bounded-wait self-test."""
    st = ctypes.c_int32(0)
    waited = ctypes.c_int64(0)
    _check(lib.hj_wait_selftest(int(limit_ns), ctypes.byref(st), ctypes.byref(waited)))
    return int(st.value), int(waited.value)


def hj_fp64_fma_probe(iters: int, blocks_per_sm: int = 8, cuda_stream=None) -> int:
    """Launches the FP64 FMA throughput probe on cuda_stream; returns the FMAs issued."""
    n = ctypes.c_int64(0)
    stream = None if cuda_stream is None else ctypes.c_void_p(int(cuda_stream))
    _check(lib.hj_fp64_fma_probe(int(iters), int(blocks_per_sm), stream, ctypes.byref(n)))
    return int(n.value)


def hj_barrier_selftest(limit_ns: int):
    """(status, waited_ns) of the bounded grid-barrier self-test."""
    st = ctypes.c_int32(0)
    waited = ctypes.c_int64(0)
    _check(lib.hj_barrier_selftest(int(limit_ns), ctypes.byref(st), ctypes.byref(waited)))
    return int(st.value), int(waited.value)


def hj_read_value(g, out: np.ndarray | None = None, shape=None) -> np.ndarray:
    info = hj_get_info(g)
    n = tuple(info.n)
    if out is None:
        out = np.empty(n if shape is None else shape, dtype=np.float64)
    if out.dtype != np.float64 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float64 array")
    _check(lib.hj_read_value(g, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size))
    return out


def hj_read_value_device(g, out_device, count: int | None = None, dtype: int | None = None):
    cnt = int(out_device.numel()) if count is None else int(count)
    code = _dtype_code(out_device) if dtype is None else int(dtype)
    _check(lib.hj_read_value_device(g, ctypes.c_void_p(_dptr(out_device)), code, cnt))
    return out_device


def hj_set_kernel(g, kernel: int):
    _check(lib.hj_set_kernel(g, int(kernel)))


def hj_set_tile_shape(g, shape):
    arr = (ctypes.c_int32 * 4)(*[int(v) for v in shape])
    _check(lib.hj_set_tile_shape(g, arr))


def hj_autotune(g, steps_per_trial: int = 8, max_results: int = 32):
    """Returns the list of tried shapes (hj_tile_result) in the order tried."""
    res = (hj_tile_result * max_results)()
    cnt = ctypes.c_int32(0)
    _check(lib.hj_autotune(g, int(steps_per_trial), res, int(max_results), ctypes.byref(cnt)))
    return [res[i] for i in range(min(cnt.value, max_results))]


def hj_step_noalloc(n, lo, hi, periodic_mask, prec, kind, params, v_in, v0, v_out, dt, cuda_stream=None,
                    want_alpha: bool = True):
    """One step on caller-owned device arrays without any allocation; returns
    alpha^max (4 values), or None when want_alpha is false (the C call then
    gets a NULL alpha_max_out).  v_in, v0 and v_out are contiguous device
    tensors of the precision's element type (float64 for HJ_FP64, float32 for
    HJ_FP32) with N1*N2*N3*N4 elements each; v_out may overlap neither
    input."""
    import torch
    want = torch.float64 if int(prec) == HJ_FP64 else torch.float32
    ncell = int(np.prod([int(v) for v in n], dtype=np.int64))
    for name, t in (("v_in", v_in), ("v0", v0), ("v_out", v_out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if t.dtype != want:
            raise ValueError(f"{name} has dtype {t.dtype}, the precision needs {want}")
        if t.numel() != ncell:
            raise ValueError(f"{name} has {t.numel()} elements, the grid has {ncell}")
    nbytes = ncell * (8 if want == torch.float64 else 4)
    o0 = v_out.data_ptr()
    for name, t in (("v_in", v_in), ("v0", v0)):
        if t.data_ptr() < o0 + nbytes and o0 < t.data_ptr() + nbytes:
            raise ValueError(f"v_out overlaps {name}")
    cn = (ctypes.c_int32 * 4)(*[int(v) for v in n])
    clo = (ctypes.c_double * 4)(*[float(v) for v in lo])
    chi = (ctypes.c_double * 4)(*[float(v) for v in hi])
    p = (ctypes.c_double * len(params))(*[float(v) for v in params])
    alpha = (ctypes.c_double * 4)()
    stream = None if cuda_stream is None else ctypes.c_void_p(int(cuda_stream))
    _check(lib.hj_step_noalloc(cn, clo, chi, int(periodic_mask), int(prec), int(kind), p, len(params),
                               ctypes.c_void_p(_dptr(v_in)), ctypes.c_void_p(_dptr(v0)), ctypes.c_void_p(_dptr(v_out)),
                               nbytes, float(dt), stream, alpha if want_alpha else None))
    return list(alpha) if want_alpha else None


def hj_get_info(g) -> hj_grid_info:
    info = hj_grid_info()
    _check(lib.hj_get_info(g, ctypes.byref(info)))
    return info


def hj_destroy_grid(g):
    lib.hj_destroy_grid(g)


# ------------------------------------------------------------- convenience

class Grid:
    """Owns one hj_grid; the methods are the C calls above."""

    def __init__(self, n, lo, hi, periodic_mask=PERIODIC_THETA, prec=HJ_FP32, cuda_stream=None):
        self.n = tuple(int(v) for v in n)
        self.handle = hj_create_grid(n, lo, hi, periodic_mask, prec, cuda_stream)

    @classmethod
    def for_workload(cls, w, prec=HJ_FP32, cuda_stream=None):
        g = cls(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, prec, cuda_stream)
        g.set_dynamics(HJ_DYN_CAR4D, (w.a_max, w.w_max))
        return g

    def set_dynamics(self, kind, params):
        hj_set_dynamics(self.handle, kind, params)

    def set_initial_value_xy(self, v0_xy):
        hj_set_initial_value_xy(self.handle, v0_xy)

    def set_initial_value(self, v0):
        if hasattr(v0, "is_cuda") and v0.is_cuda:
            hj_set_initial_value_device(self.handle, v0)
        else:
            hj_set_initial_value(self.handle, np.asarray(v0))

    def solve_brt(self, T, cfl=0.8) -> hj_solve_stats:
        return hj_solve_brt(self.handle, T, cfl)

    def solve_converged(self, threshold, T_max, cfl=0.8, max_steps=(1 << 63) - 1) -> hj_solve_stats:
        return hj_solve_converged(self.handle, threshold, T_max, cfl, max_steps)

    def advance_brt(self, T, cfl, max_steps) -> hj_solve_stats:
        return hj_advance_brt(self.handle, T, cfl, max_steps)

    def read_value(self, out=None) -> np.ndarray:
        return hj_read_value(self.handle, out)

    def read_value_device(self, out):
        return hj_read_value_device(self.handle, out)

    def set_kernel(self, kernel):
        hj_set_kernel(self.handle, kernel)

    def set_tile_shape(self, shape):
        hj_set_tile_shape(self.handle, shape)

    def autotune(self, steps_per_trial=8):
        return hj_autotune(self.handle, steps_per_trial)

    def info(self) -> hj_grid_info:
        return hj_get_info(self.handle)

    def close(self):
        if self.handle:
            hj_destroy_grid(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- batches

def hj_batch_create(max_slots: int, memory_budget: int = 0, cuda_stream=None):
    out = _VP()
    stream = None if cuda_stream is None else ctypes.c_void_p(int(cuda_stream))
    _check(lib.hj_batch_create(int(max_slots), int(memory_budget), stream, ctypes.byref(out)))
    return out.value


def hj_batch_slot_bytes(n) -> int:
    return int(lib.hj_batch_slot_bytes((ctypes.c_int32 * 4)(*[int(v) for v in n])))


def hj_batch_add(b, n, lo, hi, params) -> int:
    slot = ctypes.c_int32(-1)
    _check(lib.hj_batch_add(b, (ctypes.c_int32 * 4)(*[int(v) for v in n]), (ctypes.c_double * 4)(*[float(v) for v in lo]),
                            (ctypes.c_double * 4)(*[float(v) for v in hi]),
                            (ctypes.c_double * 2)(*[float(v) for v in params]), ctypes.byref(slot)))
    return slot.value


def hj_batch_remove(b, slot: int):
    _check(lib.hj_batch_remove(b, int(slot)))


def hj_batch_set_initial_value(b, slot: int, v0):
    if hasattr(v0, "is_cuda") and v0.is_cuda:
        _check(lib.hj_batch_set_initial_value_device(b, int(slot), ctypes.c_void_p(_dptr(v0)), _dtype_code(v0),
                                                     int(v0.numel())))
    else:
        a = np.ascontiguousarray(v0, dtype=np.float64)
        _check(lib.hj_batch_set_initial_value(b, int(slot), a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.size))


def hj_batch_set_initial_values_device(b, slots, v0s):
    """V0 of several slots from CUDA tensors of one dtype (float32 or float64),
    with one synchronisation for all of them."""
    n = len(slots)
    if n != len(v0s):
        raise ValueError("one V0 tensor per slot")
    if n == 0:
        return
    dtypes = {_dtype_code(v) for v in v0s}
    if len(dtypes) != 1 or HJ_Q527 in dtypes:
        raise ValueError("the V0 tensors must all be float32 or all float64")
    cs = (ctypes.c_int32 * n)(*[int(s) for s in slots])
    ps = (_VP * n)(*[_dptr(v) for v in v0s])
    cnt = (ctypes.c_size_t * n)(*[int(v.numel()) for v in v0s])
    _check(lib.hj_batch_set_initial_values_device(b, n, cs, ps, dtypes.pop(), cnt))


def hj_batch_set_horizons(b, slots, T, cfl):
    """Horizons and Courant numbers of several slots in one call."""
    n = len(slots)
    if not (n == len(T) == len(cfl)):
        raise ValueError("one T and one cfl per slot")
    if n == 0:
        return
    _check(lib.hj_batch_set_horizons(b, n, (ctypes.c_int32 * n)(*[int(s) for s in slots]),
                                     (ctypes.c_double * n)(*[float(t) for t in T]),
                                     (ctypes.c_double * n)(*[float(c) for c in cfl])))


def hj_batch_set_initial_value_xy(b, slot: int, v0_xy):
    a = np.ascontiguousarray(v0_xy, dtype=np.float64)
    _check(lib.hj_batch_set_initial_value_xy(b, int(slot), a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.size))


def hj_batch_set_horizon(b, slot: int, T: float, cfl: float = 0.8):
    _check(lib.hj_batch_set_horizon(b, int(slot), float(T), float(cfl)))


def hj_batch_advance(b, max_steps: int = 1 << 40) -> hj_batch_stats:
    st = hj_batch_stats()
    _check(lib.hj_batch_advance(b, int(max_steps), ctypes.byref(st)))
    return st


def hj_batch_get_slot_info(b, slot: int) -> hj_batch_slot_info:
    info = hj_batch_slot_info()
    _check(lib.hj_batch_get_slot_info(b, int(slot), ctypes.byref(info)))
    return info


def hj_batch_read_value(b, slot: int, out=None) -> np.ndarray:
    info = hj_batch_get_slot_info(b, slot)
    if out is None:
        out = np.empty(tuple(info.n), dtype=np.float64)
    if hasattr(out, "is_cuda") and out.is_cuda:
        _check(lib.hj_batch_read_value_device(b, int(slot), ctypes.c_void_p(_dptr(out)), _dtype_code(out),
                                              int(out.numel())))
        return out
    _check(lib.hj_batch_read_value(b, int(slot), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size))
    return out


def hj_batch_set_shape(b, nconsumer: int = 0, chunks: int = 0):
    _check(lib.hj_batch_set_shape(b, int(nconsumer), int(chunks)))


def hj_batch_autotune(b, steps_per_trial: int = 4):
    nc, ch, ms = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0)
    _check(lib.hj_batch_autotune(b, int(steps_per_trial), ctypes.byref(nc), ctypes.byref(ch), ctypes.byref(ms)))
    return nc.value, ch.value, ms.value


def hj_batch_destroy(b):
    lib.hj_batch_destroy(b)


class Batch:
    """Owns one hj_batch; the methods are the C calls above."""

    def __init__(self, max_slots, memory_budget=0, cuda_stream=None):
        self.handle = hj_batch_create(max_slots, memory_budget, cuda_stream)

    def add(self, n, lo, hi, params):
        return hj_batch_add(self.handle, n, lo, hi, params)

    def add_workload(self, w):
        return self.add(w.grid.n, w.grid.lo, w.grid.hi, (w.a_max, w.w_max))

    def remove(self, slot):
        hj_batch_remove(self.handle, slot)

    def set_initial_value(self, slot, v0):
        hj_batch_set_initial_value(self.handle, slot, v0)

    def set_initial_values(self, slots, v0s):
        hj_batch_set_initial_values_device(self.handle, slots, v0s)

    def set_horizons(self, slots, T, cfl):
        hj_batch_set_horizons(self.handle, slots, T, cfl)

    def set_initial_value_xy(self, slot, v0_xy):
        hj_batch_set_initial_value_xy(self.handle, slot, v0_xy)

    def set_horizon(self, slot, T, cfl=0.8):
        hj_batch_set_horizon(self.handle, slot, T, cfl)

    def advance(self, max_steps=1 << 40):
        return hj_batch_advance(self.handle, max_steps)

    def slot_info(self, slot):
        return hj_batch_get_slot_info(self.handle, slot)

    def read_value(self, slot, out=None):
        return hj_batch_read_value(self.handle, slot, out)

    def set_shape(self, nconsumer=0, chunks=0):
        hj_batch_set_shape(self.handle, nconsumer, chunks)

    def autotune(self, steps_per_trial=4):
        return hj_batch_autotune(self.handle, steps_per_trial)

    def close(self):
        if self.handle:
            hj_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- re-solve server

REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = range(4)


class Server:
    """Owns one hj_server (continuous batching of BRT re-solve requests)."""

    def __init__(self, max_slots=64, memory_budget=0, steps_per_tick=32, cuda_stream=None):
        out = _VP()
        stream = None if cuda_stream is None else ctypes.c_void_p(int(cuda_stream))
        _check(lib.hj_server_create(int(max_slots), int(memory_budget), int(steps_per_tick), stream,
                                    ctypes.byref(out)))
        self.handle = out.value

    def submit(self, n, lo, hi, params, v0, T, cfl=0.8) -> int:
        a = np.ascontiguousarray(v0, dtype=np.float64)
        rid = ctypes.c_int64(0)
        _check(lib.hj_server_submit(self.handle, (ctypes.c_int32 * 4)(*[int(v) for v in n]),
                                    (ctypes.c_double * 4)(*[float(v) for v in lo]),
                                    (ctypes.c_double * 4)(*[float(v) for v in hi]),
                                    (ctypes.c_double * 2)(*[float(v) for v in params]),
                                    a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(T), float(cfl),
                                    ctypes.byref(rid)))
        return rid.value

    def submit_xy(self, n, lo, hi, params, v0_xy, T, cfl=0.8) -> int:
        a = np.ascontiguousarray(v0_xy, dtype=np.float64)
        rid = ctypes.c_int64(0)
        _check(lib.hj_server_submit_xy(self.handle, (ctypes.c_int32 * 4)(*[int(v) for v in n]),
                                       (ctypes.c_double * 4)(*[float(v) for v in lo]),
                                       (ctypes.c_double * 4)(*[float(v) for v in hi]),
                                       (ctypes.c_double * 2)(*[float(v) for v in params]),
                                       a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(T), float(cfl),
                                       ctypes.byref(rid)))
        return rid.value

    def submit_workload(self, w, v0) -> int:
        return self.submit(w.grid.n, w.grid.lo, w.grid.hi, (w.a_max, w.w_max), v0, w.T, w.cfl)

    def tick(self):
        c, r, q = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        _check(lib.hj_server_tick(self.handle, ctypes.byref(c), ctypes.byref(r), ctypes.byref(q)))
        return c.value, r.value, q.value

    def info(self, rid) -> hj_request_info:
        info = hj_request_info()
        _check(lib.hj_server_request_info(self.handle, int(rid), ctypes.byref(info)))
        return info

    def fetch(self, rid, shape):
        out = np.empty(shape, dtype=np.float64)
        _check(lib.hj_server_fetch(self.handle, int(rid), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   out.size))
        return out

    def fetch_device(self, rid, out):
        _check(lib.hj_server_fetch_device(self.handle, int(rid), ctypes.c_void_p(_dptr(out)), _dtype_code(out),
                                          int(out.numel())))
        return out

    def clock(self) -> float:
        return float(lib.hj_server_clock(self.handle))

    def stats(self):
        t, s = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib.hj_server_stats(self.handle, ctypes.byref(t), ctypes.byref(s)))
        return t.value, s.value

    def close(self):
        if self.handle:
            lib.hj_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
