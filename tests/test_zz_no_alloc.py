"""hj_step_noalloc: the entry point for callers that cannot allocate device
memory (their device memory belongs to a host framework's pool, a budget
fixed at start-up, or a moment where cudaMalloc must not synchronise the
device).  It steps caller-owned arrays and keeps its working data in a fixed
device array, so it must give the step the oracle gives.

Each call is checked against the FP64 oracle's step of the same V_n with the
same dt at every cell (oracle.step_cells), and against the grid API's step,
on two calls in a row: FP64 within 1e-12, FP32 within 8 FP32 epsilons of
max|V0| for one step (the tolerance of the sampled one-step parity tests).
Cases: the car on the small grid; the car on the paper's 60x60x20x36 grid
(more cells than threads, so every thread updates several); constant
dynamics with negative v and theta velocities and periodic x and y axes;
alpha_max_out = NULL.  The file name makes pytest collect it last.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2012_04011_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hj():
    from paper_2012_04011_gb300 import _build
    _build.build()
    from paper_2012_04011_gb300 import hj as mod
    return mod


def one_step_tol(prec, V0):
    return 1e-12 if prec == "fp64" else 8 * float(np.finfo(np.float32).eps) * float(np.abs(V0).max())


def run_two_calls(hj, n, lo, hi, periodic, prec, kind, params, okind, V0, dt, alpha_on_second=True):
    """Two hj_step_noalloc calls in a row from V0, each checked against the
    oracle's step of the same input and the grid API's step of size dt."""
    import torch
    p = hj.HJ_FP64 if prec == "fp64" else hj.HJ_FP32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    tol = one_step_tol(prec, V0)
    P = oracle.Problem(n, lo, hi, periodic, okind, params)
    cells = np.arange(int(np.prod(n)), dtype=np.int64)
    v0_dev = torch.from_numpy(V0).to("cuda", tdt).reshape(-1)
    V0s = v0_dev.double().cpu().numpy().reshape(n)  # V0 as stored in the precision
    outs = (torch.empty_like(v0_dev), torch.empty_like(v0_dev))
    ref = torch.empty_like(v0_dev)
    stream = torch.cuda.current_stream().cuda_stream
    with hj.Grid(n, lo, hi, periodic, p) as g:
        g.set_dynamics(kind, params)
        g.set_initial_value(v0_dev)
        src = v0_dev
        for call, out in enumerate(outs, start=1):
            want_alpha = call == 1 or alpha_on_second
            alpha = hj.hj_step_noalloc(n, lo, hi, periodic, p, kind, params, src, v0_dev, out, dt, stream,
                                       want_alpha=want_alpha)
            Vin = src.double().cpu().numpy().reshape(n)
            got = out.double().cpu().numpy().reshape(n)
            want = oracle.step_cells(P, Vin, V0s, dt, cells).reshape(n)
            err = float(np.abs(got - want).max())
            assert err <= tol, ("oracle", call, err)
            st = g.advance_brt(call * dt, 0.8, 1)
            assert st.steps == 1 and st.dt_last == dt
            g.read_value_device(ref)
            err = float((out.double() - ref.double()).abs().max())
            assert err <= tol, ("grid API", call, err)
            if want_alpha:
                _, am = oracle.rate(P, Vin)
                assert alpha[0] == pytest.approx(am[0], rel=1e-14, abs=1e-300)
                assert alpha[1] == pytest.approx(am[1], rel=1e-14, abs=1e-300)
                assert alpha[2] == am[2] and alpha[3] == am[3]
            else:
                assert alpha is None
            src = out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_car_two_calls(hj, prec):
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    # dt below the CFL step (0.0264), so the grid API takes exactly this step
    run_two_calls(hj, w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, prec, hj.HJ_DYN_CAR4D,
                  (w.a_max, w.w_max), oracle.DYN_CAR4D, V0, 0.01)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_car_grid_stride(hj, prec):
    """2,592,000 cells, several per thread of the capped launch; the second
    call passes alpha_max_out = NULL."""
    w = scenes.workload("car4d_60x60x20x36")
    V0 = scenes.initial_value(w.grid, w.scene)
    run_two_calls(hj, w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, prec, hj.HJ_DYN_CAR4D,
                  (w.a_max, w.w_max), oracle.DYN_CAR4D, V0, 0.005, alpha_on_second=False)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_constant_dynamics_periodic_xy(hj, prec):
    """Constant velocity (no control) with negative v and theta components, on
    a grid whose x and y axes are periodic as well as theta; white-noise V0."""
    n = (13, 11, 7, 10)
    lo, hi = (-2.0, 0.0, -1.0, -math.pi), (3.0, 4.0, 2.0, math.pi)
    c = (0.7, -1.1, -0.45, -0.9)
    V0 = np.random.default_rng(31).uniform(-1.0, 1.0, size=n)
    run_two_calls(hj, n, lo, hi, 0b1011, prec, hj.HJ_DYN_CONST, c, oracle.DYN_CONST, V0, 0.02)


def test_noalloc_rejects_bad_arrays(hj):
    """Sizes and overlaps are checked before anything runs: in the binding
    (dtype, element count, overlap) and in the C entry point (byte count,
    overlap), so no kernel can read or write past a caller's array."""
    import ctypes
    import torch
    n, lo, hi = (5, 6, 3, 8), (-1.0, -1.0, 0.0, -math.pi), (1.0, 1.0, 1.0, math.pi)
    ncell = int(np.prod(n))
    x = torch.zeros(ncell, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    args = (n, lo, hi, 0b1000, hj.HJ_FP32, hj.HJ_DYN_CAR4D, (1.0, 1.0))
    with pytest.raises(ValueError):
        hj.hj_step_noalloc(*args, x.double(), x.double(), y, 0.001)  # dtype of the other precision
    with pytest.raises(ValueError):
        hj.hj_step_noalloc(*args, x[:-1], x[:-1], y[:-1], 0.001)  # one element short
    with pytest.raises(ValueError):
        hj.hj_step_noalloc(*args, x, y, x, 0.001)  # v_out is v_in
    # the C entry point on its own: wrong byte count, then v_out inside v0
    cn = (ctypes.c_int32 * 4)(*n)
    clo = (ctypes.c_double * 4)(*lo)
    chi = (ctypes.c_double * 4)(*hi)
    prm = (ctypes.c_double * 2)(1.0, 1.0)
    for vout, nbytes in ((y.data_ptr(), 4 * ncell - 4), (x.data_ptr() + 64, 4 * ncell)):
        rc = hj.lib.hj_step_noalloc(cn, clo, chi, 0b1000, hj.HJ_FP32, hj.HJ_DYN_CAR4D, prm, 2,
                                    ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(vout), nbytes, 0.001, None, None)
        assert rc == hj.HJ_ERR_INVALID_ARG
    # and the table limit
    x = torch.zeros(3 * 3 * 129 * 128, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(hj.HjError) as e:
        hj.hj_step_noalloc((3, 3, 129, 128), (-1, -1, 0, -3.14), (1, 1, 1, 3.14), 0b1000, hj.HJ_FP32,
                           hj.HJ_DYN_CAR4D, (1.0, 1.0), x, x.clone(), y, 0.001)
    assert e.value.status == hj.HJ_ERR_INVALID_ARG
    assert "16384" in str(e.value)
