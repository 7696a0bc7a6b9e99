"""hj_step_noalloc: the entry point for callers that cannot allocate device
memory (their device memory belongs to a host framework's pool, a budget
fixed at start-up, or a moment where cudaMalloc must not synchronise the
device).  It steps caller-owned arrays and keeps its working data in a fixed
device array, so it must give the same step as the grid API.

Two calls in a row, each checked against the grid API's step with the same
dt, within the tolerances the parity tests use (FP64 1e-12, FP32 1e-4 of
max|V0|).  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2012_04011_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hj():
    from paper_2012_04011_gb300 import _build
    _build.build()
    from paper_2012_04011_gb300 import hj as mod
    return mod


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_grid_api_on_two_calls(hj, prec):
    import torch
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    p = hj.HJ_FP64 if prec == "fp64" else hj.HJ_FP32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-4 * float(np.abs(V0).max())
    dt = 0.01  # below the CFL step (0.0264), so the grid API takes exactly this step
    v0_dev = torch.from_numpy(V0).to("cuda", tdt).reshape(-1)
    a = torch.empty_like(v0_dev)
    b = torch.empty_like(v0_dev)
    ref = torch.empty_like(v0_dev)
    stream = torch.cuda.current_stream().cuda_stream
    with hj.Grid.for_workload(w, p) as g:
        g.set_initial_value(v0_dev)
        src = v0_dev
        for call, out in enumerate((a, b), start=1):
            alpha = hj.hj_step_noalloc(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, p, hj.HJ_DYN_CAR4D,
                                       (w.a_max, w.w_max), src, v0_dev, out, dt, stream)
            st = g.advance_brt(call * dt, w.cfl, 1)
            assert st.steps == 1 and st.dt_last == dt
            g.read_value_device(ref)
            err = float((out.double() - ref.double()).abs().max())
            assert err <= tol, (call, err)
            assert alpha[0] == pytest.approx(4.0, rel=1e-6) and alpha[1] == pytest.approx(4.0, rel=1e-6)
            assert alpha[2] == w.a_max and alpha[3] == w.w_max
            src = out


def test_noalloc_rejects_oversized_tables(hj):
    import torch
    x = torch.zeros(3 * 3 * 129 * 128, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(hj.HjError) as e:
        hj.hj_step_noalloc((3, 3, 129, 128), (-1, -1, 0, -3.14), (1, 1, 1, 3.14), 0b1000, hj.HJ_FP32,
                           hj.HJ_DYN_CAR4D, (1.0, 1.0), x, x, y, 0.001)
    assert e.value.status == hj.HJ_ERR_INVALID_ARG
    assert "16384" in str(e.value)
