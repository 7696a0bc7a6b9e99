"""The largest workload solved to its horizon against the oracle.

car4d_128x128x64x96 (28 circles and 4 rectangles, T = 2.0 s, CFL 0.8, 352
steps): the whole time loop of Alg. 2 on the GPU, compared cell by cell with
the FP64 oracle's solve of the same seeded inputs (the per-grid-point
comparison of Sec. IV-B, Table I).

  FP32, the tiled kernel with the autotuned tile (the benchmark's launch
        configuration): max |V - V_oracle| <= 1e-4 max|V0|, no BRT sign flip
        among cells with |V_oracle| >= 1e-3, and the oracle's dt sequence bit
        for bit (the time loop is FP64 bookkeeping).
  FP64, the generic kernel: max |V - V_oracle| <= 1e-12 and the dt sequence
        bit for bit.

The oracle solve (3.5e10 cell-updates) takes about 75 s on 16 host cores; it
runs once for the module.
"""
import numpy as np
import pytest

import oracle
from paper_2012_04011_gb300 import scenes

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NAME = "car4d_128x128x64x96"


@pytest.fixture(scope="module")
def hj():
    from paper_2012_04011_gb300 import _build
    _build.build()
    from paper_2012_04011_gb300 import hj as mod
    return mod


@pytest.fixture(scope="module")
def solved():
    w = scenes.workload(NAME)
    V0 = scenes.initial_value(w.grid, w.scene)
    P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D, (w.a_max, w.w_max))
    Vo, dts = oracle.solve(P, V0, w.T, w.cfl, nthreads=oracle.max_threads())
    assert len(dts) == 352
    return w, V0, Vo, dts


def stepwise_dts(g, w):
    """Steps one at a time from V0 and returns the dt of every step."""
    got = []
    while True:
        st = g.advance_brt(w.T, w.cfl, 1)
        if st.steps == 0:
            return np.array(got)
        got.append(st.dt_last)


def test_fp32_tiled_full_horizon(hj, solved):
    w, V0, Vo, dts = solved
    with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
        assert g.info().kernel == hj.HJ_KERNEL_TILED
        g.set_initial_value(V0)
        g.autotune(8)
        st = g.solve_brt(w.T, w.cfl)
        V = g.read_value()
        assert st.kernel == hj.HJ_KERNEL_TILED and st.t_final == w.T
        assert st.steps == len(dts) and st.dt_first == dts[0] and st.dt_last == dts[-1]
        # the same solve one step per call: every dt, and the same bits
        g.set_initial_value(V0)
        assert np.array_equal(stepwise_dts(g, w), dts)
        assert np.array_equal(g.read_value(), V)
    err = float(np.abs(V - Vo).max())
    assert err <= 1e-4 * float(np.abs(V0).max()), err
    band = np.abs(Vo) >= 1e-3
    assert int(np.count_nonzero(np.sign(V[band]) != np.sign(Vo[band]))) == 0
    V0f = V0.astype(np.float32).astype(np.float64)  # V0 as the FP32 grid stores it
    assert np.all(V <= V0f)


def test_fp64_generic_full_horizon(hj, solved):
    w, V0, Vo, dts = solved
    with hj.Grid.for_workload(w, hj.HJ_FP64) as g:
        assert g.info().kernel == hj.HJ_KERNEL_GENERIC
        g.set_initial_value(V0)
        assert np.array_equal(stepwise_dts(g, w), dts)
        assert g.info().t == w.T
        V = g.read_value()
    err = float(np.abs(V - Vo).max())
    assert err <= 1e-12, err
    band = np.abs(Vo) >= 1e-3
    assert int(np.count_nonzero(np.sign(V[band]) != np.sign(Vo[band]))) == 0
