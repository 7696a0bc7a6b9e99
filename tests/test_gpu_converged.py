"""GPU parity of the convergence-threshold mode (Algorithm 2's test: stop
after a step whose largest change max |V_{n+1} - V_n| is below the
threshold) against the oracle: FP64 the same steps, the same last change to
1e-12 and V to 1e-12; Q5.27 bit for bit (exact change); FP32 within a step
of the oracle's count and the FP32 tolerance on V."""
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


def problem(w):
    return oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D, (w.a_max, w.w_max))


def codes(hj, g):
    import torch
    out = torch.empty(int(np.prod(g.info().n)), dtype=torch.int32, device="cuda")
    g.read_value_device(out)
    return out.cpu().numpy().reshape(tuple(g.info().n))


THR = 2e-3


@pytest.mark.parametrize("name", ["car4d_31x31x11x16", "car4d_60x60x20x36"])
def test_converged_fp64_and_q527(hj, name):
    w = scenes.workload(name)
    V0 = scenes.initial_value(w.grid, w.scene)
    P = problem(w)
    Vo, to, dts, eps, conv = oracle.advance_converged(P, V0, V0, 0.0, THR, 40.0, w.cfl,
                                                      nthreads=oracle.max_threads())
    assert conv
    with hj.Grid.for_workload(w, hj.HJ_FP64) as g:
        g.set_initial_value(V0)
        st = g.solve_converged(THR, 40.0, w.cfl)
        assert st.converged == 1 and st.steps == len(dts) and st.t_final == to
        assert abs(st.last_change - eps) <= 1e-12
        assert float(np.abs(g.read_value() - Vo).max()) <= 1e-12
        # a second call tests again after one more step (as the oracle's loop
        # does from the converged state), and that step changes V even less
        st2 = g.solve_converged(THR, 40.0, w.cfl)
        assert st2.steps == 1 and st2.converged == 1 and st2.last_change <= st.last_change
    Qo, tq, dq, eq, cq = oracle.advance_converged_q527(P, oracle.to_q527(V0), oracle.to_q527(V0), 0.0, THR, 40.0,
                                                       w.cfl, nthreads=oracle.max_threads())
    for k in (hj.HJ_KERNEL_GENERIC, hj.HJ_KERNEL_TILED):
        with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_Q527) as g:
            g.set_dynamics(hj.HJ_DYN_CAR4D, (w.a_max, w.w_max))
            g.set_kernel(k)
            g.set_initial_value(V0)
            st = g.solve_converged(THR, 40.0, w.cfl)
            assert st.converged == int(cq) and st.steps == len(dq) and st.last_change == eq
            assert np.array_equal(codes(hj, g), Qo)


@pytest.mark.parametrize("kernel", ["generic", "tiled"])
def test_converged_fp32(hj, kernel):
    w = scenes.workload("car4d_60x60x20x36")
    V0 = scenes.initial_value(w.grid, w.scene)
    Vo, to, dts, eps, conv = oracle.advance_converged(problem(w), V0, V0, 0.0, THR, 40.0, w.cfl,
                                                      nthreads=oracle.max_threads())
    k = hj.HJ_KERNEL_TILED if kernel == "tiled" else hj.HJ_KERNEL_GENERIC
    with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
        g.set_kernel(k)
        g.set_initial_value(V0)
        st = g.solve_converged(THR, 40.0, w.cfl)
        assert st.kernel == k and st.converged == 1 and st.last_change < THR
        # the dt sequence is the FP64 one; the step at which the FP32 change of
        # V first drops below the threshold may differ by a step or two, since
        # the change itself is an FP32 value
        assert st.dt_first == dts[0]
        assert abs(st.steps - len(dts)) <= 2
        V = g.read_value()
    # compare with the oracle after the GPU's own number of steps
    Vn, _, _ = oracle.advance(problem(w), V0, V0, 0.0, 40.0, w.cfl, max_steps=st.steps,
                              nthreads=oracle.max_threads())
    assert float(np.abs(V - Vn).max()) <= 1e-4 * float(np.abs(V0).max())


def test_converged_horizon_caps_and_fixed_mode_unchanged(hj):
    """A threshold the scheme does not reach stops at T_max with the same bits
    as the fixed-horizon solve; afterwards hj_solve_brt works as before."""
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
        g.set_initial_value(V0)
        st = g.solve_converged(1e-12, 0.5, w.cfl)
        assert st.converged == 0 and st.t_final == 0.5 and st.last_change > 0
        Va = g.read_value()
        g.set_initial_value(V0)
        st2 = g.solve_brt(0.5, w.cfl)
        assert st2.steps == st.steps and st2.converged == 0 and st2.last_change == 0
        assert np.array_equal(g.read_value(), Va)
        with pytest.raises(hj.HjError) as e:
            g.solve_converged(0.0, 1.0)
        assert e.value.status == hj.HJ_ERR_INVALID_ARG
