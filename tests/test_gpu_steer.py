"""GPU parity of the steering car (Eq. car_dynamics as printed in Sec. IV-A:
th' = v tan(delta) / L, |a| <= 1.5, |delta| <= pi/18, L = 0.3 m) against the
oracle: FP64 to 1e-12 with the same dt sequence, FP32 to 1e-4 max|V0| with
no sign flips, Q5.27 bit for bit."""
import math

import numpy as np
import pytest

import oracle
from paper_2012_04011_gb300 import scenes

pytestmark = pytest.mark.gpu

STEER = (1.5, math.pi / 18, 0.3)


@pytest.fixture(scope="module")
def hj():
    from paper_2012_04011_gb300 import _build
    _build.build()
    from paper_2012_04011_gb300 import hj as mod
    return mod


def oracle_steer(w, params=STEER):
    return oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D_STEER, params)


def gpu(hj, w, prec, kernel, params=STEER, xy=False, T=None, raw=False):
    import torch
    with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, prec) as g:
        g.set_dynamics(hj.HJ_DYN_CAR4D_STEER, params)
        g.set_kernel(kernel)
        if xy:
            g.set_initial_value_xy(scenes.signed_distance_xy(w.grid, w.scene))
        else:
            g.set_initial_value(scenes.initial_value(w.grid, w.scene))
        st = g.solve_brt(w.T if T is None else T, w.cfl)
        if raw:
            dt = {hj.HJ_FP32: torch.float32, hj.HJ_FP64: torch.float64, hj.HJ_Q527: torch.int32}[prec]
            out = torch.empty(int(np.prod(w.grid.n)), dtype=dt, device="cuda")
            g.read_value_device(out)
            return out.cpu().numpy().reshape(w.grid.n), st
        return g.read_value(), st


@pytest.mark.parametrize("name", ["car4d_31x31x11x16", "car4d_60x60x20x36"])
def test_steer_fp64_and_q527(hj, name):
    w = scenes.workload(name)
    V0 = scenes.initial_value(w.grid, w.scene)
    P = oracle_steer(w)
    Vo, dts = oracle.solve(P, V0, w.T, w.cfl, nthreads=oracle.max_threads())
    V, st = gpu(hj, w, hj.HJ_FP64, hj.HJ_KERNEL_GENERIC)
    assert st.steps == len(dts) and st.dt_first == dts[0] and st.dt_last == dts[-1]
    assert float(np.abs(V - Vo).max()) <= 1e-12
    Qo, dq = oracle.solve_q527(P, V0, w.T, w.cfl, nthreads=oracle.max_threads())
    for k in (hj.HJ_KERNEL_GENERIC, hj.HJ_KERNEL_TILED):
        Q, st = gpu(hj, w, hj.HJ_Q527, k, raw=True)
        assert st.kernel == k and st.steps == len(dq)
        assert np.array_equal(Q, Qo), (k, int(np.count_nonzero(Q != Qo)))


@pytest.mark.parametrize("kernel", ["generic", "tiled"])
@pytest.mark.parametrize("name", ["car4d_31x31x11x16", "car4d_60x60x20x36"])
def test_steer_fp32(hj, name, kernel):
    w = scenes.workload(name)
    V0 = scenes.initial_value(w.grid, w.scene)
    Vo, dts = oracle.solve(oracle_steer(w), V0, w.T, w.cfl, nthreads=oracle.max_threads())
    k = hj.HJ_KERNEL_TILED if kernel == "tiled" else hj.HJ_KERNEL_GENERIC
    V, st = gpu(hj, w, hj.HJ_FP32, k)
    assert st.kernel == k and st.steps == len(dts) and st.dt_first == dts[0] and st.dt_last == dts[-1]
    assert float(np.abs(V - Vo).max()) <= 1e-4 * float(np.abs(V0).max())
    m = np.abs(Vo) >= 1e-3
    assert int(np.count_nonzero(np.sign(V[m]) != np.sign(Vo[m]))) == 0


@pytest.mark.parametrize("n", [(7, 9, 5, 6), (17, 13, 11, 26), (12, 10, 9, 33)])
def test_steer_ragged_grids(hj, n):
    w = scenes.custom_workload(n, n_circles=3, n_rects=1, T=0.4, seed=sum(n) + 1)
    V0 = scenes.initial_value(w.grid, w.scene)
    P = oracle_steer(w)
    Vo, dts = oracle.solve(P, V0, w.T, w.cfl)
    V, st = gpu(hj, w, hj.HJ_FP64, hj.HJ_KERNEL_GENERIC)
    assert st.steps == len(dts) and float(np.abs(V - Vo).max()) <= 1e-12
    Qo, _ = oracle.solve_q527(P, V0, w.T, w.cfl)
    for k in (hj.HJ_KERNEL_GENERIC, hj.HJ_KERNEL_TILED):
        Q, _ = gpu(hj, w, hj.HJ_Q527, k, raw=True)
        assert np.array_equal(Q, Qo)
        V32, _ = gpu(hj, w, hj.HJ_FP32, k)
        assert float(np.abs(V32 - Vo).max()) <= 1e-4 * float(np.abs(V0).max())


def test_steer_broadcast_v0_and_zero_angle(hj):
    w = scenes.workload("car4d_60x60x20x36")
    a, _ = gpu(hj, w, hj.HJ_FP32, hj.HJ_KERNEL_TILED, raw=True, T=0.7)
    b, _ = gpu(hj, w, hj.HJ_FP32, hj.HJ_KERNEL_TILED, raw=True, T=0.7, xy=True)
    assert np.array_equal(a, b)
    # delta_max = 0 is the heading-rate car with w_max = 0, bit for bit
    z, _ = gpu(hj, w, hj.HJ_FP32, hj.HJ_KERNEL_TILED, params=(1.5, 0.0, 0.3), raw=True, T=0.7)
    with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP32) as g:
        g.set_dynamics(hj.HJ_DYN_CAR4D, (1.5, 0.0))
        g.set_kernel(hj.HJ_KERNEL_TILED)
        g.set_initial_value(scenes.initial_value(w.grid, w.scene))
        g.solve_brt(0.7, w.cfl)
        assert np.array_equal(g.read_value().astype(np.float32), z)


@pytest.mark.parametrize("n, shape", [((26, 25, 11, 48), [12, 8, 0, 0]), ((17, 13, 11, 32), [4, 2, 5, 4]),
                                      ((10, 17, 19, 16), [16, 16, 4, 4])])
def test_steer_broadcast_v0_several_rows_per_thread(hj, n, shape):
    """The steering car's theta coefficient grows with the speed, so each of
    the two or four v rows a thread updates in the broadcast-V0 single-sided
    form has its own (theta counts a multiple of 16 give every quad one sign
    of cos and sin).  The results must be the 4D-V0 path's bits, and the
    oracle's within the FP32 tolerance."""
    import torch
    w = scenes.custom_workload(n, n_circles=3, n_rects=1, T=0.5, seed=sum(n) + 11)
    V0 = scenes.initial_value(w.grid, w.scene)
    outs = []
    for xy in (False, True):
        with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP32) as g:
            g.set_dynamics(hj.HJ_DYN_CAR4D_STEER, STEER)
            g.set_kernel(hj.HJ_KERNEL_TILED)
            if xy:
                g.set_initial_value_xy(scenes.signed_distance_xy(w.grid, w.scene))
                g.set_tile_shape(shape)
                assert g.info().tile[1] == min(shape[1], n[2])
            else:
                g.set_initial_value(V0)
            st = g.solve_brt(w.T, w.cfl)
            out = torch.empty(int(np.prod(n)), dtype=torch.float32, device="cuda")
            g.read_value_device(out)
            outs.append((out.cpu().numpy().reshape(n), st.steps))
    assert outs[0][1] == outs[1][1]
    assert np.array_equal(outs[0][0], outs[1][0])
    Vo, dts = oracle.solve(oracle_steer(w), V0, w.T, w.cfl)
    assert outs[1][1] == len(dts)
    assert float(np.abs(outs[1][0] - Vo).max()) <= 1e-4 * float(np.abs(V0).max())


def test_steer_parameter_checks(hj):
    w = scenes.workload("car4d_31x31x11x16")
    with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP32) as g:
        for bad in ((1.5, math.pi / 2, 0.3), (1.5, 0.1, 0.0), (-1.0, 0.1, 0.3), (1.5, 0.1)):
            with pytest.raises(hj.HjError) as e:
                g.set_dynamics(hj.HJ_DYN_CAR4D_STEER, bad)
            assert e.value.status == hj.HJ_ERR_INVALID_ARG


@pytest.mark.slow
def test_steer_full_size_sampled_step_parity(hj):
    """128x128x64x96 in the benchmark's launch configuration: one FP32 tiled
    step from the GPU's V_n against the oracle's step at sampled cells."""
    w = scenes.workload("car4d_128x128x64x96")
    V0 = scenes.initial_value(w.grid, w.scene)
    P = oracle_steer(w)
    rng = np.random.default_rng(29)
    cells = np.unique(rng.choice(V0.size, 4000, replace=False))
    with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP32) as g:
        g.set_dynamics(hj.HJ_DYN_CAR4D_STEER, STEER)
        assert g.info().kernel == hj.HJ_KERNEL_TILED
        g.set_initial_value(V0)
        V0d = g.read_value()
        g.advance_brt(w.T, w.cfl, 6)
        Vn = g.read_value()
        st = g.advance_brt(w.T, w.cfl, 1)
        Vn1 = g.read_value()
        want = oracle.step_cells(P, Vn, V0d, st.dt_last, cells)
        tol = 8 * np.finfo(np.float32).eps * float(np.abs(V0).max())
        assert float(np.abs(Vn1.reshape(-1)[cells] - want).max()) <= tol
        assert np.all(Vn1 <= V0d)
