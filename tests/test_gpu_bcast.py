"""Broadcast V0: when V0 depends on the position only (Eq. init_V), the grid
keeps its N1 x N2 field and the tiled kernel reads V0 from it instead of a
4D box per plane.  The values are the same, so the results must be the same
bits as with the 4D V0, and match the oracle as the 4D path does."""
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


def solve(hj, w, prec, xy, kernel=None, T=None, shape=None):
    import torch
    with hj.Grid.for_workload(w, prec) as g:
        if kernel is not None:
            g.set_kernel(kernel)
        if xy:
            g.set_initial_value_xy(scenes.signed_distance_xy(w.grid, w.scene))
            assert g.info().v0_broadcast == 1
        else:
            g.set_initial_value(scenes.initial_value(w.grid, w.scene))
            assert g.info().v0_broadcast == 0
        if shape is not None:
            g.set_tile_shape(shape)
        st = g.solve_brt(w.T if T is None else T, w.cfl)
        n = int(np.prod(w.grid.n))
        dt = torch.int32 if prec == hj.HJ_Q527 else (torch.float32 if prec == hj.HJ_FP32 else torch.float64)
        out = torch.empty(n, dtype=dt, device="cuda")
        g.read_value_device(out)
        return out.cpu().numpy().reshape(w.grid.n), st, g.info()


@pytest.mark.parametrize("name", ["car4d_31x31x11x16", "car4d_60x60x20x36"])
def test_broadcast_v0_same_bits_fp32_and_q527(hj, name):
    w = scenes.workload(name)
    for prec in (hj.HJ_FP32, hj.HJ_Q527):
        for kern in (hj.HJ_KERNEL_TILED, hj.HJ_KERNEL_RESIDENT):
            a, sta, ia = solve(hj, w, prec, xy=False, kernel=kern)
            b, stb, ib = solve(hj, w, prec, xy=True, kernel=kern)
            assert ia.kernel == ib.kernel == kern
            assert sta.steps == stb.steps
            assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [(7, 9, 5, 6), (17, 13, 11, 26), (12, 10, 9, 33), (9, 21, 4, 8)])
def test_broadcast_v0_ragged_grids(hj, n):
    w = scenes.custom_workload(n, n_circles=3, n_rects=1, T=0.4, seed=sum(n))
    for prec in (hj.HJ_FP32, hj.HJ_Q527):
        a, _, _ = solve(hj, w, prec, xy=False, kernel=hj.HJ_KERNEL_TILED)
        b, _, _ = solve(hj, w, prec, xy=True, kernel=hj.HJ_KERNEL_TILED)
        assert np.array_equal(a, b)
    # and against the oracle (fixed point: bit for bit)
    P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D, (w.a_max, w.w_max))
    Qo, _ = oracle.solve_q527(P, scenes.initial_value(w.grid, w.scene), w.T, w.cfl)
    q, _, _ = solve(hj, w, hj.HJ_Q527, xy=True, kernel=hj.HJ_KERNEL_TILED)
    assert np.array_equal(q, Qo)


def test_broadcast_v0_tile_shapes_and_mode_switch(hj):
    w = scenes.workload("car4d_60x60x20x36")
    ref, _, _ = solve(hj, w, hj.HJ_FP32, xy=False, T=0.6, kernel=hj.HJ_KERNEL_TILED)
    for shape in ([3, 5, 20, 6], [8, 4, 60, 8], [6, 6, 13, 4]):
        b, _, _ = solve(hj, w, hj.HJ_FP32, xy=True, T=0.6, shape=shape, kernel=hj.HJ_KERNEL_TILED)
        assert np.array_equal(b, ref), shape
    # switching back to a 4D V0 on the same grid leaves the broadcast mode
    with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
        g.set_kernel(hj.HJ_KERNEL_TILED)
        g.set_initial_value_xy(scenes.signed_distance_xy(w.grid, w.scene))
        assert g.info().v0_broadcast == 1
        g.set_initial_value(scenes.initial_value(w.grid, w.scene))
        assert g.info().v0_broadcast == 0
        g.solve_brt(0.6, w.cfl)
        assert np.array_equal(g.read_value().astype(np.float32), ref)


@pytest.mark.parametrize("n, shape", [((17, 13, 11, 32), [4, 2, 5, 4]), ((12, 10, 9, 16), [3, 4, 0, 0]),
                                      ((9, 21, 5, 48), [5, 4, 0, 0]), ((10, 7, 3, 16), [2, 2, 3, 4]),
                                      ((26, 25, 11, 48), [12, 8, 0, 0]), ((10, 17, 19, 16), [16, 16, 4, 4])])
def test_broadcast_v0_several_rows_per_thread(hj, n, shape):
    """An even number of v rows per tile on a grid whose theta quads have one
    sign of cos and of sin takes the form in which a thread updates two
    adjacent v rows, or four when tv is a multiple of 4 and that leaves at
    least 8 consumer warps (the last two cases); N3 not a multiple of the
    rows a thread leaves the last rows of a thread outside the grid.  Both
    solve modes must give the 4D-V0 path's bits (and those of the one-row
    or two-row form, tv - 1)."""
    w = scenes.custom_workload(n, n_circles=3, n_rects=1, T=0.4, seed=sum(n) + 7)
    ref, st_ref, _ = solve(hj, w, hj.HJ_FP32, xy=False, kernel=hj.HJ_KERNEL_TILED)
    for shp in (shape, [shape[0], shape[1] - 1, shape[2], shape[3]]):
        b, st, info = solve(hj, w, hj.HJ_FP32, xy=True, kernel=hj.HJ_KERNEL_TILED, shape=shp)
        assert info.tile[1] == min(shp[1], n[2]), (shp, list(info.tile))
        assert st.steps == st_ref.steps and st.dt_last == st_ref.dt_last
        assert np.array_equal(b, ref), shp
    # convergence mode (the step also reduces max |V_{n+1} - V_n|)
    outs = []
    for xy in (False, True):
        with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
            g.set_kernel(hj.HJ_KERNEL_TILED)
            if xy:
                g.set_initial_value_xy(scenes.signed_distance_xy(w.grid, w.scene))
                g.set_tile_shape(shape)
            else:
                g.set_initial_value(scenes.initial_value(w.grid, w.scene))
            st = g.solve_converged(1e-3, 0.6, w.cfl)
            outs.append((g.read_value(), st.steps, st.last_change))
    assert outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2]
    assert np.array_equal(outs[0][0], outs[1][0])


def test_broadcast_v0_device_field(hj):
    import torch
    w = scenes.workload("car4d_31x31x11x16")
    xy = scenes.signed_distance_xy(w.grid, w.scene)
    a, _, _ = solve(hj, w, hj.HJ_FP32, xy=True, kernel=hj.HJ_KERNEL_TILED)
    with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
        g.set_kernel(hj.HJ_KERNEL_TILED)
        hj.hj_set_initial_value_xy_device(g.handle, torch.from_numpy(xy.ravel().copy()).cuda())
        assert g.info().v0_broadcast == 1
        g.solve_brt(w.T, w.cfl)
        assert np.array_equal(g.read_value().astype(np.float32), a)
        bad = torch.from_numpy(xy.ravel().copy()).cuda()
        bad[5] = float("nan")
        with pytest.raises(hj.HjError) as e:
            hj.hj_set_initial_value_xy_device(g.handle, bad)
        assert e.value.status == hj.HJ_ERR_INVALID_ARG


@pytest.mark.slow
def test_broadcast_v0_full_size_same_bits(hj):
    """128x128x64x96 with the autotuned tile of each mode (the benchmark's
    launch configurations): the broadcast-V0 solve gives the 4D solve's bits."""
    import torch
    w = scenes.workload("car4d_128x128x64x96")
    outs = []
    for xy in (False, True):
        with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
            if xy:
                g.set_initial_value_xy(scenes.signed_distance_xy(w.grid, w.scene))
            else:
                g.set_initial_value(scenes.initial_value(w.grid, w.scene))
            g.autotune(4)
            g.solve_brt(0.3, w.cfl)
            out = torch.empty(int(np.prod(w.grid.n)), dtype=torch.float32, device="cuda")
            g.read_value_device(out)
            outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
