"""GPU parity: the CUDA path, called through the C ABI, against the FP64 CPU
oracle on the same seeded inputs.

Tolerances (from the precision of each path):
  FP64 path: max |V_gpu - V_oracle| <= 1e-12 (absolute) and the same dt
             sequence bit for bit (both sides compute alpha^max, the CFL sum
             and the cut last step in the same FP64 operation order).
  FP32 path: max |V_gpu - V_oracle| <= 1e-4 * max|V0|, and no BRT sign flip
             among cells with |V_oracle| >= 1e-3; the time loop is FP64
             bookkeeping (alpha^max from the FP64 table), so the step count
             and the dt sequence equal the oracle's exactly.
Full-size grids use sampled one-step parity: the GPU's V_n is read back, the
oracle computes one step at sampled cells from it, and the GPU's V_{n+1} must
match there; properties that hold at any size (V <= V0) are checked on every
cell.
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


def oracle_problem(w, dyn=oracle.DYN_CAR4D, params=None):
    if params is None:
        params = (w.a_max, w.w_max)
    return oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, dyn, params)


def fp32_tol(V0):
    return 1e-4 * float(np.abs(V0).max())


def sign_flips(V, Vref, band=1e-3):
    m = np.abs(Vref) >= band
    return int(np.count_nonzero(np.sign(V[m]) != np.sign(Vref[m])))


def gpu_solve(hj, w, V0, prec, kernel, T=None, cfl=None):
    with hj.Grid.for_workload(w, prec) as g:
        g.set_kernel(kernel)
        g.set_initial_value(V0)
        st = g.solve_brt(w.T if T is None else T, w.cfl if cfl is None else cfl)
        return g.read_value(), st


# ---------------------------------------------------------------- seeded workloads

@pytest.mark.parametrize("name", ["car4d_31x31x11x16", "car4d_60x60x20x36"])
def test_fp64_matches_oracle(hj, name):
    w = scenes.workload(name)
    V0 = scenes.initial_value(w.grid, w.scene)
    Vo, dts = oracle.solve(oracle_problem(w), V0, w.T, w.cfl, nthreads=16)
    V, st = gpu_solve(hj, w, V0, hj.HJ_FP64, hj.HJ_KERNEL_GENERIC)
    assert st.steps == len(dts)
    assert st.dt_first == dts[0] and st.dt_last == dts[-1]
    assert st.t_final == w.T
    assert float(np.abs(V - Vo).max()) <= 1e-12


@pytest.mark.parametrize("kernel", ["generic", "tiled"])
@pytest.mark.parametrize("name", ["car4d_31x31x11x16", "car4d_60x60x20x36"])
def test_fp32_matches_oracle(hj, name, kernel):
    w = scenes.workload(name)
    V0 = scenes.initial_value(w.grid, w.scene)
    Vo, dts = oracle.solve(oracle_problem(w), V0, w.T, w.cfl, nthreads=16)
    k = hj.HJ_KERNEL_TILED if kernel == "tiled" else hj.HJ_KERNEL_GENERIC
    V, st = gpu_solve(hj, w, V0, hj.HJ_FP32, k)
    assert st.kernel == k
    assert st.steps == len(dts) and st.dt_first == dts[0] and st.dt_last == dts[-1]
    assert st.t_final == w.T
    err = float(np.abs(V - Vo).max())
    assert err <= fp32_tol(V0), err
    assert sign_flips(V, Vo) == 0


def test_fp64_dt_sequence_bitwise(hj):
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    _, dts = oracle.solve(oracle_problem(w), V0, w.T, w.cfl)
    got = []
    with hj.Grid.for_workload(w, hj.HJ_FP64) as g:
        g.set_initial_value(V0)
        while True:
            st = g.advance_brt(w.T, w.cfl, 1)
            if st.steps == 0:
                break
            got.append(st.dt_last)
    assert np.array_equal(np.array(got), dts)


# ---------------------------------------------------------------- small and ragged grids

SMALL = [(3, 3, 3, 3), (5, 4, 3, 5), (7, 9, 5, 6), (17, 13, 11, 26), (12, 10, 9, 33), (9, 21, 4, 8)]


@pytest.mark.parametrize("n", SMALL)
def test_small_ragged_grids(hj, n):
    w = scenes.custom_workload(n, n_circles=3, n_rects=1, T=0.4, seed=sum(n))
    V0 = scenes.initial_value(w.grid, w.scene)
    Vo, dts = oracle.solve(oracle_problem(w), V0, w.T, w.cfl)
    for k in (hj.HJ_KERNEL_GENERIC, hj.HJ_KERNEL_RESIDENT):
        V, st = gpu_solve(hj, w, V0, hj.HJ_FP64, k)
        assert st.steps == len(dts) and st.dt_first == dts[0] and st.dt_last == dts[-1]
        assert float(np.abs(V - Vo).max()) <= 1e-12
    for k in (hj.HJ_KERNEL_GENERIC, hj.HJ_KERNEL_TILED, hj.HJ_KERNEL_RESIDENT):
        V, st = gpu_solve(hj, w, V0, hj.HJ_FP32, k)
        assert st.steps == len(dts) and st.dt_first == dts[0] and st.dt_last == dts[-1]
        assert float(np.abs(V - Vo).max()) <= fp32_tol(V0)
        assert sign_flips(V, Vo) == 0


def test_random_v0_tiled_vs_oracle(hj):
    """White-noise V0 (not a distance field): every neighbour and ghost value
    matters, so an indexing slip in the tile or halo shows up at once."""
    w = scenes.custom_workload((11, 19, 9, 20), T=0.2)
    V0 = np.random.default_rng(5).uniform(-1, 1, size=w.grid.n)
    Vo, _ = oracle.solve(oracle_problem(w), V0, w.T, w.cfl)
    for k in (hj.HJ_KERNEL_GENERIC, hj.HJ_KERNEL_TILED):
        V, _ = gpu_solve(hj, w, V0, hj.HJ_FP32, k)
        assert float(np.abs(V - Vo).max()) <= 1e-5
    V, _ = gpu_solve(hj, w, V0, hj.HJ_FP64, hj.HJ_KERNEL_GENERIC)
    assert float(np.abs(V - Vo).max()) <= 1e-12


@pytest.mark.parametrize("c", [(1.7, 0, 0, 0), (0, -1.3, 0, 0), (0, 0, 0.9, 0), (0, 0, 0, -2.1), (1.1, -0.6, 0.4, 0.8)])
def test_constant_dynamics_vs_oracle(hj, c):
    n = (6, 7, 5, 8)
    lo, hi = (-5.0, -4.0, 0.0, -math.pi), (5.0, 4.0, 4.0, math.pi)
    V0 = np.random.default_rng(9).uniform(-1, 1, size=n)
    P = oracle.Problem(n, lo, hi, 0b1000, oracle.DYN_CONST, c)
    for cfl in (1.0, 0.8):
        Vo, _, dts = oracle.advance(P, V0, V0, 0.0, 1.0, cfl=cfl, max_steps=5)
        with hj.Grid(n, lo, hi, 0b1000, hj.HJ_FP64) as g:
            g.set_dynamics(hj.HJ_DYN_CONST, c)
            g.set_initial_value(V0)
            st = g.advance_brt(1.0, cfl, 5)
            V = g.read_value()
        assert st.steps == len(dts)
        assert float(np.abs(V - Vo).max()) <= 1e-12


def test_all_axes_periodic_generic(hj):
    n = (6, 5, 7, 8)
    lo, hi = (0.0, 0.0, 0.0, 0.0), (1.0, 2.0, 3.0, 4.0)
    V0 = np.random.default_rng(2).normal(size=n)
    c = (0.3, -0.7, 0.5, 0.2)
    P = oracle.Problem(n, lo, hi, 0b1111, oracle.DYN_CONST, c)
    Vo, _, _ = oracle.advance(P, V0, V0, 0.0, 1.0, cfl=0.9, max_steps=6)
    with hj.Grid(n, lo, hi, 0b1111, hj.HJ_FP64) as g:
        g.set_dynamics(hj.HJ_DYN_CONST, c)
        g.set_initial_value(V0)
        g.advance_brt(1.0, 0.9, 6)
        V = g.read_value()
    assert float(np.abs(V - Vo).max()) <= 1e-12


# ---------------------------------------------------------------- API semantics on the device

def test_resume_equals_single_call(hj):
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    for prec in (hj.HJ_FP64, hj.HJ_FP32):
        with hj.Grid.for_workload(w, prec) as g:
            g.set_initial_value(V0)
            g.solve_brt(0.37, w.cfl)
            g.advance_brt(w.T, w.cfl, 5)
            st = g.solve_brt(w.T, w.cfl)
            Va = g.read_value()
            assert st.t_final == w.T
            again = g.solve_brt(w.T, w.cfl)  # T <= t: no-op
            assert again.steps == 0
        with hj.Grid.for_workload(w, prec) as g:
            g.set_initial_value(V0)
            g.solve_brt(0.37, w.cfl)
            g.solve_brt(w.T, w.cfl)
            Vb = g.read_value()
        assert np.array_equal(Va, Vb)


def test_dynamics_change_mid_solve(hj):
    """set_dynamics between two solve calls: the solve continues from V(t1)
    under the new control bounds, with alpha^max and dt taken from the new
    Hamiltonian (Alg. 2), as the oracle's advance does."""
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    t1, new = 0.37, (2.5, 0.4)
    P1, P2 = oracle_problem(w), oracle_problem(w, params=new)
    V1, _, d1 = oracle.advance(P1, V0, V0, 0.0, t1, w.cfl)
    Vo, _, d2 = oracle.advance(P2, V0, V1, t1, w.T, w.cfl)
    for prec in (hj.HJ_FP64, hj.HJ_FP32):
        kernels = (hj.HJ_KERNEL_GENERIC,) if prec == hj.HJ_FP64 else (hj.HJ_KERNEL_GENERIC, hj.HJ_KERNEL_TILED)
        for k in kernels:
            with hj.Grid.for_workload(w, prec) as g:
                g.set_kernel(k)
                g.set_initial_value(V0)
                g.solve_brt(t1, w.cfl)
                g.set_dynamics(hj.HJ_DYN_CAR4D, new)
                st = g.solve_brt(w.T, w.cfl)
                V = g.read_value()
            assert st.t_final == w.T
            if prec == hj.HJ_FP64:
                assert st.steps == len(d2) and st.dt_first == d2[0] and st.dt_last == d2[-1]
                assert float(np.abs(V - Vo).max()) <= 1e-12
            else:
                assert st.steps == len(d2) and st.dt_first == d2[0] and st.dt_last == d2[-1]
                assert float(np.abs(V - Vo).max()) <= fp32_tol(V0)
                assert sign_flips(V, Vo) == 0


def test_zero_horizon_and_zero_dynamics(hj):
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    for prec in (hj.HJ_FP64, hj.HJ_FP32):
        with hj.Grid.for_workload(w, prec) as g:
            g.set_initial_value(V0)
            st = g.solve_brt(0.0, w.cfl)
            assert st.steps == 0
            V = g.read_value()
        ref = V0 if prec == hj.HJ_FP64 else V0.astype(np.float32).astype(np.float64)
        assert np.array_equal(V, ref)
    with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP64) as g:
        g.set_dynamics(hj.HJ_DYN_CONST, (0, 0, 0, 0))
        g.set_initial_value(V0)
        st = g.solve_brt(0.5, 0.8)
        assert st.steps == 1
        assert np.array_equal(g.read_value(), V0)


def test_device_ingest_and_readback(hj):
    import torch
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    for prec in (hj.HJ_FP64, hj.HJ_FP32):
        with hj.Grid.for_workload(w, prec) as g:
            g.set_initial_value(V0)
            g.solve_brt(w.T, w.cfl)
            Vh = g.read_value()
            d64 = torch.empty(V0.size, dtype=torch.float64, device="cuda")
            d32 = torch.empty(V0.size, dtype=torch.float32, device="cuda")
            g.read_value_device(d64)
            g.read_value_device(d32)
            assert np.array_equal(d64.cpu().numpy().reshape(V0.shape), Vh)
            assert np.array_equal(d32.cpu().numpy().reshape(V0.shape), Vh.astype(np.float32))
            g.set_initial_value(torch.from_numpy(V0).cuda())
            g.solve_brt(w.T, w.cfl)
            assert np.array_equal(g.read_value(), Vh)


def test_device_arrays_follow_the_default_stream(hj):
    """A grid or batch on its own stream touches a caller's device array only
    after the work already queued on the default stream: an input whose copy
    still waits behind a long kernel arrives whole, and an output that a queued
    fill would overwrite receives the values.  (torch.cuda._sleep is a spin of
    a fixed cycle count: it ends by itself.)"""
    import torch
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    src = torch.from_numpy(V0.ravel().copy()).cuda()
    torch.cuda.synchronize()
    with hj.Grid.for_workload(w, hj.HJ_FP64) as g:
        dst = torch.zeros_like(src)
        torch.cuda._sleep(200_000_000)  # about 0.1 s
        dst.copy_(src)
        hj.hj_set_initial_value_device(g.handle, dst)
        out = torch.empty_like(src)
        torch.cuda._sleep(200_000_000)
        out.fill_(-7.0)
        g.read_value_device(out)
        assert np.array_equal(out.cpu().numpy(), V0.ravel())
    with hj.Batch(2) as b:
        slot = b.add_workload(w)
        dst = torch.zeros_like(src)
        torch.cuda._sleep(200_000_000)
        dst.copy_(src)
        b.set_initial_value(slot, dst)
        out = torch.empty(V0.size, dtype=torch.float32, device="cuda")
        torch.cuda._sleep(200_000_000)
        out.fill_(-7.0)
        b.read_value(slot, out)
        assert np.array_equal(out.cpu().numpy(), V0.ravel().astype(np.float32))


def test_pinned_host_buffers_equal_pageable(hj):
    """V0 from pinned host memory (read by the ingest kernel over the host
    link) and V into pinned host memory (written by the readback kernel) give
    the same bytes as the staged copies of pageable buffers."""
    import torch
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    V0p = torch.from_numpy(V0.copy()).pin_memory().numpy()
    for prec in (hj.HJ_FP64, hj.HJ_FP32, hj.HJ_Q527):
        outs = []
        for src in (V0, V0p):
            with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, prec) as g:
                g.set_dynamics(hj.HJ_DYN_CAR4D, (w.a_max, w.w_max))
                g.set_initial_value(src)
                assert np.array_equal(g.read_value(), g.read_value(torch.empty(V0.shape, dtype=torch.float64)
                                                                  .pin_memory().numpy()))
                g.solve_brt(w.T, w.cfl)
                pinned = torch.empty(V0.shape, dtype=torch.float64).pin_memory().numpy()
                g.read_value(pinned)
                assert np.array_equal(pinned, g.read_value())
                outs.append(pinned.copy())
        assert np.array_equal(outs[0], outs[1]), prec
    # a NaN in pinned V0 is rejected as in pageable memory
    bad = torch.from_numpy(V0.copy()).pin_memory().numpy()
    bad[1, 2, 3, 4] = np.nan
    with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
        with pytest.raises(hj.HjError) as e:
            g.set_initial_value(bad)
        assert e.value.status == hj.HJ_ERR_INVALID_ARG


def test_errors_on_device(hj):
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    g = hj.hj_create_grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP32)
    try:
        with pytest.raises(hj.HjError) as e:
            hj.hj_solve_brt(g, 1.0)
        assert e.value.status == hj.HJ_ERR_STATE
        hj.hj_set_dynamics(g, hj.HJ_DYN_CAR4D, (1.5, 1.0))
        with pytest.raises(hj.HjError) as e:
            hj.hj_solve_brt(g, 1.0)
        assert e.value.status == hj.HJ_ERR_STATE
        bad = V0.copy()
        bad[3, 4, 5, 6] = np.nan
        with pytest.raises(hj.HjError) as e:
            hj.hj_set_initial_value(g, bad)
        assert e.value.status == hj.HJ_ERR_INVALID_ARG
        with pytest.raises(hj.HjError) as e:
            hj.hj_set_initial_value(g, V0[:-1])
        assert e.value.status == hj.HJ_ERR_INVALID_ARG
        hj.hj_set_initial_value(g, V0)
        for T, cfl in ((-1.0, 0.8), (float("inf"), 0.8), (1.0, 0.0), (1.0, 1.5)):
            with pytest.raises(hj.HjError) as e:
                hj.hj_solve_brt(g, T, cfl)
            assert e.value.status == hj.HJ_ERR_INVALID_ARG
        with pytest.raises(hj.HjError) as e:
            hj.hj_set_dynamics(g, hj.HJ_DYN_CAR4D, (1.5,))
        assert e.value.status == hj.HJ_ERR_INVALID_ARG
        hj.hj_solve_brt(g, 0.1)
    finally:
        hj.hj_destroy_grid(g)
    with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP64) as g2:
        g2.set_dynamics(hj.HJ_DYN_CAR4D, (1.5, 1.0))
        with pytest.raises(hj.HjError) as e:
            g2.set_kernel(hj.HJ_KERNEL_TILED)
        assert e.value.status == hj.HJ_ERR_UNSUPPORTED


def test_grid_larger_than_device_memory(hj):
    """A grid the API accepts (2^33 cells at most) but the device cannot hold:
    8.58e9 FP64 cells with theta rows padded from 5 to 8 values need 3 x 110 GB.
    Creation reports HJ_ERR_OOM, releases what it had allocated, and the
    context goes on solving."""
    import torch
    n = (2048, 2048, 409, 5)
    assert np.prod(n, dtype=np.int64) <= 1 << 33
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    if 3 * 8 * 8 * n[0] * n[1] * n[2] <= total:  # V0 and two buffers, 8-value rows of doubles
        pytest.skip("this device could hold the grid")
    with pytest.raises(hj.HjError) as e:
        hj.hj_create_grid(n, scenes.DOMAIN_LO, scenes.DOMAIN_HI, scenes.PERIODIC_THETA, hj.HJ_FP64)
    assert e.value.status == hj.HJ_ERR_OOM
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 64 << 20
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    Vo, _ = oracle.solve(oracle_problem(w), V0, w.T, w.cfl)
    V, _ = gpu_solve(hj, w, V0, hj.HJ_FP64, hj.HJ_KERNEL_AUTO)
    assert float(np.abs(V - Vo).max()) <= 1e-12


# ---------------------------------------------------------------- full size (128x128x64x96)

@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_full_size_sampled_step_parity(hj, prec):
    """The large workload in the launch configuration the benchmark times:
    after n steps on the GPU, one more GPU step must match the oracle's step
    at sampled cells (from the same V_n); V <= V0 everywhere."""
    w = scenes.workload("car4d_128x128x64x96")
    V0 = scenes.initial_value(w.grid, w.scene)
    P = oracle_problem(w)
    p = hj.HJ_FP32 if prec == "fp32" else hj.HJ_FP64
    rng = np.random.default_rng(17)
    ncell = V0.size
    # samples: random cells plus every face, edge and corner class of the grid
    cells = list(rng.choice(ncell, 4000, replace=False))
    N = w.grid.n
    for i in (0, 1, N[0] // 2, N[0] - 2, N[0] - 1):
        for j in (0, 1, N[1] - 2, N[1] - 1):
            for k in (0, 1, N[2] // 2, N[2] - 1):
                for l in (0, 1, N[3] - 1):
                    cells.append(((i * N[1] + j) * N[2] + k) * N[3] + l)
    cells = np.unique(np.array(cells, dtype=np.int64))
    with hj.Grid.for_workload(w, p) as g:
        assert g.info().kernel == (hj.HJ_KERNEL_TILED if p == hj.HJ_FP32 else hj.HJ_KERNEL_GENERIC)
        g.set_initial_value(V0)
        if p == hj.HJ_FP32:
            g.autotune(8)  # the benchmark's launch configuration: the autotuned tile
        V0d = g.read_value()  # V0 as stored on the device (rounded in FP32)
        for n_before in (0, 7):
            if n_before:
                g.advance_brt(w.T, w.cfl, n_before)
            Vn = g.read_value()
            st = g.advance_brt(w.T, w.cfl, 1)
            Vn1 = g.read_value()
            want = oracle.step_cells(P, Vn, V0d, st.dt_last, cells)
            got = Vn1.reshape(-1)[cells]
            tol = 1e-12 if p == hj.HJ_FP64 else 8 * np.finfo(np.float32).eps * float(np.abs(V0).max())
            assert float(np.abs(got - want).max()) <= tol
            assert np.all(Vn1 <= V0d)
        if p == hj.HJ_FP32:
            st = g.solve_brt(w.T, w.cfl)
            assert st.t_final == w.T
            V = g.read_value()
            assert np.all(V <= V0d) and np.all(np.isfinite(V))


# ---------------------------------------------------------------- tile shapes and the autotuner

@pytest.mark.parametrize("name", ["car4d_31x31x11x16", "car4d_60x60x20x36"])
def test_every_tile_shape_gives_identical_bits(hj, name):
    """The per-cell arithmetic does not depend on the tiling, so every tile
    shape (ragged tiles, x chunks with halo planes, ring depth) must produce
    exactly the same values."""
    w = scenes.workload(name)
    V0 = scenes.initial_value(w.grid, w.scene)
    ref = None
    shapes = [(0, 0, 0, 0), (8, 4, 0, 4), (3, 5, 7, 3), (1, 7, 5, 5), (5, 3, 0, 8), (2, 2, 4, 0)]
    for shape in shapes:
        with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
            g.set_kernel(hj.HJ_KERNEL_TILED)
            try:
                g.set_tile_shape(shape)
            except hj.HjError as e:
                assert e.status == hj.HJ_ERR_UNSUPPORTED
                continue
            g.set_initial_value(V0)
            g.solve_brt(w.T, w.cfl)
            V = g.read_value()
        if ref is None:
            ref = V
        else:
            assert np.array_equal(V, ref), shape


def test_autotune_keeps_results_and_state(hj):
    w = scenes.workload("car4d_60x60x20x36")
    V0 = scenes.initial_value(w.grid, w.scene)
    with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
        g.set_kernel(hj.HJ_KERNEL_TILED)  # the kernel the autotuner shapes
        g.set_initial_value(V0)
        V_ref_st = g.solve_brt(w.T, w.cfl)
        V_ref = g.read_value()
        g.set_initial_value(V0)
        tried = g.autotune(4)
        assert len(tried) >= 1 and all(t.ms_per_step > 0 for t in tried)
        info = g.info()
        # the kept shape is the fastest of the re-timed ones, which are the
        # fastest of the first pass
        retimed = [t for t in tried if t.ms_retimed > 0]
        assert 1 <= len(retimed) <= 3
        first = sorted(t.ms_per_step for t in tried)
        assert all(t.ms_per_step <= first[len(retimed) - 1] for t in retimed)
        # (two shapes can re-time equal: the kept one is one of the fastest)
        kept = [t for t in retimed if list(t.shape) == list(info.tile)]
        assert kept and kept[0].ms_retimed == min(t.ms_retimed for t in retimed)
        assert info.total_steps == 0 and info.t == 0.0
        st = g.solve_brt(w.T, w.cfl)
        assert st.steps == V_ref_st.steps
        assert np.array_equal(g.read_value(), V_ref)
        with pytest.raises(hj.HjError) as e:
            g.autotune(2)  # after steps: refused
        assert e.value.status == hj.HJ_ERR_STATE


# ---------------------------------------------------------------- limits and unusual domains

def test_longest_theta_axis(hj):
    """N4 = 4096, the largest theta axis the API accepts (the tiled kernel
    takes rows of at most 256 points, so the generic kernel runs)."""
    w = scenes.custom_workload((5, 4, 3, 4096), n_circles=2, T=0.05, seed=41)
    V0 = scenes.initial_value(w.grid, w.scene)
    P = oracle_problem(w)
    Vo, dts = oracle.solve(P, V0, w.T, w.cfl)
    V, st = gpu_solve(hj, w, V0, hj.HJ_FP64, hj.HJ_KERNEL_AUTO)
    assert st.kernel == hj.HJ_KERNEL_GENERIC and st.steps == len(dts)
    assert float(np.abs(V - Vo).max()) <= 1e-12
    V, st = gpu_solve(hj, w, V0, hj.HJ_FP32, hj.HJ_KERNEL_AUTO)
    assert float(np.abs(V - Vo).max()) <= fp32_tol(V0)
    with pytest.raises(hj.HjError) as e:
        hj.hj_create_grid((5, 4, 3, 4097), w.grid.lo, w.grid.hi)
    assert e.value.status == hj.HJ_ERR_INVALID_ARG


@pytest.mark.parametrize("dyn", ["car", "steer"])
def test_negative_speeds_and_shifted_domain(hj, dyn):
    """A speed axis through zero (v in [-1, 3]) and an off-centre x/y domain:
    the steering car's heading rate changes sign with v, the heading-rate
    car's does not."""
    import math
    g = scenes.GridSpec((23, 19, 9, 16), lo=(-2.0, 1.0, -1.0, -math.pi), hi=(6.0, 7.5, 3.0, math.pi))
    rng = np.random.default_rng(12)
    sc = scenes.Scene(np.array([[1.0, 3.0, 0.8], [4.0, 5.5, 0.5]]))
    V0 = scenes.initial_value(g, sc)
    if dyn == "car":
        kind, params, okind = hj.HJ_DYN_CAR4D, (1.5, 1.0), oracle.DYN_CAR4D
    else:
        kind, params, okind = hj.HJ_DYN_CAR4D_STEER, (1.5, math.pi / 18, 0.3), oracle.DYN_CAR4D_STEER
    P = oracle.Problem(g.n, g.lo, g.hi, g.periodic, okind, params)
    Vo, dts = oracle.solve(P, V0, 0.6, 0.8)
    for prec, kern in ((hj.HJ_FP64, hj.HJ_KERNEL_GENERIC), (hj.HJ_FP32, hj.HJ_KERNEL_TILED),
                       (hj.HJ_FP32, hj.HJ_KERNEL_GENERIC)):
        with hj.Grid(g.n, g.lo, g.hi, g.periodic, prec) as gr:
            gr.set_dynamics(kind, params)
            gr.set_kernel(kern)
            gr.set_initial_value(V0)
            st = gr.solve_brt(0.6, 0.8)
            V = gr.read_value()
        if prec == hj.HJ_FP64:
            assert st.steps == len(dts) and float(np.abs(V - Vo).max()) <= 1e-12
        else:
            assert float(np.abs(V - Vo).max()) <= fp32_tol(V0) and sign_flips(V, Vo) == 0
    Qo, _ = oracle.solve_q527(P, V0, 0.6, 0.8)
    import torch
    for kern in (hj.HJ_KERNEL_GENERIC, hj.HJ_KERNEL_TILED):
        with hj.Grid(g.n, g.lo, g.hi, g.periodic, hj.HJ_Q527) as gr:
            gr.set_dynamics(kind, params)
            gr.set_kernel(kern)
            gr.set_initial_value(V0)
            gr.solve_brt(0.6, 0.8)
            out = torch.empty(V0.size, dtype=torch.int32, device="cuda")
            gr.read_value_device(out)
        assert np.array_equal(out.cpu().numpy().reshape(g.n), Qo)
