"""Batched solves: many independent car grids stepped by one persistent
kernel that runs many batch steps per launch, each slot with its own grid, V0,
horizon and dt.

Each slot must give exactly what a single-grid FP32 solve of the same grid
gives (same per-cell arithmetic, same dt sequence), and must match the FP64
oracle within the FP32 tolerance (1e-4 max|V0|, no sign flip outside
|V| < 1e-3)."""
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


def oracle_problem(w):
    return oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D, (w.a_max, w.w_max))


def single_grid(hj, w, V0, T=None):
    with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
        g.set_kernel(hj.HJ_KERNEL_TILED)
        g.set_initial_value(V0)
        st = g.solve_brt(w.T if T is None else T, w.cfl)
        return g.read_value(), st


MIXED = [(21, 19, 9, 16), (17, 23, 7, 26), (12, 10, 9, 33), (25, 25, 11, 24), (9, 21, 4, 8), (30, 14, 6, 30)]


def test_batch_slots_equal_single_grid_solves(hj):
    ws = [scenes.custom_workload(n, n_circles=3, n_rects=1, T=0.3 + 0.05 * i, seed=40 + i) for i, n in enumerate(MIXED)]
    v0s = [scenes.initial_value(w.grid, w.scene) for w in ws]
    with hj.Batch(len(ws)) as b:
        slots = [b.add_workload(w) for w in ws]
        for s, w, v0 in zip(slots, ws, v0s):
            b.set_initial_value(s, v0)
            b.set_horizon(s, w.T, w.cfl)
        st = b.advance()
        assert st.active == 0 and st.finished == len(ws)
        assert st.launches == 1  # every batch step of the solve in one launch
        for s, w, v0 in zip(slots, ws, v0s):
            ref, rst = single_grid(hj, w, v0)
            info = b.slot_info(s)
            assert info.steps == rst.steps and info.t == w.T
            assert np.array_equal(b.read_value(s), ref), (s, w.grid.n)


def test_batch_matches_oracle(hj):
    ws = [scenes.custom_workload(n, n_circles=4, T=0.4, seed=90 + i) for i, n in enumerate(MIXED[:4])]
    with hj.Batch(8) as b:
        slots = []
        for w in ws:
            s = b.add_workload(w)
            b.set_initial_value(s, scenes.initial_value(w.grid, w.scene))
            b.set_horizon(s, w.T, w.cfl)
            slots.append(s)
        b.advance()
        for s, w in zip(slots, ws):
            V0 = scenes.initial_value(w.grid, w.scene)
            Vo, dts = oracle.solve(oracle_problem(w), V0, w.T, w.cfl, nthreads=16)
            V = b.read_value(s)
            info = b.slot_info(s)  # each slot's time loop is FP64 bookkeeping
            assert info.steps == len(dts) and info.dt_last == dts[-1] and info.t == w.T
            assert float(np.abs(V - Vo).max()) <= 1e-4 * float(np.abs(V0).max())
            m = np.abs(Vo) >= 1e-3
            assert np.count_nonzero(np.sign(V[m]) != np.sign(Vo[m])) == 0


def test_batch_add_remove_between_advances_and_budget(hj):
    w1 = scenes.custom_workload((20, 20, 8, 16), n_circles=3, T=0.5, seed=1)
    w2 = scenes.custom_workload((16, 18, 6, 12), n_circles=2, T=0.3, seed=2)
    budget = hj.hj_batch_slot_bytes(w1.grid.n) + hj.hj_batch_slot_bytes(w2.grid.n)
    with hj.Batch(4, memory_budget=budget) as b:
        s1 = b.add_workload(w1)
        b.set_initial_value(s1, scenes.initial_value(w1.grid, w1.scene))
        b.set_horizon(s1, w1.T)
        st = b.advance(5)
        assert st.steps == 5 and st.active == 1
        s2 = b.add_workload(w2)  # admitted while s1 is mid-solve
        with pytest.raises(hj.HjError) as e:  # the budget is full now
            b.add_workload(w2)
        assert e.value.status == hj.HJ_ERR_OOM
        b.set_initial_value(s2, scenes.initial_value(w2.grid, w2.scene))
        b.set_horizon(s2, w2.T)
        b.advance()
        for s, w in ((s1, w1), (s2, w2)):
            ref, _ = single_grid(hj, w, scenes.initial_value(w.grid, w.scene))
            assert np.array_equal(b.read_value(s), ref)
        b.remove(s2)
        s3 = b.add_workload(w2)  # the freed memory is reusable
        b.set_initial_value(s3, scenes.initial_value(w2.grid, w2.scene))
        b.set_horizon(s3, 0.1)
        b.advance()
        assert b.slot_info(s3).t == 0.1 and b.slot_info(s1).t == w1.T


def test_batch_shapes_and_autotune_give_identical_bits(hj):
    ws = [scenes.custom_workload(n, n_circles=3, T=0.2, seed=7 + i) for i, n in enumerate(MIXED[:3])]
    v0s = [scenes.initial_value(w.grid, w.scene) for w in ws]
    results = []
    for shape in ((0, 0), (288, 1), (256, 3), (352, 1), (480, 2), (608, 4), (736, 1), ("tune", 0)):
        with hj.Batch(4) as b:
            slots = [b.add_workload(w) for w in ws]
            for s, v0 in zip(slots, v0s):
                b.set_initial_value(s, v0)
            if shape[0] == "tune":
                nc, ch, ms = b.autotune(3)
                assert nc > 0 and ms > 0
            else:
                b.set_shape(*shape)
            for s, w in zip(slots, ws):
                b.set_horizon(s, w.T)
            b.advance()
            results.append([b.read_value(s) for s in slots])
    for r in results[1:]:
        for a, c in zip(results[0], r):
            assert np.array_equal(a, c)


@pytest.mark.parametrize("shape, pieces", [((0, 0), 1), ((0, 0), 3), ((288, 2), 1)])
def test_batch_relayout_as_slots_finish(hj, shape, pieces):
    """Horizons from 0.1 to 1.2 s: as slots finish, the advance loop gives the
    remaining ones a new item layout (finer x chunks once they have fewer
    columns than CTAs).  Every slot still gives its single-grid solve's bits
    and step count, whether one advance call runs the whole solve or
    several calls with a step budget split it."""
    ns = [(44, 40, 16, 24), (30, 36, 12, 32), (50, 26, 18, 28), (24, 24, 10, 16), (40, 48, 20, 36), (36, 30, 14, 24)]
    Ts = [0.1, 1.2, 0.3, 0.9, 0.6, 1.0]
    ws = [scenes.custom_workload(n, n_circles=3, n_rects=1, T=T, seed=300 + i) for i, (n, T) in enumerate(zip(ns, Ts))]
    v0s = [scenes.initial_value(w.grid, w.scene) for w in ws]
    with hj.Batch(len(ws)) as b:
        slots = [b.add_workload(w) for w in ws]
        if shape != (0, 0):
            b.set_shape(*shape)
        for s, w, v0 in zip(slots, ws, v0s):
            b.set_initial_value(s, v0)
            b.set_horizon(s, w.T, w.cfl)
        if pieces == 1:
            st = b.advance()
        else:
            total = 0
            while True:
                st = b.advance(23)
                total += st.steps
                if st.active == 0:
                    break
        assert st.active == 0
        for s, w, v0 in zip(slots, ws, v0s):
            ref, rst = single_grid(hj, w, v0)
            info = b.slot_info(s)
            assert info.steps == rst.steps and info.t == w.T
            assert np.array_equal(b.read_value(s), ref), (s, w.grid.n)


def test_batch_advance_longer_than_one_launch(hj):
    """More batch steps than one launch runs (1024): the advance loop takes
    several launches, and the slots still give their single-grid solves'
    bits and step counts (one slot with about 1200 steps, one with a few)."""
    ws = [scenes.custom_workload((13, 11, 6, 8), n_circles=2, T=T, seed=500 + i) for i, T in enumerate((80.0, 0.5))]
    v0s = [scenes.initial_value(w.grid, w.scene) for w in ws]
    with hj.Batch(len(ws)) as b:
        slots = [b.add_workload(w) for w in ws]
        for s, w, v0 in zip(slots, ws, v0s):
            b.set_initial_value(s, v0)
            b.set_horizon(s, w.T, w.cfl)
        st = b.advance()
        assert st.active == 0 and st.launches >= 2, (st.steps, st.launches)
        for s, w, v0 in zip(slots, ws, v0s):
            ref, rst = single_grid(hj, w, v0)
            info = b.slot_info(s)
            assert info.steps == rst.steps and info.t == w.T
            assert np.array_equal(b.read_value(s), ref), s
        assert b.slot_info(slots[0]).steps > 1024


@pytest.mark.slow
def test_batch64_workload(hj):
    """The 64-instance workload: uneven grids (N1, N2 in {40, 50, 60}, N3 in
    [16, 24], N4 in [24, 36]), 4-16 circles each, T = 1.5 s.  Every slot
    matches its single-grid solve bit for bit, and the oracle's full solve of
    its grid within the FP32 tolerance, with no BRT sign flip and the
    oracle's step count and last dt."""
    ws = scenes.batch_workloads()
    with hj.Batch(len(ws)) as b:
        slots = []
        for w in ws:
            s = b.add_workload(w)
            b.set_initial_value(s, scenes.initial_value(w.grid, w.scene))
            b.set_horizon(s, w.T, w.cfl)
            slots.append(s)
        st = b.advance()
        assert st.active == 0
        worst = 0.0
        for i, w in enumerate(ws):
            V0 = scenes.initial_value(w.grid, w.scene)
            V = b.read_value(slots[i])
            ref, _ = single_grid(hj, w, V0)
            assert np.array_equal(V, ref), i
            Vo, dts = oracle.solve(oracle_problem(w), V0, w.T, w.cfl, nthreads=oracle.max_threads())
            info = b.slot_info(slots[i])
            assert info.steps == len(dts) and info.dt_last == dts[-1], i
            err = float(np.abs(V - Vo).max())
            assert err <= 1e-4 * float(np.abs(V0).max()), (i, err)
            m = np.abs(Vo) >= 1e-3
            assert np.count_nonzero(np.sign(V[m]) != np.sign(Vo[m])) == 0, i
            worst = max(worst, err)
        print(f"batch64: worst max|V - V_oracle| over 64 slots {worst:.3e}")


def test_batch_slot_with_negative_speeds(hj):
    """A slot whose speed axis runs through zero (v in [-1, 3]): x' = v cos(th)
    flips its upwind side where v < 0.  The slot equals the single-grid solve
    bit for bit and the oracle within the FP32 tolerance."""
    import math
    g = scenes.GridSpec((21, 17, 9, 16), lo=(-5.0, -5.0, -1.0, -math.pi), hi=(5.0, 5.0, 3.0, math.pi))
    w = scenes.Workload("negv", g, scenes.Scene(np.array([[0.5, -1.0, 0.7], [-2.0, 2.5, 0.9]])), 0.5, 0)
    V0 = scenes.initial_value(g, w.scene)
    with hj.Batch(2) as b:
        s = b.add_workload(w)
        b.set_initial_value(s, V0)
        b.set_horizon(s, w.T, w.cfl)
        b.advance()
        V = b.read_value(s)
    ref, _ = single_grid(hj, w, V0)
    assert np.array_equal(V, ref)
    Vo, _ = oracle.solve(oracle_problem(w), V0, w.T, w.cfl)
    assert float(np.abs(V - Vo).max()) <= 1e-4 * float(np.abs(V0).max())


def test_many_slots_set_in_one_call(hj):
    """hj_batch_set_initial_values_device and hj_batch_set_horizons: the V0
    and horizons of several slots in one call each (one synchronisation) give
    the same solve, bit for bit, as one call per slot; a NaN in one slot's V0 is reported with that slot, which is left
    without a value while the others are set."""
    import torch
    ws = [scenes.custom_workload(n, n_circles=3, T=0.25, seed=70 + i) for i, n in enumerate(MIXED[:4])]
    v0s = [torch.from_numpy(scenes.initial_value(w.grid, w.scene)).cuda().reshape(-1) for w in ws]
    out = []
    for together in (False, True):
        with hj.Batch(len(ws)) as b:
            slots = [b.add_workload(w) for w in ws]
            if together:
                b.set_initial_values(slots, v0s)
                b.set_horizons(slots, [w.T for w in ws], [w.cfl for w in ws])
            else:
                for s, v, w in zip(slots, v0s, ws):
                    b.set_initial_value(s, v)
                    b.set_horizon(s, w.T, w.cfl)
            b.advance()
            out.append([b.read_value(s) for s in slots])
    for a, c in zip(*out):
        assert np.array_equal(a, c)
    bad = v0s[2].clone()
    bad[17] = float("nan")
    with hj.Batch(len(ws)) as b:
        slots = [b.add_workload(w) for w in ws]
        with pytest.raises(hj.HjError) as e:
            b.set_initial_values(slots, [v0s[0], v0s[1], bad, v0s[3]])
        assert e.value.status == hj.HJ_ERR_INVALID_ARG and f"slot {slots[2]}" in str(e.value)
        with pytest.raises(hj.HjError) as e:  # that slot has no value
            b.set_horizon(slots[2], 0.1)
        assert e.value.status == hj.HJ_ERR_STATE
        b.set_horizon(slots[0], ws[0].T, ws[0].cfl)  # the others have theirs
        with pytest.raises(hj.HjError) as e:  # a count that does not match the slot's grid
            b.set_initial_values(slots[:1], [v0s[1]])
        assert e.value.status == hj.HJ_ERR_INVALID_ARG
