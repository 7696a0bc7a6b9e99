"""GPU parity of the query helper (value, gradient and u_opt at arbitrary
states; Eq. uopt_max, Eq. closetoboundary) against the oracle's query on the
same grid values: 1e-12 on values and gradients, identical controls wherever
the deciding derivative is not within rounding of zero."""
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


def states_for(w, m, seed):
    rng = np.random.default_rng(seed)
    lo, hi = np.array(w.grid.lo), np.array(w.grid.hi)
    s = lo + (hi - lo) * rng.random((m, 4))
    s[: m // 10, 3] += 2 * math.pi * rng.integers(-2, 3, m // 10)  # headings outside [-pi, pi)
    s[m // 10: m // 5, 0] = hi[0] + rng.random(m // 10)          # beyond the x range
    return s


def check(P, Vgrid, s, val, grad, ctl):
    vo, go, co = oracle.query(P, Vgrid, s)
    scale = max(1.0, float(np.abs(Vgrid).max()))
    assert np.abs(val - vo).max() <= 1e-12 * scale
    assert np.abs(grad - go).max() <= 1e-9 * scale
    for d, col in ((2, 0), (3, 1)):
        sure = np.abs(go[:, d]) > 1e-9 * scale
        assert np.array_equal(ctl[sure, col], co[sure, col])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "q527"])
def test_query_matches_oracle(hj, prec):
    w = scenes.workload("car4d_31x31x11x16")
    p = {"fp64": hj.HJ_FP64, "fp32": hj.HJ_FP32, "q527": hj.HJ_Q527}[prec]
    s = states_for(w, 5000, 1)
    for dyn, params, odyn in ((hj.HJ_DYN_CAR4D, (w.a_max, w.w_max), oracle.DYN_CAR4D),
                              (hj.HJ_DYN_CAR4D_STEER, (1.5, math.pi / 18, 0.3), oracle.DYN_CAR4D_STEER)):
        with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, p) as g:
            g.set_dynamics(dyn, params)
            g.set_initial_value(scenes.initial_value(w.grid, w.scene))
            g.solve_brt(0.5, w.cfl)
            Vg = g.read_value()  # exact FP64 image of the grid's values
            val, grad, ctl = hj.hj_query(g.handle, s)
        P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, odyn, params)
        check(P, Vg, s, val, grad, ctl)


def test_query_device_equals_host_and_chunks(hj):
    import torch
    w = scenes.workload("car4d_60x60x20x36")
    s = states_for(w, 20000, 2)
    with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
        g.set_initial_value(scenes.initial_value(w.grid, w.scene))
        g.solve_brt(0.3, w.cfl)
        val, grad, ctl = hj.hj_query(g.handle, s)
        sd = torch.from_numpy(s).cuda()
        vd = torch.empty(len(s), dtype=torch.float64, device="cuda")
        gd = torch.empty((len(s), 4), dtype=torch.float64, device="cuda")
        cd = torch.empty((len(s), 2), dtype=torch.float64, device="cuda")
        hj.hj_query_device(g.handle, sd, vd, gd, cd)
        assert np.array_equal(vd.cpu().numpy(), val)
        assert np.array_equal(gd.cpu().numpy(), grad)
        assert np.array_equal(cd.cpu().numpy(), ctl)
    # a tiny grid stages only a few states per chunk (its free buffer is small)
    wt = scenes.custom_workload((3, 3, 3, 4), n_circles=1, seed=9)
    st = states_for(wt, 100, 3)
    with hj.Grid(wt.grid.n, wt.grid.lo, wt.grid.hi, wt.grid.periodic, hj.HJ_FP32) as g:
        g.set_dynamics(hj.HJ_DYN_CAR4D, (1.5, 1.0))
        g.set_initial_value(scenes.initial_value(wt.grid, wt.scene))
        g.solve_brt(0.2, 0.8)
        val, grad, ctl = hj.hj_query(g.handle, st)
        P = oracle.Problem(wt.grid.n, wt.grid.lo, wt.grid.hi, wt.grid.periodic, oracle.DYN_CAR4D, (1.5, 1.0))
        check(P, g.read_value(), st, val, grad, ctl)


def test_query_errors(hj):
    w = scenes.workload("car4d_31x31x11x16")
    with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP32) as g:
        with pytest.raises(hj.HjError) as e:
            hj.hj_query(g.handle, np.zeros((3, 4)))
        assert e.value.status == hj.HJ_ERR_STATE  # no V0
        g.set_initial_value_xy(scenes.signed_distance_xy(w.grid, w.scene))
        val, _, _ = hj.hj_query(g.handle, np.zeros((3, 4)), want_control=False)  # no dynamics needed
        with pytest.raises(hj.HjError) as e:
            hj.hj_query(g.handle, np.zeros((3, 4)))
        assert e.value.status == hj.HJ_ERR_STATE  # control without dynamics
        assert hj.hj_query(g.handle, np.zeros((0, 4)), want_control=False)[0].size == 0
