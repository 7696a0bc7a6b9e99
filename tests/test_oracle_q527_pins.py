"""Pins for the Q5.27 fixed-point oracle (Sec. III-C, Sec. IV-B): facts fixed
by the format, by hand-computed special cases and by the independently pinned
FP64 oracle, not by the fixed-point code itself.

  - the format: 27 fractional bits, 5 integer bits with the sign, so the range
    is [-16, 16) with resolution 2^-27 = 7.45e-9 (Sec. IV-B); conversion is
    nearest with ties to even and saturates;
  - closed forms: a linear field moved at constant speed on one axis with
    weight dt |xdot| / dx = 1/2 drops by a fixed number of codes per step,
    which pins the rounding rule (round half up: -1.5 codes -> -1) and the
    upwind side (a field rising downstream does not move);
  - invariants: zero dynamics leave V0 unchanged bit for bit, V <= V0 exactly,
    mirror symmetries of the car up to a few codes;
  - error bounds against the FP64 oracle: one step is within half a code plus
    the weight quantisation of the FP64 step from the same data, and a whole
    solve stays within the accumulated per-step bound.  A dropped axis, a
    wrong sign or a transposed stride moves V by ~1e-2, six orders above
    these bounds.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2012_04011_gb300 import scenes

ULP = 2.0 ** -27


@pytest.fixture(scope="module")
def oracle_mod():
    oracle.build()
    return oracle


def car_problem(grid, a_max=scenes.A_MAX, w_max=scenes.W_MAX):
    return oracle.Problem(grid.n, grid.lo, grid.hi, grid.periodic, oracle.DYN_CAR4D, (a_max, w_max))


# ---------------------------------------------------------------- the format

def test_conversion_follows_the_format(oracle_mod):
    x = np.array([0.0, 1.5, -1.5, 7.2, -16.0, 15.999999992549419, 16.0, -17.0, 1e9,
                  2.5 * ULP, 3.5 * ULP, -2.5 * ULP, 0.5 * ULP, 1.5 * ULP])
    q = oracle.to_q527(x)
    assert q.dtype == np.int32
    expect = [0, 3 << 26, -(3 << 26), round(7.2 * 2 ** 27), -2 ** 31, 2 ** 31 - 1, 2 ** 31 - 1, -2 ** 31,
              2 ** 31 - 1, 2, 4, -2, 0, 2]
    assert q.tolist() == expect
    # every code is exact in FP64
    codes = np.array([-2 ** 31, -12345, -1, 0, 1, 987654321, 2 ** 31 - 1], dtype=np.int32)
    back = oracle.from_q527(codes)
    assert back.tolist() == [c * ULP for c in codes.tolist()]
    assert np.array_equal(oracle.to_q527(back), codes)
    assert back[0] == -16.0 and back[-1] == 16.0 - ULP
    with pytest.raises(ValueError):
        oracle.to_q527([0.0, float("nan")])
    with pytest.raises(ValueError):
        oracle.to_q527([float("inf")])


# ---------------------------------------------------------------- closed forms

def _line_problem(c1):
    # x: 9 points on [0, 1] (dx = 1/8); the other axes do not move (c = 0)
    return oracle.Problem((9, 3, 3, 4), (0.0, 0.0, 0.0, -math.pi), (1.0, 2.0, 2.0, math.pi), 0b1000,
                          oracle.DYN_CONST, (c1, 0.0, 0.0, 0.0))


@pytest.mark.parametrize("c1, slope, per_step", [
    (1.0, -3, -1),   # upwind difference -3 codes x weight 1/2 = -1.5 -> -1 (half up)
    (1.0, -4, -2),   # exact: -2
    (1.0, -5, -2),   # -2.5 -> -2
    (1.0, +3, 0),    # the field rises downstream: +1.5 -> +2, then the BRT min keeps V0
    (-1.0, +3, -1),  # moving the other way picks the other neighbour
    (-1.0, -3, 0),
])
def test_linear_field_half_weight_rounds_half_up(oracle_mod, c1, slope, per_step):
    P = _line_problem(c1)
    # Courant number 1/2 with one moving axis: dt = (1/2) dx / |c1| = 1/16 and
    # dt |c1| / dx = 1/2 exactly (weight 2^29 with 30 fractional bits)
    i = np.arange(9)
    codes = (1 << 27) + slope * i  # 1.0 + slope codes per cell along x
    Q0 = np.broadcast_to(codes[:, None, None, None], P.n).astype(np.int32).copy()
    Q, t, dts = oracle.advance_q527(P, Q0, Q0, 0.0, 5 / 16, cfl=0.5)
    assert dts.tolist() == [1 / 16] * 5 and t == 5 / 16
    # the end cells use the extrapolated ghost, which continues the line
    assert np.array_equal(Q, Q0 + 5 * per_step)


def test_zero_dynamics_leave_v0_bitwise(oracle_mod):
    w = scenes.custom_workload((7, 8, 5, 12), n_circles=3)
    P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CONST, (0, 0, 0, 0))
    Q0 = oracle.to_q527(scenes.initial_value(w.grid, w.scene))
    Q, t, dts = oracle.advance_q527(P, Q0, Q0, 0.0, 0.7)
    assert len(dts) == 1 and t == 0.7  # nothing moves: one step to the horizon
    assert np.array_equal(Q, Q0)


# ---------------------------------------------------------------- invariants

def test_brt_min_is_exact(oracle_mod):
    w = scenes.custom_workload((11, 12, 6, 16), n_circles=4, T=0.6, seed=7)
    P = car_problem(w.grid)
    Q0 = oracle.to_q527(scenes.initial_value(w.grid, w.scene))
    Q = Q0
    for _ in range(6):
        Q, _, _ = oracle.advance_q527(P, Q0, Q, 0.0, 10.0, max_steps=1)
        assert np.all(Q <= Q0)


def test_mirror_symmetries(oracle_mod):
    """y -> -y with th -> -th, x -> -x with th -> pi - th, x <-> y with
    th -> pi/2 - th.  FP64 cos/sin of the mirrored angles can differ in the
    last bit, which moves a weight by one unit of 2^-30 at most, so the
    mirrored solve agrees to a few codes (an index or stride mistake moves it
    by ~1e6 codes)."""
    N4 = 16
    w = scenes.custom_workload((21, 21, 5, N4), n_circles=4, T=0.5, seed=123)
    P = car_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    Q, _ = oracle.solve_q527(P, V0, w.T, nthreads=4)
    l = np.arange(N4)
    perms = {
        "y": (lambda A: A[:, ::-1, :, :][..., (N4 - l) % N4]),
        "x": (lambda A: A[::-1, :, :, :][..., (N4 // 2 - l) % N4]),
        "xy": (lambda A: A.transpose(1, 0, 2, 3)[..., (N4 // 4 - l) % N4]),
    }
    for name, f in perms.items():
        Qm, _ = oracle.solve_q527(P, np.ascontiguousarray(f(V0)), w.T, nthreads=4)
        err = int(np.abs(Qm.astype(np.int64) - f(Q).astype(np.int64)).max())
        assert err <= 8, (name, err)


# ---------------------------------------------------------------- against FP64

def _per_step_bound_codes(V_abs_max):
    """Per step: the final rounding (<= 1/2 code) plus, on each of the four
    axes, the weight error (<= 2^-31) times the upwind difference (<= 2 max|V|
    with the extrapolated ghosts), in codes."""
    return 0.5 + 4 * (2.0 ** -31) * (2 * V_abs_max) / ULP


def test_one_step_within_half_code_of_fp64(oracle_mod):
    w = scenes.custom_workload((13, 11, 7, 12), n_circles=3, n_rects=1, seed=5)
    P = car_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    Q0 = oracle.to_q527(V0)
    Q1, _, dts = oracle.advance_q527(P, Q0, Q0, 0.0, 10.0, max_steps=3)
    Q2, _, d2 = oracle.advance_q527(P, Q0, Q1, 0.0, 10.0, max_steps=1)
    # the FP64 scheme, one step of the same dt from the same (exact) values
    cells = np.arange(Q1.size)
    ref = oracle.step_cells(P, oracle.from_q527(Q1), oracle.from_q527(Q0), d2[0], cells)
    err = np.abs(oracle.from_q527(Q2).ravel() - ref) / ULP
    # per cell: 1/2 code of rounding + weight quantisation of the actual differences
    assert err.max() <= _per_step_bound_codes(np.abs(V0).max()) + 1e-6, err.max()
    # and on most cells only the rounding shows
    assert np.quantile(err, 0.99) <= 0.5 + 0.05


@pytest.mark.parametrize("name", ["car4d_31x31x11x16", "car4d_60x60x20x36"])
def test_solve_within_accumulated_bound_of_fp64(oracle_mod, name):
    """The scheme is a convex combination followed by a min, so it does not
    amplify differences in max norm: the fixed-point solve stays within
    1/2 code (conversion) + steps x the per-step bound of the FP64 solve.
    (Sec. IV-B reports 1.4e-6..1.8e-6 between the FPGA and an FP32 toolbox.)"""
    w = scenes.workload(name)
    P = car_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    Q, dq = oracle.solve_q527(P, V0, w.T, w.cfl, nthreads=oracle.max_threads())
    V, dv = oracle.solve(P, V0, w.T, w.cfl, nthreads=oracle.max_threads())
    assert np.array_equal(dq, dv)  # the FP64 dt sequence
    err = np.abs(oracle.from_q527(Q) - V).max() / ULP
    bound = 0.5 + len(dv) * _per_step_bound_codes(np.abs(V0).max())
    assert err <= bound, (err, bound)
    assert err * ULP < 1e-6


def test_steer_q527_within_bound_of_fp64(oracle_mod):
    """The fixed-point variant of the steering car (per-speed heading weight)
    stays within the accumulated per-step bound of the FP64 steering solve."""
    w = scenes.custom_workload((21, 19, 9, 16), n_circles=4, T=0.6, seed=12)
    P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D_STEER,
                       (1.5, math.pi / 18, 0.3))
    V0 = scenes.initial_value(w.grid, w.scene)
    Q, dq = oracle.solve_q527(P, V0, w.T, w.cfl)
    V, dv = oracle.solve(P, V0, w.T, w.cfl)
    assert np.array_equal(dq, dv)
    err = np.abs(oracle.from_q527(Q) - V).max() / ULP
    assert err <= 0.5 + len(dv) * _per_step_bound_codes(np.abs(V0).max()), err
    # one step from the same data: half a code plus the weight quantisation
    Q1, _, d1 = oracle.advance_q527(P, oracle.to_q527(V0), Q, 0.0, 10.0, max_steps=1)
    ref = oracle.step_cells(P, oracle.from_q527(Q), oracle.from_q527(oracle.to_q527(V0)), d1[0], np.arange(Q.size))
    e1 = np.abs(oracle.from_q527(Q1).ravel() - ref) / ULP
    assert e1.max() <= _per_step_bound_codes(np.abs(V0).max()) + 1e-6


def test_converged_q527_matches_fixed_steps(oracle_mod):
    """The fixed-point convergence loop takes the fixed-point steps; its eps is
    the largest code change of the last step times 2^-27."""
    w = scenes.custom_workload((13, 13, 6, 12), n_circles=3, seed=22)
    P = car_problem(w.grid)
    Q0 = oracle.to_q527(scenes.initial_value(w.grid, w.scene))
    Q, t, dts, eps, conv = oracle.advance_converged_q527(P, Q0, Q0, 0.0, 3e-3, 30.0)
    assert conv and eps < 3e-3
    n = len(dts)
    Qa, t1, _ = oracle.advance_q527(P, Q0, Q0, 0.0, 30.0, max_steps=n - 1)
    Qb, _, _ = oracle.advance_q527(P, Q0, Qa, t1, 30.0, max_steps=1)
    assert np.array_equal(Qb, Q)
    assert eps == float(np.abs(Qb.astype(np.int64) - Qa).max()) * ULP
