"""Pins for the FP64 oracle: facts fixed by the paper and by the mathematics,
not by the oracle's own code.

Each test names what a plausible mistake in the oracle would look like and
why the test would catch it:
  - closed forms: a linear field advected at constant speed drops by exactly
    t; a disk translated at constant velocity has the point-to-segment
    distance as exact BRT value (first-order convergence towards it);
  - textbook special cases: at Courant number 1 on one axis, first-order
    upwind is an exact one-cell shift (wrong dissipation sign, dropped
    dissipation, wrong dt, wrong axis or wrong wrap all break it); at
    Courant number 1 on two axes it is an exact convex combination;
  - invariants: V <= V0, zero dynamics leave V0 unchanged bit for bit,
    the maximising control never lowers V on monotone data, mirror
    symmetries of the car, OpenMP thread count does not change a bit;
  - the paper's own numbers: horizon 0.5 s with a 0.007497 s step is 67
    iterations (Sec. IV-A, Tables II-III).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2012_04011_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def car_problem(grid, a_max=scenes.A_MAX, w_max=scenes.W_MAX):
    return oracle.Problem(grid.n, grid.lo, grid.hi, grid.periodic, oracle.DYN_CAR4D, (a_max, w_max))


def const_problem(n, c, lo=(-5.0, -4.0, 0.0, -math.pi), hi=(5.0, 4.0, 4.0, math.pi), periodic=0b1000):
    return oracle.Problem(n, lo, hi, periodic, oracle.DYN_CONST, c)


# ---------------------------------------------------------------- grid


def test_grid_conventions(oracle_mod):
    """x_i = lo + i (hi-lo)/(N-1) with both ends on the grid; theta_l =
    -pi + l 2pi/N on the periodic axis (theta in [-pi, pi))."""
    P = car_problem(scenes.GridSpec((31, 31, 11, 16)))
    assert P.spacing(0) == pytest.approx(10.0 / 30.0, abs=0)
    assert P.coord(0, 0) == -5.0
    assert P.coord(0, 30) == pytest.approx(5.0, abs=1e-14)
    assert P.coord(2, 10) == pytest.approx(4.0, abs=1e-14)
    assert P.spacing(3) == pytest.approx(2 * math.pi / 16, abs=1e-16)
    assert P.coord(3, 0) == -math.pi
    assert P.coord(3, 8) == pytest.approx(0.0, abs=1e-15)


# ---------------------------------------------------------------- closed forms


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)])
def test_linear_field_drops_by_t(oracle_mod, axis, sign):
    """Constant velocity of size |c| along -sign*e_d with V0 = sign*x_d - 3:
    the flow runs down the slope of V0, so the exact BRT value is
    V0 - |c| t.  Linear extrapolation at the ends
    is exact for linear data, so every cell, boundary included, must match.
    Catches a wrong time accumulation, a wrong dt, a wrong extrapolation and a
    velocity applied on the wrong axis."""
    n = (9, 7, 6, 4)
    c = [0.0, 0.0, 0.0, 0.0]
    speed = 1.3
    # moving along -sign*e_d makes V0 = sign*x_d - 3 fall at rate speed
    c[axis] = -sign * speed
    P = const_problem(n, c)
    coords = P.coords(axis)
    shape = [1, 1, 1, 1]
    shape[axis] = n[axis]
    V0 = np.broadcast_to((sign * coords - 3.0).reshape(shape), n).copy()
    T = 0.9
    V, dts = oracle.solve(P, V0, T, cfl=0.8)
    assert sum(dts) == pytest.approx(T, abs=1e-14)
    np.testing.assert_allclose(V, V0 - speed * T, rtol=0, atol=1e-13)


def _segment_distance(px, py, fx, fy, T, cx, cy):
    """Distance from (cx, cy) to the segment p + f s, s in [0, T]."""
    dx, dy = fx * T, fy * T
    L2 = dx * dx + dy * dy
    s = np.where(L2 > 0, ((cx - px) * dx + (cy - py) * dy) / np.where(L2 > 0, L2, 1.0), 0.0)
    s = np.clip(s, 0.0, 1.0)
    qx, qy = px + s * dx - cx, py + s * dy - cy
    return np.sqrt(qx * qx + qy * qy)


def test_translation_closed_form_first_order(oracle_mod):
    """Car with a_max = w_max = 0: each (v, theta) slice translates at
    (v cos th, v sin th).  The exact BRT value is min_{s in [0,T]} V0(p + f s)
    = point-to-segment distance to the disk centre minus R (Eq. eq3 with
    Eq. init_V).  The first-order scheme must converge at order ~1 in L1 and
    at least 1/2 in L-inf on cells whose characteristic stays inside the
    domain.  Catches a reversed advection direction (x - f s), cos/sin swapped,
    and any unstable or inconsistent combination of H and dissipation."""
    cx, cy, R, T = 0.5, -0.3, 1.0, 1.0
    errs_inf, errs_l1 = [], []
    for N in (21, 41, 81):
        grid = scenes.GridSpec((N, N, 3, 8), lo=(-5.0, -5.0, 0.0, -math.pi), hi=(5.0, 5.0, 2.0, math.pi))
        P = car_problem(grid, 0.0, 0.0)
        sc = scenes.Scene(circles=np.array([[cx, cy, R]]))
        V0 = scenes.initial_value(grid, sc)
        V, _ = oracle.solve(P, V0, T, cfl=0.8, nthreads=4)
        x = P.coords(0)[:, None, None, None]
        y = P.coords(1)[None, :, None, None]
        v = P.coords(2)[None, None, :, None]
        th = P.coords(3)[None, None, None, :]
        fx, fy = v * np.cos(th), v * np.sin(th)
        dist = _segment_distance(x, y, fx, fy, T, cx, cy)
        exact = dist - R
        inside = (np.abs(x) <= 2.5) & (np.abs(y) <= 2.5)
        err = np.abs(V - exact)
        errs_l1.append(err[np.broadcast_to(inside, V.shape)].mean())
        # the exact value has a kink where the segment passes the centre;
        # the max-norm order is measured away from it
        smooth = np.broadcast_to(inside & (dist > 0.5), V.shape)
        errs_inf.append(err[smooth].max())
    for k in range(2):
        assert math.log2(errs_l1[k] / errs_l1[k + 1]) > 0.75, errs_l1
        assert math.log2(errs_inf[k] / errs_inf[k + 1]) > 0.5, errs_inf
    assert errs_inf[-1] < 0.2


# ---------------------------------------------------------------- textbook cases


def _shift(E, axis, direction, periodic):
    """E at index i + direction along axis; past the end: wrap (periodic) or
    the linear extrapolation 2 E_end - E_(end-1)."""
    out = np.roll(E, -direction, axis=axis)
    if not periodic:
        N = E.shape[axis]
        end = N - 1 if direction > 0 else 0
        nxt = N - 2 if direction > 0 else 1
        sl = [slice(None)] * 4
        sl[axis] = end
        sn = list(sl)
        sn[axis] = nxt
        out[tuple(sl)] = 2.0 * E[tuple(sl)] - E[tuple(sn)]
    return out


@pytest.mark.parametrize("axis", [0, 1, 2, 3])
@pytest.mark.parametrize("sign", [1, -1])
def test_courant_one_is_exact_shift(oracle_mod, axis, sign):
    """Textbook: for xdot = c e_d, first-order upwind at Courant number
    |c| dt / dx = 1 moves the data exactly one cell per step (V_i <- V_{i+1}
    for c > 0, V_i <- V_{i-1} for c < 0), here followed by the BRT min.  The
    input is white noise, so nothing but an exact shift passes.  Catches the
    sign of the dissipation (the printed minus sign gives 2 V_i - V_{i-1}), a
    dropped dissipation (central difference), a wrong CFL dt, a transposed
    axis or stride, a wrong periodic wrap and a wrong extrapolation."""
    n = (6, 7, 5, 8)
    c = [0.0] * 4
    c[axis] = 1.7 * sign
    P = const_problem(n, c)
    rng = np.random.default_rng(7 + axis)
    V0 = rng.uniform(-1.0, 1.0, size=n)
    steps = 4
    V, _, dts = oracle.advance(P, V0, V0, 0.0, 1e9, cfl=1.0, max_steps=steps)
    assert len(dts) == steps
    E = V0.copy()
    for _ in range(steps):
        E = np.minimum(V0, _shift(E, axis, 1 if sign > 0 else -1, axis == 3))
    np.testing.assert_allclose(V, E, rtol=0, atol=1e-13)


def test_courant_one_two_axes_convex_combination(oracle_mod):
    """Textbook: with velocity on two axes and sum_d |c_d| dt/dx_d = 1, one
    upwind step is the convex combination lam_1 V(i+1) + lam_2 V(j-1) with
    lam_d = |c_d| dt/dx_d.  Pins the CFL sum over axes and the per-axis
    weights."""
    n = (6, 7, 5, 8)
    c = (1.1, -0.6, 0.0, 0.0)
    P = const_problem(n, c)
    rng = np.random.default_rng(11)
    V0 = rng.uniform(-1.0, 1.0, size=n)
    V, _, dts = oracle.advance(P, V0, V0, 0.0, 1e9, cfl=1.0, max_steps=1)
    h0, h1 = P.spacing(0), P.spacing(1)
    lam0 = abs(c[0]) / h0 / (abs(c[0]) / h0 + abs(c[1]) / h1)
    lam1 = 1.0 - lam0
    E = lam0 * _shift(V0, 0, +1, False) + lam1 * _shift(V0, 1, -1, False)
    np.testing.assert_allclose(V, np.minimum(V0, E), rtol=0, atol=1e-13)


# ---------------------------------------------------------------- invariants


def test_zero_dynamics_leave_v0_bitwise(oracle_mod):
    """xdot = 0: nothing moves, the CFL sum is 0, one step straight to T, and
    V(T) = V0 bit for bit."""
    n = (5, 6, 4, 8)
    P = const_problem(n, (0.0, 0.0, 0.0, 0.0))
    V0 = np.random.default_rng(3).normal(size=n)
    V, dts = oracle.solve(P, V0, 0.7)
    assert len(dts) == 1 and dts[0] == 0.7
    assert np.array_equal(V, V0)


def test_zero_speed_slice_unchanged(oracle_mod):
    """Car with a_max = w_max = 0: the v = 0 slice has xdot = 0 and must keep
    V0 bit for bit for the whole horizon."""
    w = scenes.custom_workload((15, 15, 5, 8), n_circles=3, T=0.6)
    P = car_problem(w.grid, 0.0, 0.0)
    V0 = scenes.initial_value(w.grid, w.scene)
    V, _ = oracle.solve(P, V0, w.T)
    assert np.array_equal(V[:, :, 0, :], V0[:, :, 0, :])
    assert not np.array_equal(V[:, :, 1, :], V0[:, :, 1, :])


@pytest.mark.parametrize("slope", [1.0, -1.0])
def test_maximising_control_keeps_monotone_speed_target(oracle_mod, slope):
    """V0 = slope*(v - 2) depends only on speed.  The control maximises
    grad(V).f (Eq. uopt_max; Eq. eq3 with the control avoiding the target), so
    it always accelerates away from the target and V stays V0 exactly.  An
    argmin control would lower V at rate a_max."""
    grid = scenes.GridSpec((5, 5, 9, 8))
    P = car_problem(grid)
    v = P.coords(2)
    V0 = np.broadcast_to((slope * (v - 2.0))[None, None, :, None], grid.n).copy()
    V, dts = oracle.solve(P, V0, 0.4)
    assert len(dts) > 3
    assert np.array_equal(V, V0)


def test_maximising_heading_control_only_lowers_ridge(oracle_mod):
    """V0 = cos(theta): after one step only the ridge (theta = 0, where no
    heading change can raise V) may fall; every other heading turns uphill and
    keeps V0 exactly.  An argmin heading control would lower every cell."""
    grid = scenes.GridSpec((4, 4, 3, 16))
    P = car_problem(grid)
    th = P.coords(3)
    V0 = np.broadcast_to(np.cos(th)[None, None, None, :], grid.n).copy()
    V, _, _ = oracle.advance(P, V0, V0, 0.0, 10.0, max_steps=1)
    ridge = 8
    others = [l for l in range(16) if l != ridge]
    assert np.array_equal(V[..., others], V0[..., others])
    assert np.all(V[..., ridge] < V0[..., ridge])


def test_brt_min_bounds_and_monotone_in_time(oracle_mod):
    """V_{n+1} <= V0 exactly (the min of Algorithm 2).  The interior update
    is monotone under CFL <= 1 and the min preserves order, so V_{n+1} <= V_n
    holds on every cell that no extrapolated point has reached yet.  Linear
    extrapolation is not monotone (at an edge it can raise V), and its effect
    spreads one cell per step, so step s is checked on cells more than s
    cells from every non-periodic edge."""
    w = scenes.custom_workload((25, 25, 21, 16), n_circles=5, T=1.0, seed=77)
    P = car_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    V = V0.copy()
    t = 0.0
    rise_anywhere = 0.0
    for s in range(8):
        Vn, t, _ = oracle.advance(P, V0, V, t, w.T, max_steps=1)
        assert np.all(Vn <= V0)
        m = s + 1
        inner = (slice(m, -m), slice(m, -m), slice(m, -m), slice(None))
        assert (Vn - V)[inner].max() <= 1e-14 * np.abs(V0).max()
        rise_anywhere = max(rise_anywhere, (Vn - V).max())
        V = Vn
    # the edge band does rise, so the restriction above is needed
    assert rise_anywhere > 1e-6


def test_mirror_symmetries(oracle_mod):
    """The car is symmetric under y -> -y with th -> -th, x -> -x with
    th -> pi - th, and x <-> y with th -> pi/2 - th.  Mirroring the input
    (a 4D index permutation) must mirror the output.  Catches cos and sin
    swapped, a sign error in one velocity component and transposed x/y
    strides."""
    N4 = 16
    w = scenes.custom_workload((21, 21, 5, N4), n_circles=4, T=0.5, seed=123)
    P = car_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    V, _ = oracle.solve(P, V0, w.T, nthreads=4)
    l = np.arange(N4)
    perms = {
        "y": (lambda A: A[:, ::-1, :, :][..., (N4 - l) % N4]),
        "x": (lambda A: A[::-1, :, :, :][..., (N4 // 2 - l) % N4]),
        "xy": (lambda A: A.transpose(1, 0, 2, 3)[..., (N4 // 4 - l) % N4]),
    }
    scale = np.abs(V0).max()
    for name, f in perms.items():
        Vm, _ = oracle.solve(P, np.ascontiguousarray(f(V0)), w.T, nthreads=4)
        err = np.abs(Vm - f(V)).max()
        assert err <= 1e-12 * scale, (name, err)


def test_openmp_bit_identical(oracle_mod):
    w = scenes.workload("car4d_31x31x11x16")
    P = car_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    V1, d1 = oracle.solve(P, V0, 0.3, nthreads=1)
    V8, d8 = oracle.solve(P, V0, 0.3, nthreads=8)
    assert np.array_equal(V1, V8) and np.array_equal(d1, d8)


def test_step_cells_matches_full_step(oracle_mod):
    w = scenes.custom_workload((9, 10, 6, 12), n_circles=3)
    P = car_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    V1, _, _ = oracle.advance(P, V0, V0, 0.0, 5.0, max_steps=2)
    V2, _, dts = oracle.advance(P, V0, V1, 0.0, 5.0, max_steps=1)
    cells = np.random.default_rng(0).choice(V0.size, 200, replace=False)
    got = oracle.step_cells(P, V1, V0, dts[0], cells)
    assert np.array_equal(got, V2.reshape(-1)[cells])


# ---------------------------------------------------------------- convergence


def test_full_car_self_convergence(oracle_mod):
    """No closed form with a_max, w_max > 0: nested refinements (N, 2N-1 on
    x, y, v; 2N on the periodic theta) must have shrinking differences at the
    common nodes (observed order > 0.5)."""
    sc = scenes.Scene(circles=np.array([[0.7, 0.2, 1.0], [-2.0, -1.5, 0.6]]))
    sols = []
    for (nx, nv, nt) in ((11, 5, 8), (21, 9, 16), (41, 17, 32)):
        grid = scenes.GridSpec((nx, nx, nv, nt))
        P = car_problem(grid)
        V, _ = oracle.solve(P, scenes.initial_value(grid, sc), 0.5, nthreads=8)
        sols.append(V)
    d1 = np.abs(sols[0] - sols[1][::2, ::2, ::2, ::2])
    d2 = np.abs(sols[1][::2, ::2, ::2, ::2] - sols[2][::4, ::4, ::4, ::4])
    assert math.log2(d1.mean() / d2.mean()) > 0.5, (d1.mean(), d2.mean())
    assert d2.max() < d1.max()


# ---------------------------------------------------------------- paper numbers


def test_paper_iteration_count():
    """Sec. IV-A: horizon 0.5 s, largest stable step 0.007497 s; Tables II-III:
    67 iterations.  With the step fixed at 0.007497 s the time loop must take
    ceil(0.5/0.007497) = 67 steps, the last one cut to land on 0.5 s."""
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as f:
        g = json.load(f)
    dt_target, T, iters = g["max_stable_dt_s"], g["horizon_s"], g["iterations"]
    n = (8, 6, 5, 4)
    cfl = 0.8
    P0 = const_problem(n, (1.0, 0, 0, 0))
    c1 = cfl * P0.spacing(0) / dt_target  # S = c1/h1, dt = cfl/S
    P = const_problem(n, (c1, 0, 0, 0))
    V0 = np.random.default_rng(1).uniform(size=n)
    _, dts = oracle.solve(P, V0, T, cfl=cfl)
    assert len(dts) == iters
    assert dts[0] == pytest.approx(dt_target, rel=1e-14)
    assert sum(dts) == pytest.approx(T, abs=1e-15)
    assert 0 < dts[-1] < dt_target


def test_paper_room_workload(oracle_mod):
    """The paper's experiment as the bench rebuilds it (Sec. IV-A): spacings
    0.1 m, 0.067 m, 0.2 m/s and 2 pi/36 rad on 60x60x20x36 points, the
    steering car, and the Courant number that makes the oracle's CFL step the
    reported 0.007497 s, so the 0.5 s horizon takes the 67 iterations of
    Tables II-III."""
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as f:
        g = json.load(f)
    w = scenes.paper_room(1)
    assert tuple(w.grid.n) == tuple(g["grid"]) and w.T == g["horizon_s"]
    h = [(w.grid.hi[d] - w.grid.lo[d]) / (w.grid.n[d] - 1) for d in range(3)]
    assert h == pytest.approx([0.1, 0.067, 0.2], rel=1e-12)
    assert (w.grid.hi[3] - w.grid.lo[3]) / w.grid.n[3] == pytest.approx(2 * math.pi / 36, rel=1e-15)
    P = steer_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    _, am = oracle.rate(P, V0)
    assert oracle.cfl_dt(P, am, w.cfl) == pytest.approx(g["max_stable_dt_s"], rel=1e-12)
    _, _, dts = oracle.advance(P, V0, V0, 0.0, w.T, w.cfl, max_steps=2)
    assert dts[0] == pytest.approx(g["max_stable_dt_s"], rel=1e-12)
    assert math.ceil(w.T / dts[0]) == g["iterations"]
    # the cones lie in the room and V0 is the distance to the nearest inflated cone
    assert np.all(w.scene.circles[:, 2] == 0.75)
    assert float(V0.min()) < 0 < float(V0.max()) < 16.0  # inside the Q5.27 range (Sec. IV-B)


@pytest.mark.parametrize("name,steps", [("car4d_31x31x11x16", 38), ("car4d_60x60x20x36", 151)])
def test_car_cfl_step(oracle_mod, name, steps):
    """For the car on [-5,5]^2 x [0,4] x [-pi,pi): alpha^max = (max|v cos th|,
    max|v sin th|, a_max, w_max) = (4, 4, 1.5, 1) exactly (theta = -pi and
    -pi/2 are grid points), so dt = 0.8 / (4/dx + 4/dy + 1.5/dv + 1/dth)."""
    w = scenes.workload(name)
    P = car_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    L, am = oracle.rate(P, V0)
    assert tuple(am) == (4.0, 4.0, 1.5, 1.0)
    h = [10.0 / (w.grid.n[0] - 1), 10.0 / (w.grid.n[1] - 1), 4.0 / (w.grid.n[2] - 1), 2 * math.pi / w.grid.n[3]]
    dt = 0.8 / (4 / h[0] + 4 / h[1] + 1.5 / h[2] + 1 / h[3])
    assert oracle.cfl_dt(P, am, 0.8) == pytest.approx(dt, rel=1e-15)
    assert math.ceil(w.T / dt) == steps


# ---------------------------------------------------------------- steering form (Eq. car_dynamics)

STEER = (1.5, math.pi / 18, 0.3)  # a in [-1.5, 1.5], delta in [-pi/18, pi/18], L = 0.3 m (Sec. IV-A)


def steer_problem(grid, a_max=STEER[0], d_max=STEER[1], L=STEER[2]):
    return oracle.Problem(grid.n, grid.lo, grid.hi, grid.periodic, oracle.DYN_CAR4D_STEER, (a_max, d_max, L))


def test_steer_zero_angle_is_car_without_turning(oracle_mod):
    """delta_max = 0: th' = 0 for every control, which is the heading-rate car
    with w_max = 0, bit for bit."""
    w = scenes.custom_workload((13, 11, 7, 12), n_circles=3, T=0.5, seed=4)
    V0 = scenes.initial_value(w.grid, w.scene)
    Vs, ds = oracle.solve(steer_problem(w.grid, d_max=0.0), V0, w.T)
    Vc, dc = oracle.solve(car_problem(w.grid, scenes.A_MAX, 0.0), V0, w.T)
    assert np.array_equal(ds, dc) and np.array_equal(Vs, Vc)


def test_steer_slice_is_car_with_speed_dependent_turn_rate(oracle_mod):
    """With a_max = 0 no cell moves in v, so on the slice v = v_k the steering
    car is the heading-rate car with w_max = v_k tan(delta_max) / L: one step
    of the same dt agrees bit for bit on that slice.  A missing v factor, a
    wrong L, sin for tan or an argmin steering angle breaks it."""
    w = scenes.custom_workload((9, 10, 6, 16), n_circles=3, seed=8)
    V0 = scenes.initial_value(w.grid, w.scene)
    rng = np.random.default_rng(3)
    V = V0 + 0.05 * rng.standard_normal(V0.shape)  # a V that depends on theta too
    Ps = steer_problem(w.grid, a_max=0.0)
    dt = 0.01
    for k in (0, 2, 5):
        vk = Ps.coord(2, k)
        Pc = car_problem(w.grid, 0.0, vk * math.tan(STEER[1]) / STEER[2])
        cells = np.array([((i * 10 + j) * 6 + k) * 16 + l for i in range(9) for j in range(10) for l in range(16)])
        assert np.array_equal(oracle.step_cells(Ps, V, V0, dt, cells), oracle.step_cells(Pc, V, V0, dt, cells)), k


def test_steer_cfl_alpha_closed_form(oracle_mod):
    """alpha^max of the steering car: (max|v cos|, max|v sin|, a_max,
    v_max tan(delta_max) / L)."""
    grid = scenes.GridSpec((5, 5, 9, 8))
    P = steer_problem(grid)
    _, am = oracle.rate(P, np.zeros(grid.n))
    vmax = P.coord(2, grid.n[2] - 1)
    assert am[0] == vmax and am[2] == STEER[0]
    assert am[3] == vmax * math.tan(STEER[1]) / STEER[2]
    assert abs(am[1] - vmax) < 1e-12  # sin reaches 1 at theta = -pi/2 up to rounding


def test_steer_mirror_symmetry(oracle_mod):
    """y -> -y with th -> -th maps the steering car onto itself (delta -> -delta)."""
    N4 = 16
    w = scenes.custom_workload((17, 17, 5, N4), n_circles=3, T=0.5, seed=31)
    P = steer_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    V, _ = oracle.solve(P, V0, w.T, nthreads=4)
    l = np.arange(N4)
    f = lambda A: A[:, ::-1, :, :][..., (N4 - l) % N4]
    Vm, _ = oracle.solve(P, np.ascontiguousarray(f(V0)), w.T, nthreads=4)
    assert np.abs(Vm - f(V)).max() <= 1e-12 * np.abs(V0).max()


# ---------------------------------------------------------------- convergence test (Algorithm 2)

def test_converged_stops_at_once_when_nothing_changes(oracle_mod):
    """V0 = slope (v - 2) is a fixed point of the maximising car (see the
    speed-target test): the first step changes nothing, so the convergence
    test stops after one step with eps = 0."""
    grid = scenes.GridSpec((5, 5, 9, 8))
    P = car_problem(grid)
    v = P.coords(2)
    V0 = np.broadcast_to((v - 2.0)[None, None, :, None], grid.n).copy()
    V, t, dts, eps, conv = oracle.advance_converged(P, V0, V0, 0.0, 1e-9, 50.0)
    assert conv and eps == 0.0 and len(dts) == 1 and np.array_equal(V, V0)


def test_converged_never_stops_on_a_moving_linear_field(oracle_mod):
    """A linear field advected at constant speed drops by |c| dt every step
    (closed form), so a threshold below that never triggers: the loop runs to
    the horizon, and the last change is |c| dt_last."""
    P2 = const_problem((9, 6, 5, 8), (0.4, 0.0, 0.0, 0.0))
    x = P2.coords(0)
    V0 = np.broadcast_to((1.0 - x)[:, None, None, None], P2.n).copy()
    V, t, dts, eps, conv = oracle.advance_converged(P2, V0, V0, 0.0, 1e-3, 1.0)
    assert not conv and t == 1.0
    assert abs(eps - 0.4 * dts[-1]) <= 1e-12
    Vf, dtf = oracle.solve(P2, V0, 1.0)
    assert np.array_equal(V, Vf) and np.array_equal(dts, dtf)


def test_converged_equals_fixed_steps_and_eps_is_the_max_change(oracle_mod):
    """The convergence mode takes the same steps as the fixed-horizon loop;
    eps is the max-norm change of the last step; the car's BRT settles, so a
    moderate threshold stops it before a long horizon."""
    w = scenes.custom_workload((15, 15, 7, 12), n_circles=3, seed=21)
    P = car_problem(w.grid)
    V0 = scenes.initial_value(w.grid, w.scene)
    V, t, dts, eps, conv = oracle.advance_converged(P, V0, V0, 0.0, 2e-3, 30.0, nthreads=4)
    assert conv and eps < 2e-3 and t < 30.0
    n = len(dts)
    Vn_1, t1, _ = oracle.advance(P, V0, V0, 0.0, 30.0, max_steps=n - 1, nthreads=4)
    Vn, _, _ = oracle.advance(P, V0, Vn_1, t1, 30.0, max_steps=1, nthreads=4)
    assert np.array_equal(Vn, V)
    assert eps == float(np.abs(Vn - Vn_1).max())
    # and the step before did not pass the test
    Vm, _, _ = oracle.advance(P, V0, V0, 0.0, 30.0, max_steps=n - 2, nthreads=4)
    assert float(np.abs(Vn_1 - Vm).max()) >= 2e-3


# ---------------------------------------------------------------- query (Eq. uopt_max, Eq. closetoboundary)

def _random_states(P, m, rng):
    lo, hi = np.array(P.lo), np.array(P.hi)
    return lo + (hi - lo) * rng.random((m, 4))


def test_query_reproduces_grid_values(oracle_mod):
    w = scenes.custom_workload((7, 6, 5, 8), n_circles=2, seed=2)
    P = car_problem(w.grid)
    rng = np.random.default_rng(0)
    V = rng.standard_normal(w.grid.n)
    idx = np.array([(i, j, k, l) for i in (0, 3, 6) for j in (0, 5) for k in (0, 2, 4) for l in (0, 7)])
    states = np.stack([P.coords(d)[idx[:, d]] for d in range(4)], axis=1)
    val, _, _ = oracle.query(P, V, states)
    assert np.array_equal(val, V[tuple(idx.T)])


def test_query_matches_scipy_linear_interpolation(oracle_mod):
    """Values: scipy's RegularGridInterpolator (linear) on the same grid, the
    theta axis closed by repeating its first row at theta = +pi.  Gradients:
    central differences of that interpolant inside the cell."""
    interp_mod = pytest.importorskip("scipy.interpolate")
    w = scenes.custom_workload((9, 8, 6, 10), n_circles=2, seed=3)
    P = car_problem(w.grid)
    rng = np.random.default_rng(1)
    V = rng.standard_normal(w.grid.n)
    axes = [P.coords(d) for d in range(3)] + [np.append(P.coords(3), math.pi)]
    Vc = np.concatenate([V, V[..., :1]], axis=3)
    f = interp_mod.RegularGridInterpolator(axes, Vc, method="linear")
    states = _random_states(P, 300, rng)
    val, grad, _ = oracle.query(P, V, states)
    assert np.abs(val - f(states)).max() <= 1e-12
    h = [P.spacing(d) for d in range(4)]
    for d in range(4):
        # a step well inside the cell: the interpolant is linear along d there
        frac = ((states[:, d] - P.lo[d]) / h[d]) % 1.0
        ok = (frac > 0.05) & (frac < 0.95)
        e = np.zeros(4)
        e[d] = 0.01 * h[d]
        fd = (f(states[ok] + e) - f(states[ok] - e)) / (2 * e[d])
        assert np.abs(grad[ok, d] - fd).max() <= 1e-8, d


def test_query_linear_field_gradient_and_controls(oracle_mod):
    """On V = a x + b y + c v + d th (theta not periodic here) the interpolant
    is exact and its gradient is (a, b, c, d); the car's u_opt takes
    a = a_max sign(c), w = w_max sign(d) (the control maximises grad V . f),
    and the steering car's delta takes the sign of d v."""
    n = (6, 5, 7, 9)
    lo, hi = (-5.0, -4.0, 0.0, -1.0), (5.0, 4.0, 4.0, 1.0)
    coef = (0.3, -0.7, 0.25, -0.4)
    rng = np.random.default_rng(4)
    for dyn, params in ((oracle.DYN_CAR4D, (1.5, 1.0)), (oracle.DYN_CAR4D_STEER, (1.5, math.pi / 18, 0.3))):
        P = oracle.Problem(n, lo, hi, 0, dyn, params)
        X = np.meshgrid(*[P.coords(d) for d in range(4)], indexing="ij")
        V = sum(c * x for c, x in zip(coef, X))
        states = _random_states(P, 200, rng)
        val, grad, ctl = oracle.query(P, V, states)
        assert np.abs(val - states @ np.array(coef)).max() <= 1e-12
        assert np.abs(grad - np.array(coef)).max() <= 1e-12
        assert np.all(ctl[:, 0] == 1.5)
        if dyn == oracle.DYN_CAR4D:
            assert np.all(ctl[:, 1] == -1.0)
        else:
            assert np.all(ctl[:, 1] == -math.pi / 18)  # d < 0, v >= 0


def test_query_wraps_theta_and_clamps_other_axes(oracle_mod):
    w = scenes.custom_workload((7, 6, 5, 8), n_circles=2, seed=5)
    P = car_problem(w.grid)
    V = np.random.default_rng(6).standard_normal(w.grid.n)
    s = _random_states(P, 50, np.random.default_rng(7))
    v0, g0, _ = oracle.query(P, V, s)
    s2 = s.copy()
    s2[:, 3] += 2 * math.pi
    v2, g2, _ = oracle.query(P, V, s2)
    assert np.abs(v2 - v0).max() <= 1e-12 and np.abs(g2 - g0).max() <= 1e-9
    s3 = s.copy()
    s3[:, 0] = P.hi[0] + 3.0
    s4 = s.copy()
    s4[:, 0] = P.hi[0]
    assert np.array_equal(oracle.query(P, V, s3)[0], oracle.query(P, V, s4)[0])
