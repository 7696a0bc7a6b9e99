"""GPU parity of the resident step kernel (HJ_KERNEL_RESIDENT): many time
steps per cooperative launch, with a bounded grid barrier between steps and
the per-cell update of the generic kernel.

Checked against the oracle with each precision's tolerance (FP64 1e-12 and
the same dt sequence, Q5.27 bit for bit, FP32 1e-4 max|V0| with no BRT sign
flip where |V| >= 1e-3), and against the generic kernel bit for bit: both
evaluate the same per-cell arithmetic on the same dt sequence, so any
difference would come from the barrier, the per-CTA finaliser, the table
rescale inside the launch or a stale read.
"""
import numpy as np
import pytest

import oracle
from paper_2012_04011_gb300 import scenes

pytestmark = pytest.mark.gpu

THR = 2e-3
STEER = (1.5, np.pi / 18, 0.3)


@pytest.fixture(scope="module")
def hj():
    from paper_2012_04011_gb300 import _build
    _build.build()
    from paper_2012_04011_gb300 import hj as mod
    return mod


def prec_code(hj, prec):
    return {"fp64": hj.HJ_FP64, "fp32": hj.HJ_FP32, "q527": hj.HJ_Q527}[prec]


def read_raw(hj, g, prec):
    """The grid's values as stored: codes for Q5.27, else FP64 (exact for FP32)."""
    if prec != "q527":
        return g.read_value()
    import torch
    out = torch.empty(int(np.prod(g.info().n)), dtype=torch.int32, device="cuda")
    g.read_value_device(out)
    return out.cpu().numpy().reshape(tuple(g.info().n))


def run(hj, w, prec, kernel, V0, T=None, dyn=None, params=None, chunk=None, converged=False, periodic=None):
    T = w.T if T is None else T
    per = w.grid.periodic if periodic is None else periodic
    with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, per, prec_code(hj, prec)) as g:
        g.set_dynamics(hj.HJ_DYN_CAR4D if dyn is None else dyn, (w.a_max, w.w_max) if params is None else params)
        g.set_kernel(kernel)
        assert g.info().kernel == kernel
        g.set_initial_value(V0)
        if converged:
            st = g.solve_converged(THR, T, w.cfl)
        elif chunk:
            steps = 0
            while True:
                st = g.advance_brt(T, w.cfl, chunk)
                steps += st.steps
                assert st.steps <= chunk
                if st.t_final == T:
                    break
            st.steps = steps
        else:
            st = g.solve_brt(T, w.cfl)
        assert st.kernel == kernel
        return read_raw(hj, g, prec), st


def check_oracle(prec, V, V0, P, T, cfl, st):
    if prec == "q527":
        Qo, dts = oracle.solve_q527(P, V0, T, cfl, nthreads=oracle.max_threads())
        assert st.steps == len(dts) and st.dt_first == dts[0] and st.dt_last == dts[-1]
        assert np.array_equal(V, Qo), int(np.count_nonzero(V != Qo))
        return
    Vo, dts = oracle.solve(P, V0, T, cfl, nthreads=oracle.max_threads())
    # the time loop is FP64 bookkeeping in every precision
    assert st.steps == len(dts) and st.dt_first == dts[0] and st.dt_last == dts[-1]
    if prec == "fp64":
        assert float(np.abs(V - Vo).max()) <= 1e-12
    else:
        assert float(np.abs(V - Vo).max()) <= 1e-4 * float(np.abs(V0).max())
        m = np.abs(Vo) >= 1e-3
        assert int(np.count_nonzero(np.sign(V[m]) != np.sign(Vo[m]))) == 0


def problem(w, dyn=oracle.DYN_CAR4D, params=None, periodic=None):
    return oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic if periodic is None else periodic, dyn,
                          (w.a_max, w.w_max) if params is None else params)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "q527"])
@pytest.mark.parametrize("name", ["car4d_31x31x11x16", "car4d_60x60x20x36"])
def test_resident_matches_oracle_and_generic(hj, name, prec):
    w = scenes.workload(name)
    V0 = scenes.initial_value(w.grid, w.scene)
    V, st = run(hj, w, prec, hj.HJ_KERNEL_RESIDENT, V0)
    assert st.launches == 2  # the prologue and one resident launch for the whole solve
    check_oracle(prec, V, V0, problem(w), w.T, w.cfl, st)
    Vg, sg = run(hj, w, prec, hj.HJ_KERNEL_GENERIC, V0)
    assert (st.steps, st.dt_first, st.dt_last, st.t_final) == (sg.steps, sg.dt_first, sg.dt_last, sg.t_final)
    assert list(st.alpha_max) == list(sg.alpha_max)
    assert np.array_equal(V, Vg)


SMALL = [(3, 3, 3, 3), (5, 4, 3, 5), (7, 9, 5, 6), (17, 13, 11, 26), (12, 10, 9, 33), (9, 21, 4, 8)]


@pytest.mark.parametrize("n", SMALL)
def test_resident_small_ragged_grids(hj, n):
    w = scenes.custom_workload(n, n_circles=3, n_rects=1, T=0.4, seed=sum(n) + 5)
    V0 = scenes.initial_value(w.grid, w.scene)
    for prec in ("fp64", "fp32", "q527"):
        V, st = run(hj, w, prec, hj.HJ_KERNEL_RESIDENT, V0)
        Vg, sg = run(hj, w, prec, hj.HJ_KERNEL_GENERIC, V0)
        assert st.steps == sg.steps and np.array_equal(V, Vg), prec
    check_oracle("q527", V, V0, problem(w), w.T, w.cfl, st)


def test_resident_all_periodic_constant_and_steering_dynamics(hj):
    w = scenes.custom_workload((10, 12, 6, 8), n_circles=3, T=0.5, seed=11)
    V0 = scenes.initial_value(w.grid, w.scene)
    for prec in ("fp64", "q527"):
        V, st = run(hj, w, prec, hj.HJ_KERNEL_RESIDENT, V0, periodic=0b1111)
        check_oracle(prec, V, V0, problem(w, periodic=0b1111), w.T, w.cfl, st)
    c = (0.7, -0.4, 0.3, -0.9)
    for prec in ("fp64", "q527"):
        V, st = run(hj, w, prec, hj.HJ_KERNEL_RESIDENT, V0, dyn=hj.HJ_DYN_CONST, params=c)
        check_oracle(prec, V, V0, problem(w, oracle.DYN_CONST, c), w.T, w.cfl, st)
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    for prec in ("fp64", "fp32", "q527"):
        V, st = run(hj, w, prec, hj.HJ_KERNEL_RESIDENT, V0, dyn=hj.HJ_DYN_CAR4D_STEER, params=STEER)
        Vg, _ = run(hj, w, prec, hj.HJ_KERNEL_GENERIC, V0, dyn=hj.HJ_DYN_CAR4D_STEER, params=STEER)
        assert np.array_equal(V, Vg), prec
        if prec != "fp32":
            check_oracle(prec, V, V0, problem(w, oracle.DYN_CAR4D_STEER, STEER), w.T, w.cfl, st)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "q527"])
def test_resident_chunked_advance_equals_one_call(hj, prec):
    """advance_brt with a step limit: every launch starts from the state the
    previous one wrote back (t, n, dt, the table's dt)."""
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    V1, s1 = run(hj, w, prec, hj.HJ_KERNEL_RESIDENT, V0)
    for chunk in (1, 5, 37):
        V2, s2 = run(hj, w, prec, hj.HJ_KERNEL_RESIDENT, V0, chunk=chunk)
        assert s2.steps == s1.steps and np.array_equal(V1, V2), chunk


@pytest.mark.parametrize("prec", ["fp64", "fp32", "q527"])
def test_resident_converged_mode(hj, prec):
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    V, st = run(hj, w, prec, hj.HJ_KERNEL_RESIDENT, V0, T=40.0, converged=True)
    Vg, sg = run(hj, w, prec, hj.HJ_KERNEL_GENERIC, V0, T=40.0, converged=True)
    assert st.converged == sg.converged == 1
    assert st.steps == sg.steps and st.last_change == sg.last_change and st.t_final == sg.t_final
    assert np.array_equal(V, Vg)
    if prec == "fp64":
        Vo, to, dts, eps, conv = oracle.advance_converged(problem(w), V0, V0, 0.0, THR, 40.0, w.cfl,
                                                          nthreads=oracle.max_threads())
        assert conv and st.steps == len(dts) and abs(st.last_change - eps) <= 1e-12
        assert float(np.abs(V - Vo).max()) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "q527"])
def test_resident_dynamics_change_mid_solve(hj, prec):
    """New bounds after t1: the prologue re-reduces alpha^max and rebuilds the
    dt-carrying table; the resident launch continues from there."""
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    t1, new = 0.37, (2.5, 0.4)
    out = {}
    for k in (hj.HJ_KERNEL_GENERIC, hj.HJ_KERNEL_RESIDENT):
        with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, prec_code(hj, prec)) as g:
            g.set_dynamics(hj.HJ_DYN_CAR4D, (w.a_max, w.w_max))
            g.set_kernel(k)
            g.set_initial_value(V0)
            g.solve_brt(t1, w.cfl)
            g.set_dynamics(hj.HJ_DYN_CAR4D, new)
            st = g.solve_brt(w.T, w.cfl)
            out[k] = (read_raw(hj, g, prec), st.steps, st.dt_last)
    a, b = out[hj.HJ_KERNEL_GENERIC], out[hj.HJ_KERNEL_RESIDENT]
    assert a[1:] == b[1:] and np.array_equal(a[0], b[0])
    if prec == "q527":
        Q0 = oracle.to_q527(V0)
        Q1, _, _ = oracle.advance_q527(problem(w), Q0, Q0, 0.0, t1, w.cfl)
        Qo, _, _ = oracle.advance_q527(problem(w, params=new), Q0, Q1, t1, w.T, w.cfl)
        assert np.array_equal(b[0], Qo)


def test_resident_zero_steps_and_done_grid(hj):
    """A call at the horizon takes no step; the state stays as it was."""
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    with hj.Grid.for_workload(w, hj.HJ_FP64) as g:
        g.set_kernel(hj.HJ_KERNEL_RESIDENT)
        g.set_initial_value(V0)
        st = g.solve_brt(w.T, w.cfl)
        V = g.read_value()
        st2 = g.solve_brt(w.T, w.cfl)
        assert st2.steps == 0 and st2.t_final == w.T and st2.total_steps == st.total_steps
        assert np.array_equal(g.read_value(), V)
        st3 = g.advance_brt(w.T + 0.5, w.cfl, 0)
        assert st3.steps == 0 and np.array_equal(g.read_value(), V)


def test_resident_solves_on_two_streams_at_once(hj):
    """Two grids whose resident launches overlap on two streams (each launch
    sized to fill the GPU): each cooperative launch waits until all its CTAs
    can be resident, so neither barrier runs out (HJ_ERR_TIMEOUT otherwise) and
    each result equals the same solve alone."""
    import threading

    import torch
    runs = [("fp32", scenes.workload("car4d_60x60x20x36")), ("q527", scenes.workload("car4d_31x31x11x16"))]
    solo = {}
    for prec, w in runs:
        solo[prec], _ = run(hj, w, prec, hj.HJ_KERNEL_RESIDENT, scenes.initial_value(w.grid, w.scene))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    out, errors = {}, []

    def worker(idx):
        prec, w = runs[idx]
        try:
            V0 = scenes.initial_value(w.grid, w.scene)
            with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, prec_code(hj, prec),
                         streams[idx].cuda_stream) as g:
                g.set_dynamics(hj.HJ_DYN_CAR4D, (w.a_max, w.w_max))
                g.set_kernel(hj.HJ_KERNEL_RESIDENT)
                g.set_initial_value(V0)
                for _ in range(3):
                    g.set_initial_value(V0)
                    g.solve_brt(w.T, w.cfl)
                out[prec] = read_raw(hj, g, prec)
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for prec, _ in runs:
        assert np.array_equal(out[prec], solo[prec]), prec


def test_paper_room_experiment_matches_oracle(hj):
    """The bench's reconstruction of the paper's experiment (Sec. IV-A: the
    60x60x20x36 room, the steering car, R = 0.75 m cones, 0.5 s in steps of
    0.007497 s) through HJ_KERNEL_AUTO: Q5.27 codes bit for bit against the
    fixed-point oracle with the 67 steps of Table II, FP64 within 1e-12, FP32
    within the FP32 tolerance."""
    w = scenes.paper_room(1)
    V0 = scenes.initial_value(w.grid, w.scene)
    P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D_STEER,
                       scenes.PAPER_STEER)
    for prec in ("q527", "fp64", "fp32"):
        with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, prec_code(hj, prec)) as g:
            g.set_dynamics(hj.HJ_DYN_CAR4D_STEER, scenes.PAPER_STEER)
            g.set_initial_value(V0)
            st = g.solve_brt(w.T, w.cfl)
            V = read_raw(hj, g, prec)
        assert st.steps == 67
        assert st.kernel == (hj.HJ_KERNEL_GENERIC if prec == "fp64" else hj.HJ_KERNEL_RESIDENT)
        check_oracle(prec, V, V0, P, w.T, w.cfl, st)


@pytest.mark.parametrize("prec", ["fp32", "q527"])
def test_resident_many_quads_per_thread(hj, prec):
    """100x100x30x48 (14.4 M cells: about 20 theta quads per thread and step)
    equals the generic kernel bit for bit."""
    w = scenes.custom_workload((100, 100, 30, 48), n_circles=8, T=0.15, seed=77)
    V0 = scenes.initial_value(w.grid, w.scene)
    V, st = run(hj, w, prec, hj.HJ_KERNEL_RESIDENT, V0)
    Vg, sg = run(hj, w, prec, hj.HJ_KERNEL_GENERIC, V0)
    assert st.steps == sg.steps > 3
    assert np.array_equal(V, Vg)


def test_resident_rejected_when_tables_do_not_fit(hj):
    """An FP64 grid whose per-(v, theta) tables exceed the shared memory the
    resident kernel keeps them in: HJ_KERNEL_RESIDENT is refused and AUTO
    keeps the generic kernel."""
    w = scenes.custom_workload((4, 4, 200, 256), n_circles=2, T=0.05, seed=5)
    with hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP64) as g:
        g.set_dynamics(hj.HJ_DYN_CAR4D, (w.a_max, w.w_max))
        with pytest.raises(hj.HjError) as e:
            g.set_kernel(hj.HJ_KERNEL_RESIDENT)
        assert e.value.status == hj.HJ_ERR_UNSUPPORTED
        assert g.info().kernel == hj.HJ_KERNEL_GENERIC
