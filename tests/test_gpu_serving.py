"""Re-solve server (continuous batching): requests admitted while others are
on the GPU, by slot and device-memory budget; each result must be exactly
what the request gives when it runs alone, must match the FP64 oracle's solve
of the same request within the FP32 tolerance (1e-4 max|V0|, no BRT sign flip
among cells with |V_oracle| >= 1e-3), and a Poisson trace must meet the
200 ms (5 Hz) deadline of the paper's real-time use."""
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


def solo(hj, w, v0_xy):
    with hj.Grid.for_workload(w, hj.HJ_FP32) as g:
        g.set_kernel(hj.HJ_KERNEL_TILED)
        g.set_initial_value_xy(v0_xy)
        g.solve_brt(w.T, w.cfl)
        return g.read_value()


def test_xy_ingest_equals_full_v0(hj):
    w = scenes.workload("car4d_31x31x11x16")
    for prec in (hj.HJ_FP64, hj.HJ_FP32):
        with hj.Grid.for_workload(w, prec) as g:
            g.set_initial_value(scenes.initial_value(w.grid, w.scene))
            g.solve_brt(w.T)
            a = g.read_value()
            g.set_initial_value_xy(scenes.signed_distance_xy(w.grid, w.scene))
            g.solve_brt(w.T)
            assert np.array_equal(g.read_value(), a)


def test_result_same_alone_and_in_the_mix(hj):
    trace = scenes.serving_trace(50.0, 0.3, seed=11, sizes=((31, 31, 11, 16), (60, 60, 20, 36), (40, 44, 12, 26)))
    assert len(trace) >= 6
    # fewer slots than requests: results are fetched as they complete, which
    # frees slots for the requests still queued
    with hj.Server(max_slots=8, steps_per_tick=4) as srv:
        ids = [srv.submit_xy(r.workload.grid.n, r.workload.grid.lo, r.workload.grid.hi,
                             (r.workload.a_max, r.workload.w_max), r.v0_xy(), r.workload.T) for r in trace]
        got = {}
        ticks = 0
        while len(got) < len(ids):
            srv.tick()
            ticks += 1
            for rid, r in zip(ids, trace):
                if rid not in got and srv.info(rid).state == hj.REQ_DONE:
                    got[rid] = srv.fetch(rid, r.workload.grid.n)
            assert ticks < 10000
        mixed = [got[rid] for rid in ids]
    for r, v in zip(trace, mixed):
        assert np.array_equal(v, solo(hj, r.workload, r.v0_xy()))
    # and one request alone through the server
    with hj.Server(max_slots=2) as srv:
        r = trace[2]
        rid = srv.submit_xy(r.workload.grid.n, r.workload.grid.lo, r.workload.grid.hi,
                            (r.workload.a_max, r.workload.w_max), r.v0_xy(), r.workload.T)
        while srv.info(rid).state != hj.REQ_DONE:
            srv.tick()
        assert np.array_equal(srv.fetch(rid, r.workload.grid.n), mixed[2])


def test_served_results_match_oracle(hj):
    """A dense Poisson trace (400 req/s for 40 ms, so requests overlap on the
    GPU) over all four serving sizes, 31x31x11x16 up to 100x100x30x48, replayed
    in real time through the server: every served result against the
    oracle's full solve of its request (T = 0.5 s from that request's V0)."""
    from paper_2012_04011_gb300 import serving
    trace = scenes.serving_trace(400.0, 0.04, seed=scenes.SEED_BASE + 60)
    assert {r.workload.grid.n for r in trace} == set(scenes.SERVING_SIZES)
    st = serving.run_server(trace, keep_results=True)
    assert sorted(st["results"]) == list(range(len(trace)))
    for i, r in enumerate(trace):
        w = r.workload
        V0 = scenes.initial_value(w.grid, w.scene)
        P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D, (w.a_max, w.w_max))
        Vo, dts = oracle.solve(P, V0, w.T, w.cfl, nthreads=oracle.max_threads())
        V = st["results"][i]
        assert st["steps"][i] == len(dts), (i, w.grid.n)
        err = float(np.abs(V - Vo).max())
        assert err <= 1e-4 * float(np.abs(V0).max()), (i, w.grid.n, err)
        band = np.abs(Vo) >= 1e-3
        assert int(np.count_nonzero(np.sign(V[band]) != np.sign(Vo[band]))) == 0, (i, w.grid.n)


def test_admission_by_memory_budget(hj):
    trace = scenes.serving_trace(100.0, 0.1, seed=12, sizes=((60, 60, 20, 36),))
    n = trace[0].workload.grid.n
    budget = 2 * hj.hj_batch_slot_bytes(n) + 1000
    with hj.Server(max_slots=8, memory_budget=budget, steps_per_tick=2) as srv:
        ids = [srv.submit_xy(n, r.workload.grid.lo, r.workload.grid.hi, (r.workload.a_max, r.workload.w_max),
                             r.v0_xy(), r.workload.T) for r in trace]
        results = {}
        max_running = 0
        while len(results) < len(ids):
            _, running, queued = srv.tick()
            max_running = max(max_running, running)
            for rid, r in zip(ids, trace):
                if rid not in results and srv.info(rid).state == hj.REQ_DONE:
                    results[rid] = srv.fetch(rid, n)  # frees the slot and its memory
        assert max_running <= 2
    for rid, r in zip(ids, trace):
        assert np.array_equal(results[rid], solo(hj, r.workload, r.v0_xy()))


def test_failed_request_does_not_disturb_others(hj):
    w = scenes.custom_workload((20, 20, 8, 16), T=0.2)
    bad = scenes.custom_workload((5, 5, 3, 1100), T=0.2)  # theta rows too long for a batch slot
    with hj.Server(max_slots=4) as srv:
        ok = srv.submit_xy(w.grid.n, w.grid.lo, w.grid.hi, (w.a_max, w.w_max),
                           scenes.signed_distance_xy(w.grid, w.scene), w.T)
        ko = srv.submit_xy(bad.grid.n, bad.grid.lo, bad.grid.hi, (bad.a_max, bad.w_max),
                           scenes.signed_distance_xy(bad.grid, bad.scene), bad.T)
        while srv.info(ok).state != hj.REQ_DONE:
            srv.tick()
        assert srv.info(ko).state == hj.REQ_FAILED
        with pytest.raises(hj.HjError) as e:
            srv.fetch(ko, bad.grid.n)
        assert e.value.status == hj.HJ_ERR_UNSUPPORTED
        v = srv.fetch(ok, w.grid.n)
    assert np.array_equal(v, solo(hj, w, scenes.signed_distance_xy(w.grid, w.scene)))


@pytest.mark.slow
def test_poisson_trace_meets_200ms(hj):
    from paper_2012_04011_gb300 import serving
    trace = scenes.serving_trace(40.0, 3.0, seed=13, sizes=((60, 60, 20, 36),))
    st = serving.run_server(trace)
    assert st["latency_ms"]["p99"] < 200.0, st
    mixed = scenes.serving_trace(40.0, 3.0, seed=14)
    st = serving.run_server(mixed)
    assert st["latency_ms"]["p99"] < 200.0, st
