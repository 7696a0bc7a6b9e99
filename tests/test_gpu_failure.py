"""Failure detection without a GPU fault: a device-side wait that runs out
returns an error status the host reads, and the context stays usable.

The self-test kernel waits, with the step kernels' own bounded mbarrier
wait, on a barrier phase that nothing completes (a flag nothing sets); the
wait gives up at its deadline and records HJ_ERR_TIMEOUT.  The grid-barrier
self-test does the same for the resident kernel's barrier: two CTAs wait for
a third arrival that never comes."""
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


def test_bounded_wait_times_out_and_context_survives(hj):
    status, waited = hj.hj_wait_selftest(50_000_000)  # 50 ms
    assert status == hj.HJ_ERR_TIMEOUT
    assert 50_000_000 <= waited < 1_000_000_000
    # the same context keeps working: a solve still matches the oracle
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    with hj.Grid.for_workload(w, hj.HJ_FP64) as g:
        g.set_initial_value(V0)
        g.solve_brt(w.T, w.cfl)
        V = g.read_value()
    P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D, (w.a_max, w.w_max))
    Vo, _ = oracle.solve(P, V0, w.T, w.cfl, nthreads=oracle.max_threads())
    assert float(np.abs(V - Vo).max()) <= 1e-12


def test_grid_barrier_times_out_and_context_survives(hj):
    status, waited = hj.hj_barrier_selftest(50_000_000)  # 50 ms
    assert status == hj.HJ_ERR_TIMEOUT
    assert 50_000_000 <= waited < 1_000_000_000
    # a resident solve on the same context completes and matches the oracle
    w = scenes.workload("car4d_31x31x11x16")
    V0 = scenes.initial_value(w.grid, w.scene)
    with hj.Grid.for_workload(w, hj.HJ_FP64) as g:
        g.set_kernel(hj.HJ_KERNEL_RESIDENT)
        g.set_initial_value(V0)
        st = g.solve_brt(w.T, w.cfl)
        assert st.kernel == hj.HJ_KERNEL_RESIDENT
        V = g.read_value()
    P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D, (w.a_max, w.w_max))
    Vo, _ = oracle.solve(P, V0, w.T, w.cfl, nthreads=oracle.max_threads())
    assert float(np.abs(V - Vo).max()) <= 1e-12


def test_selftest_limits(hj):
    for fn in (hj.hj_wait_selftest, hj.hj_barrier_selftest):
        for bad in (0, 10, 3_000_000_000):
            with pytest.raises(hj.HjError) as e:
                fn(bad)
            assert e.value.status == hj.HJ_ERR_INVALID_ARG


def test_fp64_probe_counts_and_runs(hj):
    """The FP64 rate probe the FP64 rooflines are held against: it issues the
    FMAs it reports (8 chains x iters per thread, 8 CTAs of 256 threads per
    SM) and finishes in the time that count allows at a plausible rate."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    iters = 512
    stream = torch.cuda.current_stream()
    hj.hj_fp64_fma_probe(iters, 8, stream.cuda_stream)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n = hj.hj_fp64_fma_probe(iters, 8, stream.cuda_stream)
    e1.record(stream)
    e1.synchronize()
    assert n == sms * 8 * 256 * 8 * iters
    tflops = 2.0 * n / (e0.elapsed_time(e1) * 1e-3) / 1e12
    assert 0.05 < tflops < 10.0, tflops
