"""Real-time re-solve loop over the C-ABI server (continuous batching).

Replays a trace of requests (arrival times and scenes) in real time: each
request is submitted when its arrival time has come, the server admits it
into the running batch as soon as a slot and memory are free, and its result
is fetched as soon as it is done.  Latency is measured from the scheduled
arrival to the moment the result is on the device (the server marks it
done), on the server's clock.

run_plain_fp64 replays the same trace through the plain FP64 path: one
request at a time, each solved alone on an FP64 grid; its latency also ends
when the result is on the device.
"""
from __future__ import annotations

import time

import numpy as np

from . import hj


def _percentiles(lat_ms):
    a = np.asarray(lat_ms, dtype=np.float64)
    if a.size == 0:
        return {"p50": None, "p99": None, "max": None, "mean": None}
    return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "max": float(a.max()),
            "mean": float(a.mean())}


def run_server(trace, max_slots: int = 64, memory_budget: int = 0, steps_per_tick: int = 32, fetch: bool = True,
               cuda_stream=None, keep_results: bool = False):
    """Replays the trace through an hj.Server.  Returns stats (and, when
    keep_results, the results and the time steps taken, by request index)."""
    lat, cell_updates, results, steps_by_req = [], 0, {}, {}
    with hj.Server(max_slots, memory_budget, steps_per_tick, cuda_stream) as srv:
        t0 = srv.clock()
        pending = list(enumerate(trace))
        pending.reverse()
        outstanding = {}
        while pending or outstanding:
            now = srv.clock() - t0
            while pending and pending[-1][1].t_arrival <= now:
                i, r = pending.pop()
                w = r.workload
                rid = srv.submit_xy(w.grid.n, w.grid.lo, w.grid.hi, (w.a_max, w.w_max), r.v0_xy(), w.T, w.cfl)
                outstanding[rid] = (i, r)
            if not outstanding:
                if pending:
                    time.sleep(max(0.0, min(0.002, pending[-1][1].t_arrival - (srv.clock() - t0))))
                continue
            completed, running, queued = srv.tick()
            if completed:
                for rid in list(outstanding):
                    info = srv.info(rid)
                    if info.state == hj.REQ_DONE:
                        i, r = outstanding.pop(rid)
                        lat.append(1e3 * (info.t_done - (t0 + r.t_arrival)))
                        cell_updates += int(np.prod(r.workload.grid.n)) * info.steps
                        if fetch:
                            v = srv.fetch(rid, r.workload.grid.n)
                            if keep_results:
                                results[i] = v
                                steps_by_req[i] = info.steps
                    elif info.state == hj.REQ_FAILED:
                        raise RuntimeError(f"request {rid} failed")
        wall = srv.clock() - t0
        ticks, steps = srv.stats()
    out = {"requests": len(trace), "latency_ms": _percentiles(lat), "wall_s": wall,
           "cell_updates_per_s": cell_updates / wall if wall > 0 else None, "ticks": ticks, "batch_steps": steps}
    if keep_results:
        out["results"] = results
        out["steps"] = steps_by_req
    return out


def run_plain_fp64(trace, cuda_stream=None, fetch: bool = True):
    """Replays the trace through the plain FP64 path (FIFO, one grid at a
    time on the same GPU)."""
    lat, cell_updates = [], 0
    grids = {}
    t0 = time.perf_counter()
    for r in trace:
        now = time.perf_counter() - t0
        if r.t_arrival > now:
            time.sleep(r.t_arrival - now)
        w = r.workload
        key = w.grid.n
        if key not in grids:
            g = hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP64, cuda_stream)
            g.set_dynamics(hj.HJ_DYN_CAR4D, (w.a_max, w.w_max))
            grids[key] = g
        g = grids[key]
        g.set_initial_value_xy(r.v0_xy())
        st = g.solve_brt(w.T, w.cfl)
        # done = the result is on the device (solve_brt returns after the last
        # step), as the server measures it; the fetch is not part of it
        lat.append(1e3 * ((time.perf_counter() - t0) - r.t_arrival))
        if fetch:
            g.read_value()
        cell_updates += int(np.prod(w.grid.n)) * st.steps
    wall = time.perf_counter() - t0
    for g in grids.values():
        g.close()
    return {"requests": len(trace), "latency_ms": _percentiles(lat), "wall_s": wall,
            "cell_updates_per_s": cell_updates / wall if wall > 0 else None}
