"""Benchmark: 4D HJ reachability BRT solves on GB300 through libhj.

One benchmark step is one whole BRT solve of the 128x128x64x96 car workload
(seeded obstacles, T = 2.0 s, CFL 0.8, 352 time steps): V0 ingest from a
device-resident array, the full time loop, and the readback of V into a
device-resident array.  Throughput is cell-updates/s (cells x time steps /
s); the dominant kernel's roofline is the HBM bound (12 algorithmic bytes per
FP32 cell-update: read V_n, read V0, write V_{n+1}).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica (no data-path
collective); the JSON line reports the whole-job rate.  --impl reference
times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4D HJ cell-updates/s (fraction of HBM peak) + p99 re-solve latency vs FP64 path"
UNIT = "cell-updates/s"
WORKLOAD = "car4d_128x128x64x96"
STEER = (1.5, math.pi / 18, 0.3)  # Sec. IV-A: a in [-1.5, 1.5], delta in [-pi/18, pi/18], L = 0.3 m
BYTES_PER_UPDATE = {"f32": 12, "f64": 24, "q527": 12, "f32_bcast": 8}
KERNEL_NAMES = {1: "generic", 2: "tiled", 3: "resident"}
PROFILE = os.path.join(ROOT, "profiles", "hj_step_tiled_car4d_128x128x64x96.md")
KERNEL_SOURCES = ["hj_tiled_kernel.cuh", "hj_tiled_f32.cu", "hj_device.cuh", "hj_tma.cuh", "hj_scaled.cuh",
                  "hj_internal.h"]
# FP64 path: bound by the FP64 unit.  Algorithmic FP64 flops per cell-update
# of the FP64 step kernel: V_new = w0 V_c + |w1| V_up1 + |w2| V_up2 + dt k3
# V_up3 + w4 V_up4 with the dt-scaled table, 1 DMUL + 4 DFMA = 9 flops (the
# BRT min is an integer compare of the bit patterns).  The peak is measured
# in the run by the library's FP64 FMA probe; the nominal GB300 figure is the
# fallback only if the probe cannot run.
FP64_FLOPS_PER_UPDATE = 9
FP64_NOMINAL_TFLOPS = 1.25
# Query kernel: FP64 flops per query, counted from its source: the cell
# search (3 flops on each of the three clamped axes, 6 on the periodic one),
# 15 linear interpolations for V and 11 for the gradient (a difference and an
# FMA each: 3 flops) and 4 multiplications by the reciprocal spacings.  The
# 16 float-to-double conversions and 4 floors also run on the FP64 unit but
# are not flops.
QUERY_FP64_FLOPS = 3 * 3 + 6 + 3 * 15 + 3 * 11 + 4


# ------------------------------------------------------------------ helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_max(x: float, world: int, device: str = "cpu") -> float:
    """Max of x over all ranks (each rank times its own replica; the job
    takes as long as the slowest)."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, seconds_max: float) -> float:
    """Whole-job rate: every rank processed units_per_rank (replicas, weak
    scaling) in at most seconds_max."""
    return world * units_per_rank / seconds_max


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2012_04011_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the tiled step kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_tr or m_hash.group(1) != kernel_hash():
        return None
    return float(m_tr.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def visible_gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip() != ""]
    if ids and ids[local_rank % len(ids)].strip().isdigit():
        return int(ids[local_rank % len(ids)])
    return local_rank


def measure_fp64_peak(hj, torch, stream, gpu_index, iters=4096, launches=5):
    """FP64 FMA throughput of this GPU, from the library's probe kernel:
    CUDA events on the launching stream around `launches` launches after two
    warm-up launches, SM clocks sampled meanwhile.  2 flops per FMA."""
    for _ in range(2):
        hj.hj_fp64_fma_probe(iters, 8, stream.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index) as cs:
        e0.record(stream)
        fmas = 0
        for _ in range(launches):
            fmas += hj.hj_fp64_fma_probe(iters, 8, stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        time.sleep(0.25)  # let the sampler see the clocks of the run
    ms = e0.elapsed_time(e1)
    clk = cs.summary()
    tflops = 2.0 * fmas / (ms * 1e-3) / 1e12
    return {"tflops": tflops, "ms_per_launch": ms / launches, "fma_per_launch": fmas // launches,
            "sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
            "tflops_x_mhz_ratio": (tflops / clk["sm_mhz"] * clk["sm_max_mhz"]) if clk["sm_mhz"] else None,
            "how": "hj_fp64_fma_probe: 8 CTAs of 256 threads per SM, 8 independent DFMA chains of "
                   f"{iters} steps per thread, {launches} launches timed with CUDA events"}


def oracle_accuracy(w, V0, results_host, nthreads):
    """Every precision's full-horizon result on the workload against the FP64
    oracle's solve of the same input: max |V - V_oracle| and the BRT sign
    flips among cells with |V_oracle| >= 1e-3."""
    import oracle
    P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D, (w.a_max, w.w_max))
    t0 = time.perf_counter()
    Vo, dts = oracle.solve(P, V0, w.T, w.cfl, nthreads=nthreads)
    el = time.perf_counter() - t0
    band = np.abs(Vo) >= 1e-3
    out = {"oracle": {"time_steps": len(dts), "dt_first": float(dts[0]), "dt_last": float(dts[-1]),
                      "seconds": el, "threads": nthreads}, "sign_band": 1e-3,
           "fp32_tolerance": 1e-4 * float(np.abs(V0).max()), "fp64_tolerance": 1e-12}
    for name, (V, st) in results_host.items():
        V = V.reshape(Vo.shape)
        out[name] = {"max_abs_vs_oracle": float(np.abs(V - Vo).max()),
                     "sign_flips_vs_oracle": int(np.count_nonzero(np.sign(V[band]) != np.sign(Vo[band]))),
                     "time_steps_equal": bool(st[0] == len(dts)),
                     "dt_first_last_equal": bool(st[1] == dts[0] and st[2] == dts[-1])}
    return out


# ------------------------------------------------------------------ oracle (CPU baseline)

def oracle_sample(w, V0, steps: int, nthreads: int):
    """Time `steps` oracle time steps of the workload (the whole per-step hot
    path: alpha reduction, CFL step, stencil update, BRT min)."""
    import oracle
    P = oracle.Problem(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, oracle.DYN_CAR4D, (w.a_max, w.w_max))
    t0 = time.perf_counter()
    _, _, dts = oracle.advance(P, V0, V0, 0.0, w.T, w.cfl, max_steps=steps, nthreads=nthreads)
    el = time.perf_counter() - t0
    return len(dts) * V0.size / el, el, len(dts)


def cpu_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2012_04011_gb300 import scenes
    w = scenes.workload(WORKLOAD)
    V0 = scenes.initial_value(w.grid, w.scene)
    nthreads = cpu_threads()
    per_step = args.cpu_sample_steps
    for _ in range(args.warmup):
        oracle_sample(w, V0, per_step, nthreads)
    updates, elapsed = 0, 0.0
    for _ in range(args.steps):
        _, el, nst = oracle_sample(w, V0, per_step, nthreads)
        updates += nst * V0.size
        elapsed += el
    value = updates / elapsed
    sample = (f"{per_step} oracle time steps of the {WORKLOAD} solve per benchmark step "
              f"({per_step * V0.size:.3e} cell-updates), FP64, OpenMP over x")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded obstacles)",
        "config": {"workload": WORKLOAD, "grid": list(w.grid.n), "horizon_s": w.T, "cfl": w.cfl,
                   "sample_time_steps_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line, default=json_default), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def run_small(hj, scenes, torch, stream, with_oracle=True):
    """The small single-instance workloads and the paper's own experiment
    (all fit in the 129 MB L2, so they are reported as cell-updates/s and
    solve latency, not against HBM).  Each precision runs the kernel
    HJ_KERNEL_AUTO picks (the resident kernel for FP32 and Q5.27 grids this
    small) and, for comparison, the per-step kernel it replaces.  With
    with_oracle, every result is held against the FP64 oracle's solve of the
    same input (max |difference| and BRT sign flips among cells with
    |V_oracle| >= 1e-3), and the oracle's own solve is timed on the host
    cores: all of them, and one thread for the 31x31x11x16 grid."""
    def time_small(wl, prec, kernel, dyn, params, v0d, reps=5):
        gs = hj.Grid(wl.grid.n, wl.grid.lo, wl.grid.hi, wl.grid.periodic, prec, stream.cuda_stream)
        gs.set_dynamics(dyn, params)
        gs.set_kernel(kernel)
        o = torch.empty(v0d.numel(), dtype=torch.float64, device="cuda")
        for _ in range(2):
            hj.hj_set_initial_value_device(gs.handle, v0d)
            gs.solve_brt(wl.T, wl.cfl)
        ms_, loops = [], []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hj.hj_set_initial_value_device(gs.handle, v0d)
            st_ = gs.solve_brt(wl.T, wl.cfl)
            e1.record(stream)
            e1.synchronize()
            ms_.append(e0.elapsed_time(e1))
            loops.append(st_.loop_ms)
        hj.hj_read_value_device(gs.handle, o)
        kern = gs.info().kernel
        gs.close()
        med = float(np.median(ms_))
        return {"ms_per_solve_median": med, "time_steps": st_.steps,
                "us_per_step": 1e3 * float(np.median(loops)) / max(st_.steps, 1),
                "value": v0d.numel() * st_.steps / (med * 1e-3), "unit": UNIT,
                "kernel": KERNEL_NAMES.get(kern, kern)}, o

    def vs_oracle(o, Vo):
        V = o.cpu().numpy().reshape(Vo.shape)  # FP64 values (a Q5.27 grid reads back code * 2^-27)
        m = np.abs(Vo) >= 1e-3
        return float(np.abs(V - Vo).max()), int(np.count_nonzero(np.sign(V[m]) != np.sign(Vo[m])))

    def oracle_solve(ws_, dyn, params, V0, nthreads):
        import oracle
        okind = oracle.DYN_CAR4D_STEER if dyn == hj.HJ_DYN_CAR4D_STEER else oracle.DYN_CAR4D
        P = oracle.Problem(ws_.grid.n, ws_.grid.lo, ws_.grid.hi, ws_.grid.periodic, okind, params)
        t0 = time.perf_counter()
        Vo, dts = oracle.solve(P, V0, ws_.T, ws_.cfl, nthreads=nthreads)
        return Vo, dts, time.perf_counter() - t0

    small = {}
    cases = [(name, scenes.workload(name), hj.HJ_DYN_CAR4D, None)
             for name in ("car4d_31x31x11x16", "car4d_60x60x20x36")]
    cases.append(("paper_room_60x60x20x36_steer", scenes.paper_room(1), hj.HJ_DYN_CAR4D_STEER, scenes.PAPER_STEER))
    for name, ws_, dyn, params in cases:
        params = params or (ws_.a_max, ws_.w_max)
        V0h = scenes.initial_value(ws_.grid, ws_.scene)
        v0s = torch.from_numpy(V0h).to("cuda")
        res = {}
        Vo = None
        if with_oracle:
            nth = cpu_threads()
            Vo, dts, el = oracle_solve(ws_, dyn, params, V0h, nth)
            res["oracle"] = {"seconds_per_solve": el, "threads": nth, "time_steps": len(dts),
                             "value": V0h.size * len(dts) / el, "unit": UNIT}
            if name == "car4d_31x31x11x16":
                _, _, el1 = oracle_solve(ws_, dyn, params, V0h, 1)
                res["oracle"]["seconds_per_solve_one_thread"] = el1
        for pname, pr, per_step in (("f64", hj.HJ_FP64, None), ("f32", hj.HJ_FP32, hj.HJ_KERNEL_TILED),
                                    ("q527", hj.HJ_Q527, hj.HJ_KERNEL_TILED)):
            r, o = time_small(ws_, pr, hj.HJ_KERNEL_AUTO, dyn, params, v0s)
            if Vo is not None:
                r["max_abs_vs_oracle"], r["sign_flips_vs_oracle"] = vs_oracle(o, Vo)
            if per_step is not None:
                rp, _ = time_small(ws_, pr, per_step, dyn, params, v0s)
                r["per_step_kernel"] = {k: rp[k] for k in ("kernel", "ms_per_solve_median", "us_per_step")}
            res[pname] = r
        small[name] = {**res, "l2_resident": True, "T": ws_.T, "cfl": ws_.cfl}
        if name.startswith("paper_room"):
            # context only (another machine): Table II, the FPGA's 67 iterations
            # on its 60x60x20x36 grid in fixed point, 0.176 s
            small[name]["published_fpga_brt_ms"] = 176.0
            small[name]["dynamics"] = "steering car, a in [-1.5, 1.5], delta in [-pi/18, pi/18], L = 0.3 m"
    return small


DEADLINE_MS = 200.0  # the paper's 5 Hz re-solve rate (Sec. IV-C)


def saturation_sweep(srv_mod, scenes, stream, sizes, rates, seconds, seed0):
    """Poisson traces at rising rates, replayed in real time through the FP32
    server (continuous batching) and through the plain FP64 path.  An arm
    stops at the first rate whose p99 latency reaches the deadline; its
    saturation point is the highest rate it served with p99 below it."""
    rows, alive, sat = {}, {"fp32_batched": True, "fp64_plain": True}, {"fp32_batched": None, "fp64_plain": None}
    for rate in rates:
        if not any(alive.values()):
            break
        trs = scenes.serving_trace(rate, seconds, seed=seed0 + int(rate), sizes=sizes)
        row = {"requests": len(trs)}
        for arm, fn in (("fp32_batched", srv_mod.run_server), ("fp64_plain", srv_mod.run_plain_fp64)):
            if not alive[arm]:
                continue
            r = fn(trs, cuda_stream=stream.cuda_stream)
            lat = r["latency_ms"]
            row[arm] = {"p50": lat["p50"], "p99": lat["p99"], "served_req_per_s": len(trs) / r["wall_s"],
                        "cell_updates_per_s": r["cell_updates_per_s"]}
            if lat["p99"] is not None and lat["p99"] < DEADLINE_MS:
                sat[arm] = {"req_per_s": rate, **row[arm]}
            else:
                alive[arm] = False
        rows[f"{rate:g}"] = row
    return {"sizes": ["x".join(map(str, s)) for s in sizes], "seconds_per_rate": seconds,
            "deadline_ms": DEADLINE_MS, "req_per_s": rows, "saturation": sat,
            "note": "saturation = the highest swept rate whose p99 stayed below the deadline; null = none did"}


LARGE_GRID = (2048, 2048, 32, 33)


def run_large(hj, scenes, torch, stream, steps=10):
    """Grids past 32-bit offsets: the 2048x2048x32x33 car (4.4e9 cells, 4.8e9
    stored values, 58 GB of FP32 or Q5.27 buffers), V0 from its (x, y) field
    (so the tiled kernel is its broadcast-V0 variant, 8 B per update; the
    generic kernel reads the 4D V0, 12 B), and the tiled kernel once more
    with the same V0 as a 4D device array (12 B).  Each precision runs the
    tiled kernel (autotuned) both ways and the generic one;
    ms per step from the library's CUDA events around `steps` steps, after 3
    warm-up steps."""
    n = LARGE_GRID
    grid = scenes.GridSpec(n)
    v0_xy = scenes.signed_distance_xy(grid, scenes.random_scene(np.random.default_rng(scenes.SEED_BASE + 7), 12))
    ncell = int(np.prod(n))
    peak = measured_peaks()[0]
    res = {"workload": "car4d_%dx%dx%dx%d" % n, "cells": ncell}
    for pname, prec in (("f32", hj.HJ_FP32), ("q527", hj.HJ_Q527)):
        for kname, kern in (("tiled", hj.HJ_KERNEL_TILED), ("tiled_4d", hj.HJ_KERNEL_TILED),
                            ("generic", hj.HJ_KERNEL_GENERIC)):
            with hj.Grid(n, grid.lo, grid.hi, grid.periodic, prec, stream.cuda_stream) as g:
                g.set_dynamics(hj.HJ_DYN_CAR4D, (scenes.A_MAX, scenes.W_MAX))
                if kname == "tiled_4d":
                    # the same V0 as a 4D array (the field replicated over v and
                    # theta on the device, 17.7 GB of FP32): the 12-byte kernel
                    v4 = torch.from_numpy(np.ascontiguousarray(v0_xy, dtype=np.float32)).to("cuda")
                    v4 = v4[:, :, None, None].expand(n[0], n[1], n[2], n[3]).contiguous().reshape(-1)
                    hj.hj_set_initial_value_device(g.handle, v4)
                    del v4
                    torch.cuda.empty_cache()
                else:
                    g.set_initial_value_xy(v0_xy)
                g.set_kernel(kern)
                if kern == hj.HJ_KERNEL_TILED:
                    g.autotune(4)
                g.advance_brt(10.0, scenes.CFL, 3)
                st = g.advance_brt(10.0, scenes.CFL, steps)
                ms = st.loop_ms / max(st.steps, 1)
                # V0 came as its (x, y) field: the tiled kernel reads that field
                # (8 B per update), the generic kernel the 4D V0 (12 B)
                bpu = BYTES_PER_UPDATE["f32_bcast"] if kname == "tiled" else BYTES_PER_UPDATE[pname]
                res[f"{pname}_{kname}"] = {
                    "ms_per_step": ms, "value": ncell / (ms * 1e-3), "unit": UNIT, "bytes_per_update": bpu,
                    "hbm_frac": bpu * ncell / (ms * 1e-3) / 1e9 / peak,
                    "kernel": KERNEL_NAMES.get(g.info().kernel, g.info().kernel),
                    "tile": list(g.info().tile) if kern == hj.HJ_KERNEL_TILED else None}
            torch.cuda.empty_cache()
    return res


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_04011_gb300 import hj, scenes

    if args.small_only:
        if rank == 0:
            print(json.dumps({"small_configs": run_small(hj, scenes, torch, torch.cuda.current_stream())}, default=json_default))
        return 0
    if args.large_only:
        if rank == 0:
            print(json.dumps({"large_grid": run_large(hj, scenes, torch, torch.cuda.current_stream())}, default=json_default))
        return 0

    w = scenes.workload(WORKLOAD)
    V0 = scenes.initial_value(w.grid, w.scene)
    ncell = V0.size
    stream = torch.cuda.current_stream()
    V0_dev = torch.from_numpy(V0).to("cuda")
    V0xy_dev = torch.from_numpy(np.ascontiguousarray(scenes.signed_distance_xy(w.grid, w.scene))).to("cuda")
    out32 = torch.empty(ncell, dtype=torch.float32, device="cuda")
    out64 = torch.empty(ncell, dtype=torch.float64, device="cuda")
    outq = torch.empty(ncell, dtype=torch.int32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        return rank_max(x, world, "cuda")

    def solve_once(g, out, xy=False):
        if xy:  # V0 from its position-only field: the broadcast-V0 kernel
            hj.hj_set_initial_value_xy_device(g.handle, V0xy_dev)
        else:
            hj.hj_set_initial_value_device(g.handle, V0_dev)
        st = hj.hj_solve_brt(g.handle, w.T, w.cfl)
        hj.hj_read_value_device(g.handle, out)
        return st

    results = {}
    accuracy = None
    results_host = {}  # precision -> (V as FP64 host array, (steps, dt_first, dt_last)) of the 4D-V0 car solves
    for prec_name, prec, out, K, W in (("f32", hj.HJ_FP32, out32, args.steps, args.warmup),
                                       ("f64", hj.HJ_FP64, out64, max(1, min(args.steps, args.fp64_steps)), 1),
                                       ("q527", hj.HJ_Q527, outq, max(1, min(args.steps, args.q527_steps)), 1),
                                       ("f32_bcast", hj.HJ_FP32, out32, max(1, min(args.steps, args.bcast_steps)),
                                        1),
                                       ("f32_steer", hj.HJ_FP32, out32, max(1, min(args.steps, args.steer_steps)),
                                        1)):
        if (prec_name == "f64" and args.no_fp64) or (prec_name == "q527" and args.no_q527) or \
                (prec_name == "f32_bcast" and args.no_bcast) or (prec_name == "f32_steer" and args.no_steer):
            continue
        xy = prec_name == "f32_bcast"
        g = hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, prec, stream.cuda_stream)
        if prec_name == "f32_steer":  # Eq. car_dynamics as printed: th' = v tan(delta) / L
            g.set_dynamics(hj.HJ_DYN_CAR4D_STEER, STEER)
        else:
            g.set_dynamics(hj.HJ_DYN_CAR4D, (w.a_max, w.w_max))
        tuned = None
        tile_arg = {"f32_bcast": args.bcast_tile, "q527": args.q527_tile}.get(prec_name) or args.tile
        if prec != hj.HJ_FP64 and tile_arg:
            if xy:  # the tile's room depends on whether V0 comes as a box
                hj.hj_set_initial_value_xy_device(g.handle, V0xy_dev)
            g.set_tile_shape([int(v) for v in tile_arg.split(",")])
            tuned = {"shape": list(g.info().tile), "ctas": g.info().tile_ctas, "tried": []}
        elif prec != hj.HJ_FP64 and not args.no_autotune:
            # pick the tile shape by timing candidates (outside the timed region)
            if xy:
                hj.hj_set_initial_value_xy_device(g.handle, V0xy_dev)
            else:
                hj.hj_set_initial_value_device(g.handle, V0_dev)
            tried = g.autotune(8)
            tuned = {"shape": list(g.info().tile), "ctas": g.info().tile_ctas,
                     "tried": [t.as_dict() for t in tried]}
        for _ in range(W):
            solve_once(g, out, xy)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lat, loop_ms, steps_total, launches = [], 0.0, 0, 0
        sampler = ClockSampler(visible_gpu_index(local)) if prec_name == "f32" else None
        if sampler:
            sampler.__enter__()
        ev0.record(stream)
        for _ in range(K):
            e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            st = solve_once(g, out, xy)
            e_b.record(stream)
            e_b.synchronize()
            lat.append(e_a.elapsed_time(e_b))
            loop_ms += st.loop_ms
            steps_total += st.steps
            launches += st.launches + 2  # + ingest and readback kernels
        ev1.record(stream)
        barrier()
        if sampler:
            sampler.__exit__(None, None, None)
        ms = max_over_ranks(ev0.elapsed_time(ev1))
        kernel = g.info().kernel
        g.close()
        if prec_name in ("f32", "f64", "q527"):
            vals = out.double() * (2.0 ** -27) if prec_name == "q527" else out.double()
            results_host[prec_name] = (vals.cpu().numpy(), (st.steps, st.dt_first, st.dt_last))
        results[prec_name] = {
            "ms_total": ms, "K": K, "value": job_throughput(world, ncell * steps_total, ms * 1e-3), "ms_per_step": ms / K,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "avg_step_kernel_ms": loop_ms / steps_total, "time_steps_per_solve": steps_total // K,
            "launches": launches, "kernel": kernel, "clocks": sampler.summary() if sampler else None,
            "tile": tuned,
        }

    # queries: V, grad V and u_opt at 2^20 random states of the solved grid
    # (the controller of Sec. IV-A), device arrays, one kernel per call
    query = None
    if not args.no_query:
        g = hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP32, stream.cuda_stream)
        g.set_dynamics(hj.HJ_DYN_CAR4D, (w.a_max, w.w_max))
        solve_once(g, out32)
        mq = 1 << 20
        rng = np.random.default_rng(scenes.SEED_BASE + 7)
        lo_, hi_ = np.array(w.grid.lo), np.array(w.grid.hi)
        sq = torch.from_numpy(lo_ + (hi_ - lo_) * rng.random((mq, 4))).to("cuda")
        vq = torch.empty(mq, dtype=torch.float64, device="cuda")
        gq = torch.empty((mq, 4), dtype=torch.float64, device="cuda")
        cq = torch.empty((mq, 2), dtype=torch.float64, device="cuda")
        for _ in range(3):
            hj.hj_query_device(g.handle, sq, vq, gq, cq)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kq = 10
        e0.record(stream)
        for _ in range(kq):
            hj.hj_query_device(g.handle, sq, vq, gq, cq)
        e1.record(stream)
        barrier()
        qms = max_over_ranks(e0.elapsed_time(e1)) / kq
        g.close()
        qbytes = 32 + 8 + 32 + 16 + 16 * 4  # state in, value, gradient, control out, 16 grid values
        query = {"workload": f"{mq} random states on the solved {WORKLOAD} FP32 grid: value, gradient, u_opt",
                 "value": job_throughput(world, mq, qms * 1e-3), "unit": "queries/s", "ms_per_call": qms,
                 "hbm": {"achieved_gbs": qbytes * mq / (qms * 1e-3) / 1e9,
                         "frac": qbytes * mq / (qms * 1e-3) / 1e9 / measured_peaks()[0], "bytes_per_query": qbytes}}

    small = None if args.no_small else run_small(hj, scenes, torch, stream, with_oracle=world == 1)
    fp64_peak = measure_fp64_peak(hj, torch, stream, visible_gpu_index(local))

    # batched solves: the 64-instance workload (uneven grids, own obstacles,
    # T = 1.5 s), V0 already on the device, one persistent launch per batch solve
    batch = None
    if not args.no_batch:
        ws = scenes.batch_workloads()
        v0d = [torch.from_numpy(scenes.initial_value(bw.grid, bw.scene)).to("cuda").reshape(-1) for bw in ws]
        b = hj.Batch(len(ws), cuda_stream=stream.cuda_stream)
        slots = [b.add_workload(bw) for bw in ws]
        for sl, v in zip(slots, v0d):
            hj.hj_batch_set_initial_value(b.handle, sl, v)
        if args.batch_shape:
            nc, ch = [int(v) for v in args.batch_shape.split(",")]
            b.set_shape(nc, ch)
        else:
            nc, ch, _ = b.autotune(4)

        def batch_solve():
            b.set_initial_values(slots, v0d)  # every slot's V0, one synchronisation
            b.set_horizons(slots, [bw.T for bw in ws], [bw.cfl for bw in ws])
            return b.advance()

        for _ in range(2):
            batch_solve()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kb = max(1, min(args.steps, 5))
        e0.record(stream)
        adv_ms, bsteps = 0.0, 0
        for _ in range(kb):
            st = batch_solve()
            adv_ms += st.device_ms
            bsteps += st.steps
        e1.record(stream)
        barrier()
        # every solve takes each slot through the same steps: count them once,
        # after the timed region
        upd = kb * sum(int(np.prod(bw.grid.n)) * b.slot_info(sl).steps for sl, bw in zip(slots, ws))
        bms = max_over_ranks(e0.elapsed_time(e1))
        cells = sum(int(np.prod(bw.grid.n)) for bw in ws)
        b.close()
        batch = {"workload": "batch64: 64 car instances, N1,N2 in {40,50,60}, N3 in [16,24], N4 in [24,36], "
                             "4-16 circles, T = 1.5 s, FP32",
                 "value": job_throughput(world, upd, bms * 1e-3), "unit": UNIT, "ms_per_solve": bms / kb,
                 "cells": cells, "batch_steps_per_solve": bsteps // kb, "nconsumer": nc, "chunks": ch,
                 "hbm_frac": 12 * (upd / kb) / (adv_ms / kb * 1e-3) / 1e9 / measured_peaks()[0]}

    # serving: Poisson re-solve requests (each moves or adds 1-4 obstacles of
    # a resident scene), T = 0.5 s, continuous batching vs the plain FP64 path
    serving = None
    if not args.no_serving and world == 1:
        from paper_2012_04011_gb300 import serving as srv_mod
        tr = scenes.serving_trace(args.serving_rate, args.serving_seconds, sizes=((60, 60, 20, 36),))
        s32 = srv_mod.run_server(tr, cuda_stream=stream.cuda_stream)
        s64 = srv_mod.run_plain_fp64(tr, cuda_stream=stream.cuda_stream)
        mixed = srv_mod.run_server(scenes.serving_trace(args.serving_rate, args.serving_seconds),
                                   cuda_stream=stream.cuda_stream)
        serving = {"workload": f"60x60x20x36 re-solves, T = 0.5 s, Poisson {args.serving_rate:g} req/s for "
                               f"{args.serving_seconds:g} s", "deadline_ms": 200.0,
                   "fp32_batched": {k: s32[k] for k in ("requests", "latency_ms", "cell_updates_per_s")},
                   "fp64_plain": {k: s64[k] for k in ("requests", "latency_ms", "cell_updates_per_s")},
                   "mixed_sizes_fp32_batched": {"sizes": "31x31x11x16, 60x60x20x36, 80x80x25x40, 100x100x30x48",
                                                **{k: mixed[k] for k in ("requests", "latency_ms",
                                                                         "cell_updates_per_s")}}}
        # rising arrival rates, FP32 continuous batching against the plain
        # FP64 path, each arm until its p99 reaches the 200 ms deadline: the
        # 60x60x20x36 re-solves, then the mixed sizes
        if args.serving_sweep:
            serving["rate_sweep_60x60x20x36"] = saturation_sweep(
                srv_mod, scenes, stream, ((60, 60, 20, 36),), args.serving_sweep, args.serving_sweep_seconds,
                scenes.SEED_BASE + 200)
            serving["rate_sweep_mixed_sizes"] = saturation_sweep(
                srv_mod, scenes, stream, scenes.SERVING_SIZES, args.serving_sweep, args.serving_sweep_seconds,
                scenes.SEED_BASE + 40)

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        h_v0 = torch.from_numpy(V0).pin_memory()
        h_out = torch.empty(ncell, dtype=torch.float64).pin_memory()
        g = hj.Grid(w.grid.n, w.grid.lo, w.grid.hi, w.grid.periodic, hj.HJ_FP32, stream.cuda_stream)
        g.set_dynamics(hj.HJ_DYN_CAR4D, (w.a_max, w.w_max))
        if results["f32"]["tile"]:
            g.set_tile_shape(results["f32"]["tile"]["shape"])
        v0_np, out_np = h_v0.numpy(), h_out.numpy()

        def e2e_once():
            hj.hj_set_initial_value(g.handle, v0_np)
            st = hj.hj_solve_brt(g.handle, w.T, w.cfl)
            hj.hj_read_value(g.handle, out_np.reshape(V0.shape))
            return st

        for _ in range(max(1, args.warmup)):
            e2e_once()
        barrier()
        t0 = time.perf_counter()
        st_steps = 0
        Ke = max(1, min(args.steps, args.e2e_steps))
        for _ in range(Ke):
            st_steps += e2e_once().steps
        barrier()
        el = max_over_ranks(time.perf_counter() - t0)
        g.close()
        e2e = {"value": job_throughput(world, ncell * st_steps, el), "unit": UNIT,
               "h2d_bytes_per_step": int(V0.nbytes), "d2h_bytes_per_step": int(h_out.numel() * 8),
               "ms_per_step": 1e3 * el / Ke}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    r32 = results["f32"]
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_UPDATE["f32"] * ncell / (r32["avg_step_kernel_ms"] * 1e-3) / 1e9
    traffic = profiled_traffic()
    line = {
        "metric": METRIC, "value": r32["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r32["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded obstacles)",
        "config": {"workload": WORKLOAD, "grid": list(w.grid.n), "horizon_s": w.T, "cfl": w.cfl,
                   "time_steps_per_solve": r32["time_steps_per_solve"],
                   "step": "one BRT solve: V0 ingest from HBM, full time loop, V readback to HBM",
                   "l2": "no flush needed: V0 and both V buffers are 403 MB each (> 129 MB L2)",
                   "parallelism": f"replicas x{world}",
                   "tile": r32["tile"]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "hj_step_tiled_kernel", "peak_source": f"{peak_kind} hbm_gbs",
                     "bytes_per_update": BYTES_PER_UPDATE["f32"],
                     "avg_launch_ms": r32["avg_step_kernel_ms"]},
        "latency_ms": r32["latency_ms"],
        "accuracy": accuracy,
        "clocks": r32["clocks"],
        "gpu_launches": r32["launches"],
        "e2e": e2e,
        "batch64": batch,
        "query": query,
        "small_configs": small,
        "serving": serving,
    }
    if "f64" in results:
        r64 = results["f64"]
        # the FP64 path is bound by the FP64 ALU on this GPU, not by HBM
        fpk = fp64_peak["tflops"] if fp64_peak else FP64_NOMINAL_TFLOPS
        fpk_src = ("measured in this run by hj_fp64_fma_probe (DFMA throughput)" if fp64_peak
                   else "nominal GB300 FP64 rate (the probe did not run)")
        a64 = FP64_FLOPS_PER_UPDATE * ncell / (r64["avg_step_kernel_ms"] * 1e-3) / 1e12
        line["fp64_path"] = {
            "value": r64["value"], "unit": UNIT, "ms_per_step": r64["ms_per_step"], "steps": r64["K"],
            "latency_ms": r64["latency_ms"], "avg_step_kernel_ms": r64["avg_step_kernel_ms"],
            "hbm_frac": BYTES_PER_UPDATE["f64"] * ncell / (r64["avg_step_kernel_ms"] * 1e-3) / 1e9 / peak,
            "roofline": {"bound": "alu", "kernel": "hj_step_generic_kernel<double>", "achieved": a64,
                         "peak": fpk, "unit": "TFLOP/s", "frac": a64 / fpk, "peak_source": fpk_src,
                         "flops_per_update": FP64_FLOPS_PER_UPDATE,
                         "flops_counted": "1 DMUL + 4 DFMA per cell-update (dt folded into the coefficient table)"},
            "speedup_fp32_over_fp64": r32["value"] / r64["value"],
        }
    line["fp64_peak"] = fp64_peak
    if query is not None:
        fpk = fp64_peak["tflops"] if fp64_peak else FP64_NOMINAL_TFLOPS
        aq = QUERY_FP64_FLOPS * query["value"] / world / 1e12
        query["roofline"] = {"bound": "alu", "kernel": "query_kernel<float>", "achieved": aq, "peak": fpk,
                             "unit": "TFLOP/s", "frac": aq / fpk, "flops_per_query": QUERY_FP64_FLOPS,
                             "peak_source": "fp64_peak" if fp64_peak else "nominal GB300 FP64 rate",
                             "note": "FP64 flops only; 16 float-to-double conversions and 4 floors per query "
                                     "also occupy the FP64 unit"}
    if "q527" in results:
        rq = results["q527"]
        # Q5.27 codes move like FP32 (4 bytes); Sec. IV-B's error table compares
        # the fixed-point result with a floating-point one
        err = None
        if "f64" in results:
            err = float((outq.double() * 2.0 ** -27 - out64).abs().max().item())
        aq = BYTES_PER_UPDATE["q527"] * ncell / (rq["avg_step_kernel_ms"] * 1e-3) / 1e9
        line["q527_path"] = {
            "value": rq["value"], "unit": UNIT, "ms_per_step": rq["ms_per_step"], "steps": rq["K"],
            "latency_ms": rq["latency_ms"], "avg_step_kernel_ms": rq["avg_step_kernel_ms"],
            "kernel": "hj_step_tiled_kernel<FIXED>" if rq["kernel"] == hj.HJ_KERNEL_TILED else "hj_step_q527_kernel",
            "roofline": {"bound": "hbm", "achieved": aq, "peak": peak, "unit": "GB/s", "frac": aq / peak,
                         "bytes_per_update": BYTES_PER_UPDATE["q527"], "peak_source": f"{peak_kind} hbm_gbs"},
            "max_abs_err_vs_fp64": err,
            "tile": {k: v for k, v in (rq["tile"] or {}).items() if k != "tried"},
        }
    if "f32_bcast" in results:
        rb = results["f32_bcast"]
        ab = BYTES_PER_UPDATE["f32_bcast"] * ncell / (rb["avg_step_kernel_ms"] * 1e-3) / 1e9
        line["broadcast_v0_path"] = {
            "workload": WORKLOAD + " with V0 given as its 128x128 (x, y) field (Eq. init_V), FP32",
            "value": rb["value"], "unit": UNIT, "ms_per_step": rb["ms_per_step"], "steps": rb["K"],
            "avg_step_kernel_ms": rb["avg_step_kernel_ms"],
            "roofline": {"bound": "hbm", "achieved": ab, "peak": peak, "unit": "GB/s", "frac": ab / peak,
                         "bytes_per_update": BYTES_PER_UPDATE["f32_bcast"], "peak_source": f"{peak_kind} hbm_gbs"},
            "tile": {k: v for k, v in (rb["tile"] or {}).items() if k != "tried"},
        }
    if "f32_steer" in results:
        rs = results["f32_steer"]
        a_s = BYTES_PER_UPDATE["f32"] * ncell / (rs["avg_step_kernel_ms"] * 1e-3) / 1e9
        line["steer_path"] = {
            "workload": WORKLOAD + " with the steering car (a_max 1.5, delta_max pi/18, L 0.3 m), FP32",
            "value": rs["value"], "unit": UNIT, "ms_per_step": rs["ms_per_step"], "steps": rs["K"],
            "time_steps_per_solve": rs["time_steps_per_solve"], "avg_step_kernel_ms": rs["avg_step_kernel_ms"],
            "roofline": {"bound": "hbm", "achieved": a_s, "peak": peak, "unit": "GB/s", "frac": a_s / peak,
                         "bytes_per_update": BYTES_PER_UPDATE["f32"], "peak_source": f"{peak_kind} hbm_gbs"},
            "tile": {k: v for k, v in (rs["tile"] or {}).items() if k != "tried"},
        }
    if world == 1 and not args.no_oracle_accuracy and results_host:
        # after every timed region: the oracle's full solve of the same input
        line["accuracy"] = oracle_accuracy(w, V0, results_host, cpu_threads())
    if world == 1 and not args.no_cpu_baseline:
        nthreads = cpu_threads()
        rate, el, nst = oracle_sample(w, V0, args.cpu_sample_steps, nthreads)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                                "sample": f"{nst} oracle time steps of the {WORKLOAD} solve "
                                          f"({nst * ncell:.3e} cell-updates, {el:.1f} s), FP64, OpenMP over x"}
        # and the plain single-threaded oracle (one time step)
        rate1, el1, nst1 = oracle_sample(w, V0, 1, 1)
        line["cpu_baseline_single_thread"] = {
            "value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{nst1} oracle time step of the {WORKLOAD} solve ({nst1 * ncell:.3e} cell-updates, "
                      f"{el1:.1f} s), FP64, one thread"}
    print(json.dumps(line, default=json_default), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def json_default(o):
    """numpy scalars and arrays in the result line as plain JSON values."""
    if isinstance(o, np.generic):
        return o.item()
    if isinstance(o, np.ndarray):
        return o.tolist()
    raise TypeError(f"not JSON serialisable: {type(o).__name__}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-sample-steps", type=int, default=8)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--q527-steps", type=int, default=5)
    ap.add_argument("--no-q527", action="store_true")
    ap.add_argument("--bcast-steps", type=int, default=5)
    ap.add_argument("--no-bcast", action="store_true")
    ap.add_argument("--steer-steps", type=int, default=3)
    ap.add_argument("--no-steer", action="store_true")
    ap.add_argument("--no-query", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--small-only", action="store_true",
                    help="time only the small workloads and the paper's room (prints their JSON; not a bench line)")
    ap.add_argument("--large-only", action="store_true",
                    help="time only the 2048x2048x32x33 grid, tiled and generic kernels (prints its JSON; not a bench line)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-accuracy", action="store_true",
                    help="skip the oracle's full solve of the workload (about 75 s on 16 cores)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tile", default="", help="fixed tile shape ty,tv,xc,stages instead of autotuning")
    ap.add_argument("--bcast-tile", default="", help="fixed tile shape of the broadcast-V0 variant (default: --tile)")
    ap.add_argument("--q527-tile", default="", help="fixed tile shape of the Q5.27 variant (default: --tile)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-shape", default="", help="fixed batch kernel shape nconsumer,chunks instead of autotuning")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-rate", type=float, default=40.0)
    ap.add_argument("--serving-seconds", type=float, default=4.0)
    ap.add_argument("--serving-sweep", type=float, nargs="*",
                    default=[5.0, 10.0, 20.0, 40.0, 80.0, 120.0, 160.0, 240.0, 320.0, 480.0, 640.0, 960.0, 1280.0,
                             1920.0, 2560.0, 3840.0, 5120.0])
    ap.add_argument("--serving-sweep-seconds", type=float, default=1.5)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
