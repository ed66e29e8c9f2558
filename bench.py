#!/usr/bin/env python3
"""Benchmark of the Loop-of-stencil-reduce hot path on one GB300 (or N replicas).

A step is one complete solve of the workload through the C ABI: reset the
state to the seeded input, create a handle, run the device loop to its stop
rule, and (at the end of the timed region) read the reduced value.  The
default workload is the 8192 x 8192 Game of Life torus, uint8 cells,
Bernoulli(0.3), B3/S23, live-count + any-changed reduce, stop at a still state
or 2000 generations (it always runs the 2000).

Metric: Gcell-updates/s = cells x generations / device time.

Output: ONE JSON line on rank 0 with value (device-resident inputs), e2e (host
buffers, copies inside the timed region), roofline of the dominant kernel
(algorithmic bytes / CUDA-event time vs the measured HBM copy bandwidth),
cpu_baseline (the plain C oracle on the host cores, bounded sample), clocks
sampled during the timed region, and the plain one-launch-per-sweep path for
comparison.

--impl reference times the oracle itself (the CPU program that defines the
method) on the host cores for the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "life": dict(name="life_8192x8192_u8_torus_b3s23_{gens}gens", nx=8192, ny=8192, gens=2000,
                 bytes_per_cell_pass=2.0),
}
# Logic operations per 32 cells per generation in the bit-sliced update of the
# temporal-blocked kernel: 2 funnel shifts and 4 logic operations for the row's
# horizontal 2-bit sums, 6 for the vertical combination and the rule, and 3 for
# the two reduces the method takes every generation (popcount and add for the
# live count, or for "any cell changed").  The kernel runs the reduces in a
# pass's last generation only (a still state stays still), so this counts the
# method's work per cell update, not the instructions the kernel issues.
ALU_OPS_PER_CELL_GEN = 15.0 / 32.0
# Logic/shift lanes per SM per clock on sm_103: 4 sub-partitions x 16 lanes
# (ncu: one pipe_alu warp instruction per sub-partition every other cycle)
ALU_LANES_PER_SM = 64
SMS = 152
# bytes written between timed steps to flush the 129 MB L2
L2_FLUSH_BYTES = 256 << 20
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SOURCES = ["paper_1609_04567_gb300/csrc/life.cu", "paper_1609_04567_gb300/csrc/life_tb.cu",
                  "paper_1609_04567_gb300/csrc/slr_internal.cuh"]


def strip_comments(src: str) -> str:
    """C/C++ source without its comments and blank lines (string literals kept)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c == '"' or c == "'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(l.rstrip() for l in "".join(out).splitlines() if l.strip())


def kernel_hash() -> str:
    """Hash of the dominant kernel's code (comments left out: editing one does
    not invalidate the recorded ncu traffic)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic(workload: str, k: int):
    """DRAM bytes per launch of the dominant kernel, scaled from a committed ncu
    capture of a shorter run of the same kernel (bytes per pass x passes), if
    it was taken on the current kernel source; else None."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    with open(PROFILE_TRAFFIC) as fh:
        d = json.load(fh)
    e = d.get(f"life_8192_k{k}")
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    gens = int(workload.rsplit("_", 1)[-1].replace("gens", ""))
    return float(e.get("fixed_bytes", 0.0)) + float(e["dram_bytes_per_pass"]) * (-(-gens // k))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_cores() -> int:
    """Host cores this process may run on (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_life_sample(nx: int, ny: int, budget_s: float, cores: int = 1):
    """Time the oracle on the same torus for as many generations as fit in
    about budget_s seconds (at least one), on `cores` host threads (the
    oracle's OpenMP build; 1 = the plain single-threaded build).  Returns
    (gcells_per_s, gens, secs, threads used)."""
    import oracle
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(ny, nx)
    with oracle.threads(cores) as used:
        t0 = time.perf_counter()
        state, _ = oracle.life(cells, wrap=True, max_gens=1)
        one = time.perf_counter() - t0
        gens = max(1, min(16, int(budget_s / max(one, 1e-9)) - 1))
        t0 = time.perf_counter()
        oracle.life(state, wrap=True, max_gens=gens)
        secs = time.perf_counter() - t0
    total_gens, total_secs = gens + 1, secs + one
    return nx * ny * total_gens / total_secs / 1e9, total_gens, total_secs, used


def run_reference(args, wl, world, rank):
    if rank != 0:
        return 0
    import oracle
    from paper_1609_04567_gb300 import inputs
    oracle.build()
    # each step: one generation of the workload's own 8192 x 8192 torus through
    # the oracle on every host core (its OpenMP build: the rows of the sweep
    # shared among threads, the same values as the plain build); a bounded
    # sample of the 2000-generation run, the metric is per cell-update
    cores = host_cores()
    state = inputs.life_cells(wl["ny"], wl["nx"])
    with oracle.threads(cores) as used:
        for _ in range(args.warmup):
            state, _ = oracle.life(state, wrap=True, max_gens=1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            state, _ = oracle.life(state, wrap=True, max_gens=1)
        secs = time.perf_counter() - t0
    value = wl["nx"] * wl["ny"] * args.steps / secs / 1e9
    sample = (f"1 generation of the {wl['nx']}x{wl['ny']} torus per step, generations {args.warmup + 1}.."
              f"{args.warmup + args.steps} of the seeded input, plain C oracle on {used} threads")
    line = {
        "impl": "reference", "metric": "Gcell-updates/s", "value": value, "unit": "Gcell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": wl["name"].format(gens=wl["gens"]), "sample": sample},
        "cpu_baseline": {"value": value, "unit": "Gcell-updates/s", "cores": used, "kind": "oracle", "sample": sample,
                         "host_cores": cores},
        "e2e": {"value": value, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, wl, world, rank, local):
    import numpy as np
    import torch

    from paper_1609_04567_gb300 import build as slr_build
    from paper_1609_04567_gb300 import inputs, slr

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0 and not os.path.exists(slr.LIB_PATH):
        slr_build.build()
    barrier(world)
    slr.load()
    nx, ny, gens = wl["nx"], wl["ny"], args.gens
    cells = inputs.life_cells(ny, nx)
    pristine = torch.from_numpy(cells).to(dev)
    u = torch.empty_like(pristine)
    stream = torch.cuda.Stream(dev)
    desc = slr.slr_desc_init(slr.SLR_LIFE, nx, ny, 1, temporal_k=args.k, grid_ctas=args.grid_ctas)
    ws_bytes = slr.slr_workspace_size(desc)
    ws_t = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
    ws = ws_t.data_ptr() + ((-ws_t.data_ptr()) % 256)
    cell_updates = nx * ny * gens
    # written between timed steps so that no step finds the previous one's
    # lines in the L2 (129 MB): the 64 MiB input is smaller than the L2
    l2_flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # autotune the launch choices left to the library (untimed set-up: the
    # tuner's cache then feeds every slr_create below)
    tuned = None
    if not args.no_tune:
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            tuned = slr.tune(slr.SLR_LIFE, pristine, stream=stream, trial_iters=args.tune_iters,
                             loop=slr.SLR_LOOP_PERSISTENT, temporal_k=args.k, grid_ctas=args.grid_ctas)
        tuned["seconds"] = time.perf_counter() - t0

    def step(launch_events=None, loop=slr.SLR_LOOP_PERSISTENT):
        u.copy_(pristine, non_blocking=True)
        desc.loop = loop
        h = slr.slr_create(desc, u.data_ptr(), 0, ws, ws_bytes, stream.cuda_stream)
        if launch_events is not None:
            launch_events[0].record(stream)
        slr.slr_run_until(h, gens)
        if launch_events is not None:
            launch_events[1].record(stream)
        return h

    handles = []
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            handles.append(step())
        torch.cuda.synchronize(dev)
        first = slr.slr_reduce_value(handles[-1])
        for h in handles:
            slr.slr_destroy(h)
        handles = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
        clocks = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize(dev)
        clocks.start()
        for i in range(args.steps):
            l2_flush.zero_()                           # evict the previous step's lines, outside the step's events
            step_ev[i][0].record(stream)
            handles.append(step(ev[i]))
            step_ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        clk = clocks.stop()
        res = slr.slr_reduce_value(handles[-1])
        for h in handles:
            slr.slr_destroy(h)
    ms_total = sum(a.elapsed_time(b) for a, b in step_ev)
    ms_step = max_over_ranks(ms_total / args.steps, world)
    value = world * cell_updates / (ms_step / 1e3) / 1e9
    kern_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    # generations per pass: the tuner's choice, else the built-in default for
    # 8192 x 8192 on 152 SMs, 25 (the largest k up to 32 whose 1024 x (482 - 2k)
    # tiles fit the 152 co-resident CTAs)
    if tuned is not None:
        k_eff = tuned["temporal_k"]
    else:
        k_eff = 1 if args.k == 1 else (args.k if args.k > 0 else 25)
    passes = -(-gens // k_eff)
    # k = 1 moves every cell as uint8 per pass; the temporal-blocked path reads
    # and writes the uint8 grid once per launch and the bit-packed grid once
    # per pass (1/8 byte per cell each way)
    if k_eff == 1:
        algo_bytes = wl["bytes_per_cell_pass"] * nx * ny * passes
    else:
        algo_bytes = 2.0 * nx * ny + (0.25 * nx * ny) * (passes + 1)
    peak, peak_src = measured_peaks()
    achieved = algo_bytes / (kern_ms / 1e3) / 1e9
    traffic = recorded_traffic(wl["name"].format(gens=gens), k_eff)
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "peak_source": peak_src, "kernel_ms": kern_ms,
           "algorithmic_bytes_per_launch": algo_bytes, "passes_per_launch": passes,
           "generations_per_pass": k_eff}
    alu_ops = ALU_OPS_PER_CELL_GEN * nx * ny * gens
    alu_nominal = ALU_LANES_PER_SM * SMS * (clk.get("sm_mhz") or 2070.0) * 1e6 / 1e12
    # the logic pipe's rate measured on this GPU (independent three-input
    # logic operations on every SM, CUDA events), the roofline's denominator
    with torch.cuda.stream(stream):
        logic_rate, logic_ms = slr.slr_measure_logic_rate(stream.cuda_stream)
    alu_peak = logic_rate / 1e12
    alu = {"bound": "alu", "achieved": alu_ops / (kern_ms / 1e3) / 1e12, "peak": alu_peak, "unit": "Tops/s",
           "frac": alu_ops / (kern_ms / 1e3) / 1e12 / alu_peak, "traffic": traffic,
           "peak_source": "measured: slr_measure_logic_rate (independent lop3 on every SM, 64 warps/SM, "
                          f"CUDA events, {logic_ms:.2f} ms kernel)",
           "peak_nominal": alu_nominal,
           "peak_nominal_source": f"{ALU_LANES_PER_SM} lanes/SM x {SMS} SMs x median SM clock under load",
           "kernel_ms": kern_ms, "algorithmic_ops_per_launch": alu_ops}
    if k_eff == 1:
        roof = dict(hbm, kernel="life persistent loop, one generation per pass (all generations in one launch)")
    else:
        roof = dict(alu, kernel=f"life temporal-blocked persistent loop, {k_eff} generations per HBM pass",
                    hbm_per_pass=hbm)

    # plain path: one sweep launch + one reduce launch + host test per generation
    plain = None
    if not args.no_plain:
        with torch.cuda.stream(stream):
            pe = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            h = step(pe, loop=slr.SLR_LOOP_HOST)
            torch.cuda.synchronize(dev)
            wall = time.perf_counter() - t0
            pr = slr.slr_reduce_value(h)
            slr.slr_destroy(h)
        plain = {"value": cell_updates / wall / 1e9, "unit": "Gcell-updates/s", "ms_per_step": wall * 1e3,
                 "iters": pr[2], "count": pr[4], "same_result": pr[1:] == res[1:],
                 "what": "host-driven loop: per generation one sweep launch, one reduce launch, "
                         "a D2H copy of the reduced value and the test on the host"}

    # the same fused kernel family with one generation per pass (k = 1): the
    # "fused + device loop" column next to "fused + k-blocking" (the default)
    fused_k1 = None
    if not args.no_plain and args.k != 1:
        with torch.cuda.stream(stream):
            saved_k = desc.temporal_k
            desc.temporal_k = 1
            k1_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
            step()                                     # warm-up of the k = 1 kernel
            hs = [step(k1_ev[i]) for i in range(2)]
            torch.cuda.synchronize(dev)
            k1_ms = statistics.mean(a.elapsed_time(b) for a, b in k1_ev)
            k1r = slr.slr_reduce_value(hs[-1])
            for h in hs:
                slr.slr_destroy(h)
            desc.temporal_k = saved_k
        fused_k1 = {"value": cell_updates / (k1_ms / 1e3) / 1e9, "unit": "Gcell-updates/s", "kernel_ms": k1_ms,
                    "same_result": k1r[1:] == res[1:],
                    "what": "one generation per pass: uint8 grid read and written every generation"}

    # end to end through the C ABI with host buffers: every step copies its
    # input from pinned host memory, solves, and copies the final state and the
    # reduced value back.  Two slots (stream, device state, workspace, pinned
    # output) alternate, as a caller streaming grids would run them: a step's
    # copies overlap its neighbours' solves, and each solve's launch waits for
    # the previous one's (an event), so the solves still run one at a time
    host_in = torch.from_numpy(cells).pin_memory()
    desc.loop = slr.SLR_LOOP_PERSISTENT
    slots = []
    for i in range(2):
        s_ws = ws_t if i == 0 else torch.empty_like(ws_t)
        slots.append({"stream": stream if i == 0 else torch.cuda.Stream(dev),
                      "u": u if i == 0 else torch.empty_like(u),
                      "ws": s_ws.data_ptr() + ((-s_ws.data_ptr()) % 256), "ws_t": s_ws,
                      "out": torch.empty_like(host_in).pin_memory()})
    e2e_steps = max(2, min(args.steps, 10))
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    pending, prev = [], None
    e2e_res = None
    for i in range(e2e_steps + 1):
        if i < e2e_steps:
            sl = slots[i % 2]
            with torch.cuda.stream(sl["stream"]):
                sl["u"].copy_(host_in, non_blocking=True)
                if prev is not None:
                    sl["stream"].wait_event(prev)
                h = slr.slr_create(desc, sl["u"].data_ptr(), 0, sl["ws"], ws_bytes, sl["stream"].cuda_stream)
                slr.slr_run_until(h, gens)
                prev = torch.cuda.Event()
                prev.record(sl["stream"])
                sl["out"].copy_(sl["u"], non_blocking=True)
            pending.append(h)
        if len(pending) == 2 or (i == e2e_steps and pending):
            # the older step's reduced value (waits for its stream, the D2H included)
            h0 = pending.pop(0)
            e2e_res = slr.slr_reduce_value(h0)
            slr.slr_destroy(h0)
    wall = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    torch.cuda.synchronize(dev)
    for sl in slots:
        assert np.array_equal(sl["out"].numpy(), sl["u"].cpu().numpy())
    assert e2e_res[1:] == res[1:]
    e2e = {"value": world * cell_updates / wall / 1e9, "unit": "Gcell-updates/s",
           "h2d_bytes_per_step": int(host_in.numel()), "d2h_bytes_per_step": int(host_in.numel()) + 1024,
           "ms_per_step": wall * 1e3, "steps": e2e_steps,
           "what": "through the C ABI from pinned host buffers, two slots alternating: each step's H2D, "
                   "solve, D2H of the state and read of the reduced value are all inside the timed region; "
                   "copies overlap the neighbouring steps' solves, solves run one at a time"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle on every host core (OpenMP over rows) and on one core
        cores = host_cores()
        v, g, s, used = oracle_life_sample(nx, ny, args.cpu_budget, cores)
        v1, g1, s1, _ = oracle_life_sample(nx, ny, args.cpu_budget, 1)
        cpu = {"value": v, "unit": "Gcell-updates/s", "cores": used, "kind": "oracle", "host_cores": cores,
               "sample": f"{g} generations of the 8192x8192 torus, {s:.1f} s, plain C oracle on {used} threads",
               "single_core": {"value": v1, "unit": "Gcell-updates/s", "cores": 1, "kind": "oracle",
                               "sample": f"{g1} generations of the 8192x8192 torus, {s1:.1f} s, single-threaded"}}

    if rank == 0:
        line = {
            "metric": "Gcell-updates/s", "value": value, "unit": "Gcell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": wl["name"].format(gens=gens), "cells": nx * ny, "generations": gens,
                       "parallelism": f"replicas{world}", "loop": "persistent cooperative kernel",
                       "temporal_k": k_eff, "grid_ctas": tuned["grid_ctas"] if tuned else args.grid_ctas,
                       "tuned": tuned,
                       "l2": f"flushed: a {L2_FLUSH_BYTES >> 20} MiB buffer written between timed steps, "
                             "outside the per-step CUDA events"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "plain": plain,
            "fused_k1": fused_k1,
            "gpu_launches": args.steps,
            "clocks": clk,
            "result": {"iters": res[2], "live": res[4], "converged": res[3],
                       "same_as_warmup": first[1:] == res[1:]},
        }
        if world == 1 and not args.no_configs:
            line["configs"] = measure_configs(args)
        print(json.dumps(line), flush=True)
    return 0


def measure_configs(args):
    """The other configurations of the metric, each with its own CUDA-event
    times and clock record: the 256^2 FP64 Helmholtz solve (plain vs fused vs
    tuned), the 4096^2 restoration (fused EXACT/FAST vs plain, HBM and
    special-function fractions), the large single Jacobi grids (one sweep per
    HBM pass and temporal-blocked), the batch of 512 bf16 grids and a 512^3
    grid, FP64 defect correction on a batch of small grids, and a short run
    of the serving configuration."""
    import torch
    out = {}
    for name, fn in (("helmholtz_256_f64", measure_helmholtz), ("restore_4096_f32", measure_restore),
                     ("jacobi_large_grids", measure_jacobi),
                     ("batch_c4_bf16", lambda a: measure_batch(a, cpu_budget=min(a.cpu_budget, 5.0))),
                     ("batch_dc_2d_to_1e-10", lambda a: measure_batch_dc(a, max_side=80, plain_grids=2)),
                     ("serve_2000rps", lambda a: measure_serve_short(a, args.configs_serve_seconds))):
        t0 = time.perf_counter()
        try:
            out[name] = fn(args)
        except Exception as e:                     # one failed leg must not hide the others
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    return out


def _stream_time(stream, fn, steps, flush=None):
    """CUDA-event time of `steps` calls of fn() on `stream` (ms per call).
    With `flush` (a device buffer larger than the L2) the buffer is written
    before every call, outside that call's events, and the calls' own times
    are summed."""
    import torch
    if flush is None:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def run_helmholtz(args):
    print(json.dumps(measure_helmholtz(args)), flush=True)
    return 0


def measure_helmholtz(args):
    """2D Helmholtz Jacobi 256 x 256 FP64, tol 1e-6, cap 5000: time to solution."""
    import numpy as np
    import torch
    import oracle
    from paper_1609_04567_gb300 import inputs, slr
    slr.load()
    n = 256
    f = torch.from_numpy(inputs.helmholtz_rhs((n, n))).cuda()
    u = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    l2_flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    res = {}
    tuned = None
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    runs = [("fused_device_loop", slr.SLR_LOOP_PERSISTENT), ("plain", slr.SLR_LOOP_HOST)]
    if not args.no_tune:
        runs.append(("fused_tuned", slr.SLR_LOOP_AUTO))
    for name, loop in runs:
        if loop == slr.SLR_LOOP_AUTO:
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                tuned = slr.tune(slr.SLR_J2D5, u, f, stream=stream, trial_iters=64, tol=1e-6)
            tuned["seconds"] = time.perf_counter() - t0
        with torch.cuda.stream(stream):
            s = slr.Solver(slr.SLR_J2D5, u, f, stream=stream, tol=1e-6, loop=loop)

            def step():
                u.zero_()
                slr.slr_destroy(s.handle)
                s.handle = slr.slr_create(s.desc, u.data_ptr(), f.data_ptr(),
                                          s.ws.data_ptr() + ((-s.ws.data_ptr()) % 256),
                                          slr.slr_workspace_size(s.desc), stream.cuda_stream)
                s.run(5000)
            for _ in range(args.warmup):
                step()
            if loop == slr.SLR_LOOP_HOST:
                t0 = time.perf_counter()
                for _ in range(args.steps):
                    step()
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t0) / args.steps * 1e3
            else:
                ms = _stream_time(stream, step, args.steps, flush=l2_flush)
            r = s.result()
            s.close()
        res[name] = {"ms_per_solve": ms, "iters": r.iters, "gcell_per_s": n * n * r.iters / ms / 1e6}
    # fixed sweeps (test off): the per-sweep cost at steady state, which the
    # 26-sweep solve above hides behind its start-up
    fixed = {}
    fixed_sweeps = 1000
    for name, loop in (("fused_device_loop", slr.SLR_LOOP_PERSISTENT), ("plain", slr.SLR_LOOP_HOST)):
        with torch.cuda.stream(stream):
            s = slr.Solver(slr.SLR_J2D5, u, f, stream=stream, tol=0.0, loop=loop)

            def fstep():
                u.zero_()
                slr.slr_destroy(s.handle)
                s.handle = slr.slr_create(s.desc, u.data_ptr(), f.data_ptr(),
                                          s.ws.data_ptr() + ((-s.ws.data_ptr()) % 256),
                                          slr.slr_workspace_size(s.desc), stream.cuda_stream)
                s.run(fixed_sweeps)
            fstep()
            if loop == slr.SLR_LOOP_HOST:
                t0 = time.perf_counter()
                fstep()
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t0) * 1e3
            else:
                ms = _stream_time(stream, fstep, 3, flush=l2_flush)
            r = s.result(check=False)
            s.close()
        fixed[name] = {"ms": ms, "sweeps": r.iters, "us_per_sweep": ms * 1e3 / r.iters,
                       "gcell_per_s": n * n * r.iters / ms / 1e6}
    # the same solve written as user elemental functions (compiled at run time,
    # host-driven loop): the cost of the general form next to the fixed one
    user_src = """
__device__ slr_t slr_update(const slr_nbr &u, slr_t f, long long i, long long j, const double *p)
{
    const slr_t s = ((u(-1, 0) + u(1, 0)) + u(0, -1)) + u(0, 1);
    return (p[0] * f + s) / p[1];
}
__device__ double slr_delta(slr_t a, slr_t b) { return fabs(a - b); }
"""
    h = 1.0 / (n + 1)
    with torch.cuda.stream(stream):
        us = slr.UserSolver(user_src, u, f, params=(h * h, 4.0 + h * h), tol=1e-6, stream=stream)
    us.close()
    t0 = time.perf_counter()
    for _ in range(max(args.steps, 3)):
        u.zero_()
        with torch.cuda.stream(stream):
            us = slr.UserSolver(user_src, u, f, params=(h * h, 4.0 + h * h), tol=1e-6, stream=stream)
            us.run(5000)
            _, uit, _ = us.result()
            us.close()
    user_ms = (time.perf_counter() - t0) / max(args.steps, 3) * 1e3
    res["user_functions"] = {"ms_per_solve": user_ms, "iters": uit, "gcell_per_s": n * n * uit / user_ms / 1e6,
                             "what": "slr_update / slr_delta compiled at run time, the loop in one cooperative "
                                     "launch; wall time per solve including the handle's set-up and result read"}
    clk = clocks.stop()
    t0 = time.perf_counter()
    _, rr = oracle.j2d5(np.zeros((n, n)), f.cpu().numpy(), tol=1e-6, max_iters=5000)
    cpu_ms = (time.perf_counter() - t0) * 1e3
    cores = host_cores()
    with oracle.threads(cores) as used:
        t0 = time.perf_counter()
        oracle.j2d5(np.zeros((n, n)), f.cpu().numpy(), tol=1e-6, max_iters=5000)
        cpu_mt_ms = (time.perf_counter() - t0) * 1e3
    best = res.get("fused_tuned", res["fused_device_loop"])
    return {"workload": "helmholtz_256x256_f64_tol1e-6", "metric": "time-to-solution", "unit": "ms",
            "value": best["ms_per_solve"], "higher_is_better": False, "sweeps": rr.iters,
            "same_sweeps_as_oracle": all(v["iters"] == rr.iters for v in res.values()),
            "l2": "device-loop solves: L2 flushed before each, outside its events",
            "fused": res["fused_device_loop"], "plain": res["plain"], "tuned": res.get("fused_tuned"),
            "user_functions": res["user_functions"], "tuner": tuned, "clocks": clk,
            "fixed_1000_sweeps": dict(fixed, what="the convergence test off, 1000 sweeps: steady-state cost per "
                                                  "sweep of the fused device loop and of the plain host-driven one"),
            "cpu_baseline": {"value": cpu_mt_ms, "unit": "ms", "cores": used, "kind": "oracle",
                             "sample": "full solve", "host_cores": cores,
                             "single_core": {"value": cpu_ms, "unit": "ms", "cores": 1, "kind": "oracle",
                                             "sample": "full solve"}}}


def run_restore(args):
    print(json.dumps(measure_restore(args)), flush=True)
    return 0


# MUFU (special-function) lanes per SM per clock: 4 sub-partitions x 4
XU_LANES_PER_SM = 16


def measure_restore(args):
    """Restoration 4096 x 4096 FP32, 50% salt-and-pepper, tol 1e-3."""
    import numpy as np
    import torch
    import oracle
    from paper_1609_04567_gb300 import inputs, slr
    slr.load()
    n = 4096
    frame, _ = inputs.noisy_frame(n, n)
    mask = torch.from_numpy(inputs.noise_mask(frame)).cuda()
    init = torch.from_numpy(frame.astype(np.float32)).cuda()
    u = init.clone()
    stream = torch.cuda.Stream()
    l2_flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    res = {}
    tuned = None
    peak, peak_src = measured_peaks()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    # fused: the library default (temporal blocking, 8 sweeps per HBM pass);
    # fused_exact_k1: one sweep per pass (the TMA-tiled one-sweep kernel)
    runs = [("fused_exact", slr.SLR_LOOP_PERSISTENT, slr.SLR_MATH_EXACT, 0),
            ("fused_exact_k1", slr.SLR_LOOP_PERSISTENT, slr.SLR_MATH_EXACT, 1),
            ("fused_exact_k2", slr.SLR_LOOP_PERSISTENT, slr.SLR_MATH_EXACT, 2),
            ("fused_exact_k4", slr.SLR_LOOP_PERSISTENT, slr.SLR_MATH_EXACT, 4),
            ("fused_fast", slr.SLR_LOOP_PERSISTENT, slr.SLR_MATH_FAST, 0),
            ("plain_exact", slr.SLR_LOOP_HOST, slr.SLR_MATH_EXACT, 0)]
    if not args.no_tune:
        runs.append(("tuned_exact", slr.SLR_LOOP_AUTO, slr.SLR_MATH_EXACT, 0))
    for name, loop, math, k in runs:
        if loop == slr.SLR_LOOP_AUTO:
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                tuned = slr.tune(slr.SLR_RESTORE8, init, mask, stream=stream, trial_iters=16)
            tuned["seconds"] = time.perf_counter() - t0
        with torch.cuda.stream(stream):
            desc = slr.slr_desc_init(slr.SLR_RESTORE8, n, n, 1, loop=loop, math=math, temporal_k=k)
            wsb = slr.slr_workspace_size(desc)
            ws = torch.empty(wsb + 256, dtype=torch.uint8, device="cuda")
            wp = ws.data_ptr() + ((-ws.data_ptr()) % 256)
            hs = []

            def step():
                u.copy_(init)
                h = slr.slr_create(desc, u.data_ptr(), mask.data_ptr(), wp, wsb, stream.cuda_stream)
                slr.slr_run_until(h, 5000)
                hs.append(h)
            for _ in range(args.warmup):
                step()
            steps = args.steps if loop != slr.SLR_LOOP_HOST else 2
            if loop == slr.SLR_LOOP_HOST:
                t0 = time.perf_counter()
                for _ in range(steps):
                    step()
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t0) / steps * 1e3
            else:
                ms = _stream_time(stream, step, steps, flush=l2_flush)
            r = slr.slr_reduce_value(hs[-1])
            for h in hs:
                slr.slr_destroy(h)
        res[name] = {"ms_per_solve": ms, "iters": r[2], "value": r[1], "gcell_per_s": n * n * r[2] / ms / 1e6,
                     "hbm_gbs": 9.0 * n * n * r[2] / ms / 1e6}
    clk = clocks.stop()
    # the two ceilings of this stencil: HBM (9 algorithmic bytes per pixel and
    # sweep: the binary32 state read and written, the uint8 mask read) and the
    # special-function unit (each weight 1/sqrt(alpha + t^2) takes a square
    # root and a reciprocal: two MUFU operations per in-range neighbour of a
    # noisy pixel)
    m = inputs.noise_mask(frame).astype(bool)
    nbrs = np.zeros((n + 2, n + 2), dtype=np.int64)
    inside = np.zeros((n + 2, n + 2), dtype=np.int64)
    inside[1:-1, 1:-1] = 1
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy or dx:
                nbrs[1:-1, 1:-1] += inside[1 + dy:n + 1 + dy, 1 + dx:n + 1 + dx]
    weights = int(nbrs[1:-1, 1:-1][m].sum())
    clock_mhz = clk.get("sm_mhz") or 2070.0
    xu_peak = XU_LANES_PER_SM * SMS * clock_mhz * 1e6 / 1e12          # T MUFU ops/s
    for name, r in res.items():
        if name.startswith("plain"):
            continue
        r["hbm_frac"] = r["hbm_gbs"] / peak
        r["xu_tops"] = 2.0 * weights * r["iters"] / (r["ms_per_solve"] / 1e3) / 1e12
        r["xu_frac"] = r["xu_tops"] / xu_peak
    t0 = time.perf_counter()
    oracle.restore8(frame.astype(np.float32), inputs.noise_mask(frame), tol=0.0, max_iters=2)
    cpu_s = time.perf_counter() - t0
    cores = host_cores()
    with oracle.threads(cores) as used:
        t0 = time.perf_counter()
        oracle.restore8(frame.astype(np.float32), inputs.noise_mask(frame), tol=0.0, max_iters=4)
        cpu_mt_s = time.perf_counter() - t0
    return {"workload": "restore_4096x4096_f32_tol1e-3", "metric": "Gcell-updates/s", "unit": "Gcell-updates/s",
            "l2": "device-loop solves: L2 flushed before each, outside its events",
            "value": res.get("tuned_exact", res["fused_exact"])["gcell_per_s"], "fused_exact": res["fused_exact"],
            "fused_exact_k1": res["fused_exact_k1"], "fused_exact_k2": res["fused_exact_k2"],
            "fused_exact_k4": res["fused_exact_k4"],
            "fused_fast": res["fused_fast"], "plain_exact": res["plain_exact"], "tuned_exact": res.get("tuned_exact"),
            "tuner": tuned, "clocks": clk,
            "roofline": {"hbm_peak_gbs": peak, "peak_source": peak_src, "algorithmic_bytes_per_pixel_sweep": 9,
                         "xu_peak_tops": xu_peak, "mufu_ops_per_sweep": 2 * weights,
                         "xu_peak_source": f"{XU_LANES_PER_SM} MUFU lanes/SM x {SMS} SMs x median SM clock"},
            "cpu_baseline": {"value": n * n * 4 / cpu_mt_s / 1e9, "unit": "Gcell-updates/s", "cores": used,
                             "kind": "oracle", "sample": "4 sweeps of the 4096x4096 frame", "host_cores": cores,
                             "single_core": {"value": n * n * 2 / cpu_s / 1e9, "unit": "Gcell-updates/s",
                                             "cores": 1, "kind": "oracle",
                                             "sample": "2 sweeps of the 4096x4096 frame"}}}


def jacobi_case_of(name: str, slr, torch):
    """A Jacobi grid named {j2d5|j3d7}_{side x side[ x side]}_{f32|bf16|f16}[_k{K}][_s{S}]:
    stencil, shape (listed x first), storage, sweeps per pass (default 1) and
    sweeps (default 200 in 2D, 50 in 3D)."""
    parts = name.split("_")
    stencil = {"j2d5": slr.SLR_J2D5, "j3d7": slr.SLR_J3D7}[parts[0]]
    shape = tuple(int(v) for v in reversed(parts[1].split("x")))
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[parts[2]]
    k, sweeps = 1, 200 if len(shape) == 2 else 50
    for extra in parts[3:]:
        if extra[0] == "k":
            k = int(extra[1:])
        elif extra[0] == "s":
            sweeps = int(extra[1:])
        else:
            raise ValueError(f"unknown field {extra!r} in {name!r}")
    if (stencil == slr.SLR_J3D7) != (len(shape) == 3):
        raise ValueError(f"{name!r}: the stencil does not match the shape")
    return name, stencil, shape, dt, sweeps, k


def run_jacobi(args):
    print(json.dumps(measure_jacobi(args)), flush=True)
    return 0


def measure_jacobi(args):
    """Large single Jacobi grids, HBM-bound: 2D 5-point 8192 x 8192 in FP32 and
    BF16 storage, 3D 7-point 512^3 in BF16 storage; a fixed number of sweeps
    (convergence test never met) in one persistent launch; HBM GB/s from the
    algorithmic bytes per cell per sweep (read u and f, write u')."""
    import torch
    from paper_1609_04567_gb300 import inputs, slr
    slr.load()
    peak, peak_src = measured_peaks()
    stream = torch.cuda.Stream()
    # one sweep per HBM pass, and temporal blocking: k = 8 sweeps per pass in
    # 2D, k = 4 in 3D
    names = (args.jacobi_cases.split(",") if getattr(args, "jacobi_cases", "") else
             ["j2d5_8192x8192_f32", "j2d5_8192x8192_bf16", "j3d7_512x512x512_bf16", "j2d5_8192x8192_f32_k8",
              "j2d5_8192x8192_bf16_k8", "j3d7_512x512x512_bf16_k4_s48"])
    cases = [jacobi_case_of(n, slr, torch) for n in names]
    out = {}
    rhs = {}                                       # the seeded f of each shape, generated once
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for name, stencil, shape, dt, sweeps, k in cases:
        if shape not in rhs:
            rhs[shape] = torch.from_numpy(inputs.helmholtz_rhs(shape)).to(torch.float32)
        f = rhs[shape].to(dt).cuda()
        u = torch.zeros(shape, dtype=dt, device="cuda")
        with torch.cuda.stream(stream):
            s = slr.Solver(stencil, u, f, stream=stream, tol=0.0, temporal_k=k)

            def step():
                slr.slr_destroy(s.handle)
                s.handle = slr.slr_create(s.desc, u.data_ptr(), f.data_ptr(),
                                          s.ws.data_ptr() + ((-s.ws.data_ptr()) % 256),
                                          slr.slr_workspace_size(s.desc), stream.cuda_stream)
                s.run(sweeps)
            for _ in range(args.warmup):
                step()
            ms = _stream_time(stream, step, args.steps)
            r = s.result(check=False)
            s.close()
        cells = u.numel()
        bpc = 3 * u.element_size()
        gbs = bpc * cells * r.iters / (ms / 1e3) / 1e9
        out[name] = {"ms": ms, "sweeps": r.iters, "gcell_per_s": cells * r.iters / ms / 1e6,
                     "hbm_gbs": gbs, "frac": gbs / peak, "bytes_per_cell_sweep": bpc, "sweeps_per_pass": k}
        if k > 1:
            # HBM bytes the passes move (u and f read, u' written once per k sweeps)
            # next to the one-sweep-per-pass equivalent above
            out[name]["pass_hbm_gbs"] = gbs / k
            out[name]["pass_frac"] = gbs / k / peak
        del f, u
    clk = clocks.stop()
    return {"workload": "jacobi_large_grids", "metric": "HBM GB/s per sweep", "unit": "GB/s",
            "peak": peak, "peak_source": peak_src, "cases": out, "clocks": clk,
            "what": "fixed sweeps (tol 0) in one persistent launch; GB/s = 3 x element size x cells x sweeps / "
                    "CUDA-event time (u and f read, u' written once per sweep); k > 1: sweeps per HBM pass"}


def run_precision(args):
    """Mixed precision at the same accuracy: 2D Helmholtz (sigma 1, h = 1/(n+1),
    f ~ U[-1, 1], zero Dirichlet) solved until the change of the next FP64
    sweep, max |h^2 r / (4 + sigma h^2)|, is below 1e-10, three ways: the plain
    loop (one FP64 sweep launch, one reduce launch and a host test per
    iteration), the fused FP64 device loop, and FP32 inner Jacobi solves under
    FP64 defect correction.  Storage precisions (FP32, BF16, FP16 state with
    FP32 arithmetic) run the fused loop to tol 1e-6 next to FP64 at the same
    tol, and the plain FP32 loop to tol 1e-6.  Every result's error is
    max |u - u*| / max |u*| against the discrete solution u* (the FP64 oracle
    iterated to 1e-14); the oracle's own 1e-10 solve is the CPU leg of this
    workload and is timed.  Storage with fewer bits can stop at the cap: its
    +-1-ulp updates may never meet the tolerance."""
    import numpy as np
    import torch
    import oracle
    from paper_1609_04567_gb300 import inputs, slr
    slr.load()
    stream = torch.cuda.Stream()
    out = {}
    for n in args.precision_sides:
        f64 = inputs.helmholtz_rhs((n, n))
        f = torch.from_numpy(f64).cuda()
        t0 = time.perf_counter()
        ref10, rr10 = oracle.j2d5(np.zeros((n, n)), f64, tol=1e-10, max_iters=10 ** 6)
        cpu10 = time.perf_counter() - t0
        # the discrete solution, to well below either stopping rule's error
        ref, _ = oracle.j2d5(ref10, f64, tol=1e-14, max_iters=10 ** 6)
        scale = float(np.max(np.abs(ref)))

        def solve(name, dtype, reps, **fields):
            fs = f.to(torch.float32).to(dtype) if dtype != torch.float64 else f
            u = torch.zeros((n, n), dtype=dtype, device="cuda")
            with torch.cuda.stream(stream):
                s = slr.Solver(slr.SLR_J2D5, u, fs, stream=stream, **fields)

                def step():
                    u.zero_()
                    slr.slr_destroy(s.handle)
                    s.handle = slr.slr_create(s.desc, u.data_ptr(), fs.data_ptr(),
                                              s.ws.data_ptr() + ((-s.ws.data_ptr()) % 256),
                                              slr.slr_workspace_size(s.desc), stream.cuda_stream)
                    s.run(args.precision_cap)
                step()                                          # warm-up
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                for _ in range(reps):
                    step()
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t1) / reps * 1e3
                r = s.result(check=False)
                s.close()
            return u.double().cpu().numpy(), r, ms

        row = {"oracle_fp64_1e-10": {"sweeps": rr10.iters, "cpu_ms": cpu10 * 1e3}}
        for name, dtype, reps, fields in (
                ("plain_fp64_1e-10", torch.float64, 1, dict(tol=1e-10, loop=slr.SLR_LOOP_HOST)),
                ("fused_fp64_1e-10", torch.float64, 3, dict(tol=1e-10)),
                ("fused_dc_fp32_inner_1e-10", torch.float64, 3, dict(tol=1e-10, defect_correction=1)),
                ("plain_fp32_1e-6", torch.float32, 1, dict(tol=1e-6, loop=slr.SLR_LOOP_HOST)),
                ("fused_fp64_1e-6", torch.float64, 3, dict(tol=1e-6)),
                ("fused_fp32_1e-6", torch.float32, 3, dict(tol=1e-6)),
                ("fused_bf16_1e-6", torch.bfloat16, 3, dict(tol=1e-6)),
                ("fused_fp16_1e-6", torch.float16, 3, dict(tol=1e-6))):
            u, r, ms = solve(name, dtype, reps, **fields)
            row[name] = {"ms": ms, "iters": r.iters, "converged": r.converged, "value": r.value,
                         "rel_err_vs_fp64_oracle": float(np.max(np.abs(u - ref)) / scale)}
        out[f"{n}x{n}"] = row
    line = {"workload": "precision_helmholtz_2d", "metric": "time to the same stopping rule", "unit": "ms",
            "note": "defect correction iterations are corrections of 50 FP32 sweeps each", "cases": out}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    print(json.dumps(measure_batch(args)), flush=True)
    return 0


def measure_batch(args, cpu_budget=None):
    """512 2D Helmholtz grids (side log-uniform in [64, 1024]) + one 512^3 3D
    grid, bfloat16 storage, tol 1e-6, in one batch; against the same grids
    solved one after another (persistent loop per grid)."""
    import numpy as np
    import torch
    from paper_1609_04567_gb300 import inputs, slr
    slr.load()
    sides = inputs.batch_sides(512)
    grids = []
    for i, sd in enumerate(sides):
        f = torch.from_numpy(inputs.helmholtz_rhs((int(sd), int(sd)), stream=inputs.STREAM_BATCH_F0 + i)
                             .astype(np.float32)).to(torch.bfloat16).cuda()
        grids.append((f, torch.zeros_like(f)))
    n3 = args.batch3d
    if n3:
        f3 = torch.empty((n3, n3, n3), dtype=torch.bfloat16, device="cuda")
        f3_host = np.empty((n3, n3, n3), dtype=np.float32)
        flat = inputs.helmholtz_rhs((n3 * n3 * n3,), stream=inputs.STREAM_BATCH_F0 + 999)
        f3_host.reshape(-1)[:] = flat
        f3.copy_(torch.from_numpy(f3_host).to(torch.bfloat16))
        grids.append((f3, torch.zeros_like(f3)))
    cells = [g[0].numel() for g in grids]
    stream = torch.cuda.Stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    b = slr.Batch(len(grids) + 1, stream=stream)
    with torch.cuda.stream(stream):
        def batch_step():
            for _, u in grids:
                u.zero_()
            slots = [b.add(slr.SLR_J3D7 if u.dim() == 3 else slr.SLR_J2D5, u, f, 5000, tol=1e-6) for f, u in grids]
            b.run(100000)
            fin, running = b.poll()
            its = [b.result(s).iters for s in slots]
            conv = [b.result(s).converged for s in slots]
            for s in slots:
                b.remove(s)
            return its, conv
        batch_step()
        t0 = time.perf_counter()
        its, conv = batch_step()
        torch.cuda.synchronize()
        batch_s = time.perf_counter() - t0
    upd = float(sum(c * i for c, i in zip(cells, its)))
    # the same grids one after another, each with its own persistent launch
    t0 = time.perf_counter()
    seq_its = []
    with torch.cuda.stream(stream):
        for f, u in grids:
            u.zero_()
            s = slr.Solver(slr.SLR_J3D7 if u.dim() == 3 else slr.SLR_J2D5, u, f, stream=stream, tol=1e-6)
            s.run(5000)
            seq_its.append(s.result().iters)
            s.close()
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    clk = clocks.stop()
    b.close()
    budget = args.cpu_budget if cpu_budget is None else cpu_budget
    # the oracle on the host cores: the 2D grids of side <= 256 in order, each
    # to the same stop, until about cpu_budget seconds are spent; the whole
    # batch's CPU time projected from its rate at the batch's sweep counts
    import oracle
    cores = host_cores()
    cpu_cells = cpu_s = 0.0
    cpu_grids = 0
    cpu_same = True
    with oracle.threads(cores) as used:
        for (f, u), it in zip(grids, its):
            if u.dim() != 2 or u.shape[0] > 256:
                continue
            fo = f.float().cpu().numpy()
            t0 = time.perf_counter()
            _, rr = oracle.j2d5(np.zeros(fo.shape, dtype=np.float32), fo, tol=1e-6, max_iters=5000, storage="bf16")
            cpu_s += time.perf_counter() - t0
            cpu_cells += float(fo.size) * rr.iters
            cpu_grids += 1
            cpu_same = cpu_same and rr.iters == it
            if cpu_s > budget:
                break
    cpu_rate = cpu_cells / cpu_s if cpu_s > 0 else float("nan")
    cpu = {"value": cpu_rate / 1e9, "unit": "Gcell-updates/s", "cores": used, "kind": "oracle", "host_cores": cores,
           "sample": f"{cpu_grids} 2D grids of side <= 256 in batch order, each to its stop ({cpu_s:.1f} s)",
           "same_sweeps_as_gpu": cpu_same, "projected_s_whole_batch": upd / cpu_rate if cpu_s > 0 else None}
    line = {"workload": f"batch_512x2d_bf16_side64-1024_plus_{n3}^3_tol1e-6", "metric": "Gcell-updates/s",
            "unit": "Gcell-updates/s", "value": upd / batch_s / 1e9, "batch_s": batch_s,
            "sequential_s": seq_s, "sequential_gcell_per_s": upd / seq_s / 1e9, "same_iters": its == seq_its,
            "cell_updates": upd, "grids": len(grids), "max_sweeps": max(its), "min_sweeps": min(its),
            "converged": int(sum(conv)), "capped_at_5000": int(len(conv) - sum(conv)),
            "cpu_baseline": cpu, "clocks": clk,
            "note": "bfloat16 storage can trap Jacobi in a +-1 ulp cycle that never meets tol; such grids stop at the cap"}
    return line


def serve_oracle_sample(reqs, pool, budget_s: float):
    """The oracle on the host cores serving the same mix: requests in arrival
    order, each solved alone to its stop, until budget_s seconds are spent;
    the mean service time and the request rate it implies."""
    import numpy as np
    import oracle
    from paper_1609_04567_gb300 import serve
    cores = host_cores()
    spent, done, cells = 0.0, 0, 0.0
    with oracle.threads(cores) as used:
        for r in reqs:
            host_u, host_aux = pool.get(r.kind, r.side)
            t0 = time.perf_counter()
            if r.kind == serve.KIND_DENOISE:
                _, rr = oracle.restore8(host_u.numpy(), host_aux.numpy(), tol=1e-3, max_iters=5000)
            else:
                _, rr = oracle.j2d5(np.zeros((r.side, r.side)), host_aux.numpy(), tol=1e-6, max_iters=5000)
            spent += time.perf_counter() - t0
            done += 1
            cells += float(r.side) * r.side * rr.iters
            if spent > budget_s:
                break
    mean_ms = spent / max(done, 1) * 1e3
    return {"value": 1e3 / mean_ms, "unit": "requests/s", "cores": used, "kind": "oracle", "host_cores": cores,
            "sample": f"the first {done} requests of the mix in arrival order, each solved alone ({spent:.1f} s)",
            "mean_service_ms": mean_ms, "gcell_per_s": cells / spent / 1e9 if spent > 0 else None}


def measure_serve_short(args, seconds: float):
    """The serving configuration (Poisson 2000 req/s, half denoise jobs of
    sides 256-4096, half Helmholtz solves of sides 64-2048) for a short run:
    1 s of warm-up arrivals and `seconds` of measured arrivals, served to the
    last request."""
    import torch
    from paper_1609_04567_gb300 import serve, slr
    slr.load()
    reqs = serve.make_requests(seconds + 1.0, args.rate)
    srv = serve.Server(max_slots=1024, step_sweeps=args.step_sweeps, solo_cells=args.solo_cells or None,
                       light_solo=args.light_solo)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    st = srv.serve(reqs, warmup_s=1.0, time_limit_s=seconds * 6 + 30)
    clk = clocks.stop()
    srv.close()
    cpu = serve_oracle_sample(reqs, srv.pool, budget_s=5.0)
    num = (lambda x: None if x != x else x)
    offered = sum(1 for r in reqs if r.arrival >= 1.0)
    return {"workload": f"serve_poisson{args.rate:g}rps_denoise256-4096_solve64-2048_{seconds:g}s",
            "metric": "p50/p99 latency and throughput", "unit": "ms", "p50_ms": num(st.p50_ms),
            "p99_ms": num(st.p99_ms), "mean_ms": num(st.mean_ms), "throughput_rps": st.throughput_rps,
            "offered_rps": args.rate, "offered_after_warmup": offered, "completed_after_warmup": st.measured,
            "requests": st.requests, "completed": st.completed, "wall_s": st.wall_s,
            "gcell_per_s": st.gcell_per_s, "max_queue": st.max_queue, "max_in_flight": st.max_in_flight,
            "clocks": clk, "cpu_baseline": cpu,
            "what": "latency = arrival to the poll that sees the request finished; every arrival is served"}


def measure_batch_dc(args, max_side=None, plain_grids=None):
    """The precision half of the batched configuration: the 2D grids of the
    batch workload (sides log-uniform in [64, 1024]) whose side is at most
    `max_side`, solved until the change the next FP64 sweep would make
    (max |h^2 r / (4 + sigma h^2)|) is below 1e-10, three ways: FP64 defect
    correction around binary32 inner sweeps, all grids in one batched launch;
    the fused FP64 device loop, one grid after another; and the plain
    one-launch-per-sweep FP64 loop with a host test per sweep (timed on the
    first `plain_grids` grids, per grid).  Every result's error is stated
    against the discrete solution (the fused FP64 loop run to 1e-14).  Larger
    grids need of the order of 10^5 to 10^6 sweeps to 1e-10 and are left out."""
    import numpy as np
    import torch
    from paper_1609_04567_gb300 import inputs, slr
    slr.load()
    max_side = max_side or args.dc_max_side
    plain_grids = plain_grids if plain_grids is not None else args.dc_plain_grids
    sides = [int(x) for x in inputs.batch_sides(512)]
    pick = [i for i, sd in enumerate(sides) if sd <= max_side]
    fs = [torch.from_numpy(inputs.batch_grid_rhs(i, sides[i])).cuda() for i in pick]
    stream = torch.cuda.Stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()

    def fused(f, tol, loop=slr.SLR_LOOP_PERSISTENT, **kw):
        u = torch.zeros_like(f)
        with torch.cuda.stream(stream):
            sv = slr.Solver(slr.SLR_J2D5, u, f, stream=stream, tol=tol, loop=loop, **kw)
            sv.run(10 ** 7)
            r = sv.result(check=False)
            sv.close()
        return u, r
    exact = [fused(f, 1e-14)[0] for f in fs]                 # the discrete solutions
    scale = [float(e.abs().max()) for e in exact]
    # FP64 defect correction, every grid in one batched launch
    b = slr.Batch(len(fs) + 1, stream=stream)
    us = [torch.zeros_like(f) for f in fs]
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        slots = [b.add(slr.SLR_J2D5, u, f, 100000, tol=1e-10, defect_correction=1) for u, f in zip(us, fs)]
        b.run(10 ** 8)
        _, running = b.poll()
        dc_s = time.perf_counter() - t0
    res = [b.result(sl) for sl in slots]
    b.close()
    dc_err = [float((u - e).abs().max()) / sc for u, e, sc in zip(us, exact, scale)]
    # the fused FP64 loop, one grid after another
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fr = [fused(f, 1e-10) for f in fs]
    fused_s = time.perf_counter() - t0
    fused_err = [float((u - e).abs().max()) / sc for (u, _), e, sc in zip(fr, exact, scale)]
    # the plain loop on the first grids
    t0 = time.perf_counter()
    pr = [fused(f, 1e-10, loop=slr.SLR_LOOP_HOST) for f in fs[:plain_grids]]
    plain_s = time.perf_counter() - t0
    plain_err = [float((u - e).abs().max()) / sc for (u, _), e, sc in zip(pr, exact, scale)]
    clk = clocks.stop()
    n_plain = max(1, len(pr))
    return {"workload": f"batch_dc_2d_sides64-{max_side}_to_1e-10", "grids": len(fs), "sides": [sides[i] for i in pick],
            "metric": "time to the FP64 stopping rule 1e-10", "unit": "s", "value": dc_s,
            "all_converged": running == 0 and all(r.converged for r in res),
            "dc_batch": {"seconds": dc_s, "corrections_max": max(r.iters for r in res),
                         "max_rel_err_vs_discrete": max(dc_err)},
            "fused_fp64_sequential": {"seconds": fused_s, "sweeps_max": max(r.iters for _, r in fr),
                                      "max_rel_err_vs_discrete": max(fused_err)},
            "plain_fp64_host_loop": {"grids": len(pr), "seconds": plain_s, "seconds_per_grid": plain_s / n_plain,
                                     "projected_seconds_all_grids": plain_s / n_plain * len(fs),
                                     "max_rel_err_vs_discrete": max(plain_err) if plain_err else None},
            "speedup_vs_plain_projected": plain_s / n_plain * len(fs) / dc_s,
            "speedup_vs_fused_sequential": fused_s / dc_s, "clocks": clk,
            "what": "defect correction: 50 binary32 sweeps per FP64 correction; the error is max |u - u*| / max |u*| "
                    "against the fused FP64 loop run to 1e-14"}


def run_batch_dc(args):
    print(json.dumps(measure_batch_dc(args)), flush=True)
    return 0


def run_serve(args):
    """Continuous-batching serving: Poisson arrivals at 2000 requests/s, half
    denoise (sides 256-4096) and half Helmholtz solves (sides 64-2048)."""
    import torch
    from paper_1609_04567_gb300 import serve, slr
    slr.load()
    reqs = serve.make_requests(args.serve_seconds + 1.0, args.rate)
    srv = serve.Server(max_slots=1024, step_sweeps=args.step_sweeps, solo_cells=args.solo_cells or None,
                       light_solo=args.light_solo)
    st = srv.serve(reqs, warmup_s=1.0, time_limit_s=args.serve_seconds * 6 + 30)
    srv.close()
    # the same arrivals served by a queue alone, one request at a time: with the
    # plain host-driven loop (one sweep launch, one reduce launch and a host
    # test per sweep) and with the fused device loop; requests not started by
    # the end of the arrival window are left unserved
    num = (lambda x: None if x != x else x)                # NaN (no latency sample) -> null
    fifo = {}
    for name, loop in (("queue_plain_host_loop", slr.SLR_LOOP_HOST), ("queue_fused_device_loop", slr.SLR_LOOP_PERSISTENT)):
        q = serve.make_requests(args.serve_seconds + 1.0, args.rate)
        fs = serve.serve_fifo(q, loop=loop, warmup_s=1.0, time_limit_s=args.serve_seconds + 1.0, pool=srv.pool)
        fifo[name] = {"p50_ms": num(fs.p50_ms), "p99_ms": num(fs.p99_ms), "mean_ms": num(fs.mean_ms),
                      "latency_sample": fs.measured, "throughput_rps": fs.throughput_rps,
                      "gcell_per_s": fs.gcell_per_s, "requests": fs.requests, "completed": fs.completed,
                      "unserved": fs.requests - fs.completed, "max_queue": fs.max_queue, "wall_s": fs.wall_s}
    line = {"workload": f"serve_poisson{args.rate:g}rps_denoise256-4096_solve64-2048",
            "metric": "p50/p99 latency and throughput", "unit": "ms", "p50_ms": num(st.p50_ms),
            "p99_ms": num(st.p99_ms), "mean_ms": num(st.mean_ms), "throughput_rps": st.throughput_rps, "gcell_per_s": st.gcell_per_s,
            "requests": st.requests, "completed": st.completed, "wall_s": st.wall_s, "steps": st.steps,
            "max_in_flight": st.max_in_flight, "max_queue": st.max_queue,
            "solo_lane": {"min_cells": args.solo_cells, "light_solo": args.light_solo,
                          "requests": sum(r.lane == "solo" for r in srv.done),
                          "what": "denoise jobs of at least min_cells pixels, and any request while fewer than "
                                  "light_solo jobs are in the lane, run to their stop on solvers of their own, "
                                  "one after another, beside the batch"},
            "latency_sample": st.measured,
            "cpu_baseline": serve_oracle_sample(reqs, srv.pool, budget_s=5.0),
            "queue_alone": dict(fifo, what="the same arrivals, one request at a time in arrival order, each "
                                           "solved alone; p50/p99 over the served requests that arrived after "
                                           "the 1 s warm-up (latency_sample of them; null when none)")}
    print(json.dumps(line), flush=True)
    return 0


def run_video(args):
    """The video restoration stream of Sec. 4.3, pipe(read, detect,
    ofarm(restore), write): 100-frame streams at VGA, 720p and 1080p (each a
    seeded permutation of 4 distinct 50% salt-and-pepper frames of the
    restoration generator), pinned host frames in and out, adaptive median
    detection (windows up to 7 x 7), EXACT restoration to mean |delta| < 1e-3,
    rounding back to uint8, with 1, 2 and 4 frames in flight.  The oracle's
    detection and restoration of one VGA frame is the CPU leg."""
    import numpy as np
    import torch
    import oracle
    from paper_1609_04567_gb300 import slr, video
    slr.load()
    out = {}
    for name, (ny, nx) in [("vga_640x480", (480, 640)), ("720p_1280x720", (720, 1280)),
                           ("1080p_1920x1080", (1080, 1920))]:
        frames, _ = video.make_video(ny, nx, args.video_frames, distinct=4)
        host_in = [torch.from_numpy(f).pin_memory() for f in frames]
        host_out = [torch.empty((ny, nx), dtype=torch.uint8).pin_memory() for _ in frames]
        row = {}
        for lanes in (1, 2, 4):
            p = video.VideoPipeline(ny, nx, lanes=lanes)
            p.run(host_in[:lanes * 2], host_out[:lanes * 2])           # warm-up
            st = p.run(host_in, host_out)
            p.close()
            row[f"lanes{lanes}"] = {"fps": st.fps, "wall_s": st.wall_s, "p50_ms": st.p50_ms, "p99_ms": st.p99_ms,
                                    "mean_sweeps": st.mean_iters, "gcell_per_s": st.gcell_per_s}
        out[name] = row
    # CPU leg: the oracle's detection and restoration of one VGA frame
    frames, _ = video.make_video(480, 640, 1, distinct=1)
    t0 = time.perf_counter()
    m = oracle.amf_detect(frames[0], wmax=7)
    ref, rr = oracle.restore8(frames[0].astype(np.float32), m, tol=1e-3, max_iters=5000)
    cpu_s = time.perf_counter() - t0
    line = {"workload": f"video_restore_{args.video_frames}frames_vga_720p_1080p", "metric": "frames/s",
            "unit": "frames/s", "cases": out,
            "cpu_baseline": {"value": 1.0 / cpu_s, "unit": "frames/s", "cores": 1, "kind": "oracle",
                             "sample": f"one 640x480 frame, detection and {rr.iters} restoration sweeps"}}
    print(json.dumps(line), flush=True)
    return 0


def run_sobel(args):
    """The Sobel edge detector of Sec. 4.2 (one stencil sweep, no reduce) on
    uint8 images of the paper's sides 512, 4096 and 16384 (smooth synthetic
    images of the restoration generator): the kernel alone with the image
    resident (HBM bytes: 1 read + 1 written per pixel; the 16384 image is
    larger than L2), end to end with the pinned host copies in and out, and
    image streams pipe(read, sobel, write) with 3 images in flight.  The
    oracle filtering one 4096 x 4096 image is the CPU leg."""
    import numpy as np
    import torch
    import oracle
    from paper_1609_04567_gb300 import inputs, slr, video
    slr.load()
    peak, peak_src = measured_peaks()
    out = {}
    base = inputs.smooth_image(4096, 4096, seed=2)
    for side, stream_n in ((512, 100), (4096, 100), (16384, 12)):
        img_np = base[:side, :side] if side <= 4096 else np.tile(base, (side // 4096, side // 4096))
        img_np = np.ascontiguousarray(img_np)
        img = torch.from_numpy(img_np).cuda()
        dst = torch.empty_like(img)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            for _ in range(args.warmup):
                slr.sobel(img, dst, stream=st)
            reps = 200 if side <= 4096 else 20
            ms = _stream_time(st, lambda: slr.sobel(img, dst, stream=st), reps)
        host_in = torch.from_numpy(img_np).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        with torch.cuda.stream(st):
            def e2e():
                img.copy_(host_in, non_blocking=True)
                slr.sobel(img, dst, stream=st)
                host_out.copy_(dst, non_blocking=True)
            for _ in range(args.warmup):
                e2e()
            e2e_ms = _stream_time(st, e2e, 20)
        px = side * side
        row = {"kernel_ms": ms, "gpixel_per_s": px / ms / 1e6, "hbm_gbs": 2 * px / ms / 1e6,
               "frac": 2 * px / ms / 1e6 / peak, "e2e_ms": e2e_ms, "e2e_gpixel_per_s": px / e2e_ms / 1e6,
               "h2d_bytes": px, "d2h_bytes": px,
               "l2_resident": 2 * px < 126 * 2 ** 20}   # in and out fit L2: the kernel rate is not an HBM rate
        imgs = [host_in] * stream_n
        outs = [torch.empty_like(host_in).pin_memory() for _ in range(min(stream_n, 8))]
        outs = [outs[k % len(outs)] for k in range(stream_n)]
        video.sobel_stream(imgs[:6], outs[:6], lanes=3)
        s = video.sobel_stream(imgs, outs, lanes=3)
        row["stream"] = {"images": s.images, "images_per_s": s.images_per_s, "gbytes_per_s": s.gbytes_per_s,
                         "in_flight": s.lanes}
        out[f"{side}x{side}"] = row
        del img, dst, host_in, host_out, imgs, outs
        torch.cuda.empty_cache()
    t0 = time.perf_counter()
    oracle.sobel(base)
    cpu_s = time.perf_counter() - t0
    line = {"workload": "sobel_512_4096_16384", "metric": "Gpixel/s", "unit": "Gpixel/s", "peak_gbs": peak,
            "peak_source": peak_src, "cases": out,
            "cpu_baseline": {"value": 4096 * 4096 / cpu_s / 1e9, "unit": "Gpixel/s", "cores": 1, "kind": "oracle",
                             "sample": "one 4096 x 4096 image"}}
    print(json.dumps(line), flush=True)
    return 0


def run_split(args):
    """One grid over row blocks (the 1:n deployment of Sec. 3.3): the 8192 x
    8192 Life torus cut into --split-blocks row blocks with `--split-halo`
    copied-in rows, exchanged every pass.  Under torchrun each rank holds one
    block on its own GPU and the halos and partial reduces travel over NCCL;
    on one process all blocks share the GPU and the halos are device copies.
    The result is checked against the same grid solved whole (the library's
    own single-grid loop).  Metric: cell-updates of the whole grid per second."""
    import hashlib
    import torch
    from paper_1609_04567_gb300 import inputs, slr
    from paper_1609_04567_gb300 import split as S
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    slr.load()
    n, gens, H = 8192, args.split_gens, args.split_halo
    cells = inputs.life_cells(n, n)
    parts = world if world > 1 else args.split_blocks
    bounds = S.row_blocks(n, parts)
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=world)
        mine = [bounds[rank]]
        ex = S.ProcessGroupExchanger(device="cuda")
    else:
        mine = bounds
        ex = S.LocalExchanger()
    desc = slr.slr_desc_init(slr.SLR_LIFE, n, n, 1)

    def solve():
        blocks = [(torch.from_numpy(cells[lo:hi]).cuda(), None, lo, hi) for lo, hi in mine]
        loop = S.SplitLoop(slr.SLR_LIFE, blocks, n, halo=H, exchanger=ex, sweeper=S.DeviceSweeper(desc), tol=0.0,
                           wrap=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = loop.run(gens)
        torch.cuda.synchronize()
        return loop, r, time.perf_counter() - t0
    solve()                                            # warm-up
    times = []
    for _ in range(max(1, args.steps)):
        loop, r, secs = solve()
        times.append(secs)
    secs = max_over_ranks(statistics.median(times), world)
    ok = None
    if rank == 0 and world == 1:
        whole = torch.from_numpy(cells).cuda()
        sv = slr.Solver(slr.SLR_LIFE, whole)
        sv.run(gens)
        rw = sv.result()
        sv.close()
        got = torch.cat([loop.own_rows(i) for i in range(len(mine))])
        ok = bool(torch.equal(got, whole)) and (r.iters, r.count) == (rw.iters, rw.count)
    if rank == 0:
        print(json.dumps({
            "workload": f"split_life_{n}x{n}_torus_{gens}gens", "metric": "Gcell-updates/s",
            "unit": "Gcell-updates/s", "value": n * n * gens / secs / 1e9, "n_gpus": world, "blocks": parts,
            "halo_rows": H, "passes": r.passes, "seconds": secs, "iters": r.iters, "live": r.count,
            "scaling": "strong", "same_as_whole_grid": ok,
            "what": "host-driven loop per pass: halo exchange, halo sweeps of the device block kernel (one cell "
                    "per thread, the whole-grid sweep's operations), partial reduces combined on the host"}),
              flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="life",
                    choices=["life", "helmholtz", "restore", "jacobi", "precision", "batch", "serve", "video", "sobel",
                             "split", "batch_dc"])
    ap.add_argument("--video-frames", type=int, default=100, help="frames per stream of the video workload")
    ap.add_argument("--dc-max-side", type=int, default=96, help="batch_dc workload: largest grid side")
    ap.add_argument("--dc-plain-grids", type=int, default=4, help="batch_dc workload: grids timed on the plain loop")
    ap.add_argument("--split-blocks", type=int, default=2, help="split workload on one process: row blocks")
    ap.add_argument("--split-halo", type=int, default=8, help="split workload: copied-in rows per side")
    ap.add_argument("--split-gens", type=int, default=200, help="split workload: generations")
    ap.add_argument("--batch3d", type=int, default=512, help="side of the 3D grid of the batch workload (0: none)")
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--step-sweeps", type=int, default=64)
    ap.add_argument("--solo-cells", type=int, default=1024 * 1024,
                    help="serving: denoise jobs of at least this many pixels take the solo lane (0: none)")
    ap.add_argument("--light-solo", type=int, default=4,
                    help="serving: any request takes the solo lane while fewer than this many jobs are in it")
    ap.add_argument("--jacobi-cases", default="",
                    help="jacobi workload: comma-separated grids named {j2d5|j3d7}_{NxN[xN]}_{f32|bf16|f16}"
                         "[_k{sweeps per pass}][_s{sweeps}] (default: the large grids)")
    ap.add_argument("--k", type=int, default=0, help="generations per HBM pass (0 = library choice)")
    ap.add_argument("--gens", type=int, default=2000,
                    help="generations per solve (the workload has 2000; shorter runs are for profiler captures "
                         "and are named as such in config.workload)")
    ap.add_argument("--precision-sides", type=int, nargs="+", default=[64, 128],
                    help="grid sides of the precision workload")
    ap.add_argument("--precision-cap", type=int, default=200000, help="iteration cap of the precision workload")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (built-in launch defaults)")
    ap.add_argument("--grid-ctas", type=int, default=0, help="CTAs of the persistent launch (0 = library choice)")
    ap.add_argument("--tune-iters", type=int, default=240, help="iterations per autotuner trial")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload: leave out the other configurations (Helmholtz, restoration, "
                         "large Jacobi grids, serving) from the line")
    ap.add_argument("--configs-serve-seconds", type=float, default=2.5,
                    help="seconds of measured arrivals of the serving configuration in the default line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload != "life":
        fn = {"helmholtz": run_helmholtz, "restore": run_restore, "jacobi": run_jacobi, "precision": run_precision,
              "batch": run_batch, "serve": run_serve, "video": run_video, "sobel": run_sobel, "split": run_split,
              "batch_dc": run_batch_dc}
        return fn[args.workload](args)
    wl = WORKLOADS[args.workload]
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, wl, world, rank)
    return run_ours(args, wl, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
