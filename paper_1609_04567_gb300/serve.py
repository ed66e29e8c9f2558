"""Continuous-batching serving loop over the batched persistent launch.

Requests (restoration "denoise" jobs and 2D Helmholtz "solve" jobs of mixed
sizes) arrive as a Poisson process.  The server keeps ONE resident batch
(``slr.Batch``): each loop iteration admits every request that has arrived,
for which device memory and a batch slot are free, runs a bounded number of
sweeps of everything in the batch (one persistent launch), and retires the
requests whose loops stopped.  A request that arrives while others are on the
GPU joins them at the next iteration; its work overlaps theirs in the same
launch.  This is the stream composition of Sec. 4.3 (read, restore, write over
a stream of frames) served on one GPU, with latency measured per request.

Admission is by device memory: a request needs its state, its auxiliary input
(f or mask) and one scratch buffer; it is admitted only while the sum of the
footprints of admitted requests stays inside the budget (by default a fraction
of the free memory reported by the driver at start-up).

Large denoise jobs (at least ``solo_cells`` pixels) take a second lane: each
gets its own solver (the temporal-blocked restoration loop, which restores a
large frame several times faster than the batch's warp units) and runs to its
stop in one launch, while the batch steps on the first stream.  Each solo job
has a stream of its own from a small pool: its input copies start at once and
overlap the jobs before it, and its launch waits (by an event) for the previous
solo job's, so the lane runs its jobs one after another in admission order;
the host sees a job finish through its event and reads its result from its own
stream, without waiting for the jobs queued behind it.  At light load any
request takes the solo lane while fewer than ``light_solo`` jobs are in it: a
request then has the GPU to itself, as in a queue over the fused loop, and
the batch takes the overflow.  Results do not depend on the lane.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs, slr

KIND_DENOISE, KIND_SOLVE = "denoise", "solve"


@dataclass
class Request:
    rid: int
    kind: str
    side: int
    arrival: float                 # seconds after the start of the run
    seed: int = 0
    admitted: float | None = None
    finished: float | None = None
    iters: int = 0
    converged: bool = False
    value: float = 0.0
    slot: int = -1
    tensors: tuple = field(default=(), repr=False)
    lane: str = ""                 # "batch" or "solo", set at admission
    solver: object = field(default=None, repr=False)   # the solo lane's solver
    event: object = field(default=None, repr=False)    # the solo lane's completion event


def bucket_sides(lo: int, hi: int, n: int) -> list[int]:
    """n log-spaced sides in [lo, hi] (rounded to multiples of 8)."""
    return sorted({int(round(math.exp(math.log(lo) + i * (math.log(hi) - math.log(lo)) / (n - 1)) / 8.0)) * 8
                   for i in range(n)})


def make_requests(duration_s: float, rate: float, *, seed: int = inputs.DEFAULT_SEED, denoise_share: float = 0.5,
                  denoise_sides=(256, 4096), solve_sides=(64, 2048), buckets: int = 8) -> list[Request]:
    """Poisson arrivals at `rate` per second for `duration_s` seconds; each
    request is a denoise job with probability `denoise_share`, else a solve;
    sides are log-uniform over a set of `buckets` log-spaced sizes."""
    n_max = int(rate * duration_s * 1.5) + 16
    gaps = inputs.exp_gaps(n_max, rate, seed=seed)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < duration_s]
    u = inputs.uniform01(seed, inputs.STREAM_ARRIVALS + 1, 2 * len(arrivals)).reshape(-1, 2)
    dsides, ssides = bucket_sides(*denoise_sides, buckets), bucket_sides(*solve_sides, buckets)
    reqs = []
    for i, t in enumerate(arrivals):
        if u[i, 0] < denoise_share:
            reqs.append(Request(i, KIND_DENOISE, dsides[min(int(u[i, 1] * len(dsides)), len(dsides) - 1)], float(t)))
        else:
            reqs.append(Request(i, KIND_SOLVE, ssides[min(int(u[i, 1] * len(ssides)), len(ssides) - 1)], float(t)))
    return reqs


class InputPool:
    """Pinned host inputs per (kind, side): the synthetic frames and
    right-hand sides of the workload, generated once."""

    def __init__(self, seed: int = inputs.DEFAULT_SEED):
        self.seed = seed
        self.cache = {}

    def get(self, kind: str, side: int):
        import torch
        key = (kind, side)
        if key not in self.cache:
            if kind == KIND_DENOISE:
                frame, _ = inputs.noisy_frame(side, side, seed=self.seed + side)
                mask = inputs.noise_mask(frame)
                self.cache[key] = (torch.from_numpy(frame.astype(np.float32)).pin_memory(),
                                   torch.from_numpy(mask).pin_memory())
            else:
                f = inputs.helmholtz_rhs((side, side), seed=self.seed + side)
                self.cache[key] = (torch.zeros((side, side), dtype=torch.float64).pin_memory(),
                                   torch.from_numpy(f).pin_memory())
        return self.cache[key]


def footprint(kind: str, side: int) -> int:
    cells = side * side
    return cells * (4 + 1 + 4) if kind == KIND_DENOISE else cells * (8 + 8 + 8)


@dataclass
class ServeStats:
    requests: int
    completed: int
    wall_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    throughput_rps: float
    cell_updates: float
    gcell_per_s: float
    steps: int
    max_in_flight: int
    max_queue: int
    budget_bytes: int
    measured: int = 0              # completed requests that arrived after the warm-up (the latency sample)


class Server:
    """One resident batch served with continuous batching."""

    def __init__(self, *, max_slots: int = 1024, budget_bytes: int | None = None, step_sweeps: int = 64,
                 denoise_tol: float = 1e-3, solve_tol: float = 1e-6, cap: int = 5000, device=None,
                 solo_cells: int | None = 1024 * 1024, solo_streams: int = 64, light_solo: int = 4):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.stream = torch.cuda.Stream(self.device)
        # one solo job per stream at a time: a job's result is read on its own
        # stream, which then holds no later job
        self.solo_streams = [torch.cuda.Stream(self.device) for _ in range(max(1, solo_streams))]
        self.solo_issued = 0
        self.solo_tail = None     # completion event of the last solo job launched
        self.batch = slr.Batch(max_slots, device=self.device, stream=self.stream)
        self.max_slots = max_slots
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(free * 0.6)
        self.budget = budget_bytes
        self.in_use = 0
        self.step_sweeps = step_sweeps
        self.tol = {KIND_DENOISE: denoise_tol, KIND_SOLVE: solve_tol}
        self.cap = cap
        self.pool = InputPool()
        self.active = {}          # batch slot -> request
        self.solo = {}            # request id -> request with its own solver (admission order)
        self.solo_cells = solo_cells
        self.light_solo = light_solo

    def is_solo(self, r: Request) -> bool:
        return self.solo_cells is not None and r.kind == KIND_DENOISE and r.side * r.side >= self.solo_cells

    def takes_solo(self, r: Request) -> bool:
        """The lane a request is admitted to: solo for large denoise jobs, and
        for any request while fewer than light_solo jobs are in the solo lane."""
        return self.is_solo(r) or len(self.solo) < self.light_solo

    def admit(self, r: Request, now: float) -> bool:
        need = footprint(r.kind, r.side)
        if len(self.active) + len(self.solo) >= self.max_slots or self.in_use + need > self.budget:
            return False
        solo = self.takes_solo(r)
        if solo and len(self.solo) >= len(self.solo_streams):
            return False
        torch = self.torch
        host_u, host_aux = self.pool.get(r.kind, r.side)
        st = self.solo_streams[self.solo_issued % len(self.solo_streams)] if solo else self.stream
        with torch.cuda.stream(st):
            u = torch.empty(host_u.shape, dtype=host_u.dtype, device=self.device)
            aux = torch.empty(host_aux.shape, dtype=host_aux.dtype, device=self.device)
            u.copy_(host_u, non_blocking=True)
            aux.copy_(host_aux, non_blocking=True)
            stencil = slr.SLR_RESTORE8 if r.kind == KIND_DENOISE else slr.SLR_J2D5
            if solo:
                # the whole loop in one launch, after the lane's previous job
                r.solver = slr.Solver(stencil, u, aux, stream=st, tol=self.tol[r.kind])
                if self.solo_tail is not None:
                    st.wait_event(self.solo_tail)
                r.solver.run(self.cap)
                r.event = torch.cuda.Event()
                r.event.record(st)
                self.solo_tail = r.event
                self.solo_issued += 1
                self.solo[r.rid] = r
            else:
                r.slot = self.batch.add(stencil, u, aux, self.cap, tol=self.tol[r.kind])
                self.active[r.slot] = r
        r.tensors = (u, aux)
        r.lane = "solo" if solo else "batch"
        r.admitted = now
        self.in_use += need
        return True

    def _finish(self, r: Request, now: float, res, keep: bool) -> Request:
        r.finished, r.iters, r.converged, r.value = now, res.iters, res.converged, res.value
        self.in_use -= footprint(r.kind, r.side)
        if not keep:
            r.tensors = ()
        return r

    def retire(self, slot: int, now: float, keep: bool) -> Request:
        r = self.active.pop(slot)
        res = self.batch.result(slot)
        self.batch.remove(slot)
        return self._finish(r, now, res, keep)

    def step(self) -> list[int]:
        """Enqueue step_sweeps more sweeps of every request in the batch, wait
        for them and return the finished batch slots; with only solo jobs in
        flight, wait for the oldest of them instead."""
        if self.active:
            self.batch.run(self.step_sweeps)
            finished, _ = self.batch.poll()
            return finished
        if self.solo:
            next(iter(self.solo.values())).event.synchronize()
        return []

    def retire_solo(self, now: float, keep: bool) -> list[Request]:
        """The solo jobs whose launch has finished, in admission order (the
        lane runs them in that order); each result is read on the job's own
        stream, which holds nothing after it."""
        out = []
        for rid in list(self.solo):
            r = self.solo[rid]
            if not r.event.query():
                break
            res = r.solver.result(check=False)
            if res.status < 0:
                raise slr.SlrError(res.status, "solo solve failed")
            del self.solo[rid]
            r.solver.close()
            r.solver = None
            r.event = None
            out.append(self._finish(r, now, res, keep))
        return out

    def serve(self, requests: list[Request], *, warmup_s: float = 0.0, keep_results: bool = False,
              time_limit_s: float | None = None) -> ServeStats:
        """Serve `requests` in real time (arrival offsets from now).  Latency
        is arrival -> the poll that sees the request's loop stopped."""
        for r in requests:
            self.pool.get(r.kind, r.side)          # inputs ready before the clock starts
        pending = sorted(requests, key=lambda r: r.arrival)
        done: list[Request] = []
        qi = 0
        queue: list[Request] = []
        steps = max_in_flight = max_queue = 0
        t0 = time.perf_counter()
        while qi < len(pending) or queue or self.active or self.solo:
            now = time.perf_counter() - t0
            if time_limit_s is not None and now > time_limit_s:
                break
            while qi < len(pending) and pending[qi].arrival <= now:
                queue.append(pending[qi])
                qi += 1
            while queue and self.admit(queue[0], now):
                queue.pop(0)
            max_queue = max(max_queue, len(queue))
            max_in_flight = max(max_in_flight, len(self.active) + len(self.solo))
            if not self.active and not self.solo:
                if qi < len(pending):
                    time.sleep(max(0.0, min(pending[qi].arrival - now, 0.001)))
                continue
            finished = self.step()
            steps += 1
            now = time.perf_counter() - t0
            for s in finished:
                done.append(self.retire(s, now, keep_results))
            done.extend(self.retire_solo(now, keep_results))
        wall = time.perf_counter() - t0
        self.done = done
        measured = [r for r in done if r.arrival >= warmup_s]
        # no request finished after the warm-up: no latency sample (NaN), not 0
        lat = np.array([(r.finished - r.arrival) * 1e3 for r in measured]) if measured else np.full(1, np.nan)
        cells = float(sum(r.side * r.side * r.iters for r in done))
        span = max(wall - warmup_s, 1e-9)
        return ServeStats(
            requests=len(requests), completed=len(done), wall_s=wall,
            p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()),
            throughput_rps=len(measured) / span, cell_updates=cells, gcell_per_s=cells / wall / 1e9,
            steps=steps, max_in_flight=max_in_flight, max_queue=max_queue, budget_bytes=self.budget,
            measured=len(measured))

    def close(self):
        for r in self.solo.values():
            r.solver.close()
        self.solo = {}
        self.batch.close()


def serve_fifo(requests: list[Request], *, loop: int, warmup_s: float = 0.0, time_limit_s: float | None = None,
               denoise_tol: float = 1e-3, solve_tol: float = 1e-6, cap: int = 5000, device=None,
               pool: InputPool | None = None) -> ServeStats:
    """The same request stream served by a queue alone, the comparator of the
    continuous-batching Server: one request at a time in arrival order, each
    copied in and solved on its own from start to finish, with no batching and
    no overlap.  loop=SLR_LOOP_HOST solves every request by the plain schema of
    Fig. 2 (per sweep one sweep launch, one reduce launch and the test on the
    host); SLR_LOOP_PERSISTENT by one device-looped launch.  Latency is arrival
    -> the read of the request's result.  Requests not started by time_limit_s
    are left unserved (completed counts the served ones)."""
    import torch
    dev = torch.device(device or "cuda")
    stream = torch.cuda.Stream(dev)
    pool = pool if pool is not None else InputPool()
    for r in requests:
        pool.get(r.kind, r.side)                  # inputs ready before the clock starts
    tol = {KIND_DENOISE: denoise_tol, KIND_SOLVE: solve_tol}
    pending = sorted(requests, key=lambda r: r.arrival)
    arrivals = np.array([r.arrival for r in pending])
    done: list[Request] = []
    max_queue = 0
    t0 = time.perf_counter()
    for i, r in enumerate(pending):
        now = time.perf_counter() - t0
        if time_limit_s is not None and now > time_limit_s:
            break
        if r.arrival > now:
            time.sleep(r.arrival - now)
            now = time.perf_counter() - t0
        max_queue = max(max_queue, int(np.searchsorted(arrivals, now, side="right")) - i)
        host_u, host_aux = pool.get(r.kind, r.side)
        with torch.cuda.stream(stream):
            u = torch.empty(host_u.shape, dtype=host_u.dtype, device=dev)
            aux = torch.empty(host_aux.shape, dtype=host_aux.dtype, device=dev)
            u.copy_(host_u, non_blocking=True)
            aux.copy_(host_aux, non_blocking=True)
            stencil = slr.SLR_RESTORE8 if r.kind == KIND_DENOISE else slr.SLR_J2D5
            solver = slr.Solver(stencil, u, aux, stream=stream, tol=tol[r.kind], loop=loop)
            solver.run(cap)
            res = solver.result(check=False)           # waits for the stream
            solver.close()
        if res.status < 0:
            raise slr.SlrError(res.status, "solve failed")
        r.admitted, r.finished = now, time.perf_counter() - t0
        r.iters, r.converged, r.value = res.iters, res.converged, res.value
        done.append(r)
    wall = time.perf_counter() - t0
    measured = [r for r in done if r.arrival >= warmup_s]
    # a queue that fell behind may serve nothing that arrived after the
    # warm-up: its latencies are then NaN (no sample), not 0
    lat = np.array([(r.finished - r.arrival) * 1e3 for r in measured]) if measured else np.full(1, np.nan)
    cells = float(sum(r.side * r.side * r.iters for r in done))
    span = max(wall - warmup_s, 1e-9)
    return ServeStats(
        requests=len(requests), completed=len(done), wall_s=wall,
        p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()),
        throughput_rps=len(measured) / span, cell_updates=cells, gcell_per_s=cells / wall / 1e9,
        steps=len(done), max_in_flight=1 if done else 0, max_queue=max_queue, budget_bytes=0,
        measured=len(measured))
