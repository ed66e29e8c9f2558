"""Image streams of Sec. 4: the video restoration pipe(read, detect,
ofarm(restore), write) of Sec. 4.3 and the Sobel pipe(read, sobel, write) of
Sec. 4.2, on one GPU.

* read: the frames of a noisy video (uint8) sit in pinned host memory and are
  copied to the device on the frame's stream;
* detect: the adaptive median noise detector (``slr.detect_noise``), which
  also writes the frame as the restoration's binary32 state in the same pass;
* restore: the RESTORE8 loop (persistent device loop) until the mean |delta|
  over the noisy pixels drops below tol;
* write: the restored state rounded back to uint8 (``slr.state_to_frame``) and
  copied to pinned host memory.

ofarm: ``lanes`` frames are in flight, each on its own CUDA stream with its
own device buffers, and each lane's persistent launch takes its share of the
SMs, so the lanes' restorations run side by side.  Frames are dealt to the
lanes in turn and written in input order: before a lane takes frame f it
hands on frame f - lanes, the oldest frame in flight, so the output order is
the input order whatever the frames' iteration counts.  Every result equals
the frame restored alone.

``make_video`` builds the synthetic input: a few distinct noisy frames of the
restoration workload's generator, dealt into a stream by a seeded
permutation (the paper's streams are permutations of a small input set)."""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs, slr


def make_video(ny: int, nx: int, frames: int, *, distinct: int = 4, seed: int = inputs.DEFAULT_SEED,
               p_noise: float = 0.5):
    """(list of uint8 frames (numpy), list of their source indices): `distinct`
    noisy frames of the restoration generator, dealt into `frames` positions
    by a seeded shuffle of whole rounds."""
    base = [inputs.noisy_frame(ny, nx, seed=seed + k, p_noise=p_noise)[0] for k in range(distinct)]
    order = []
    rnd = 0
    while len(order) < frames:
        u = inputs.uniform01(seed + 1000 + rnd, inputs.STREAM_ARRIVALS + 7, distinct)
        order.extend(int(i) for i in np.argsort(u, kind="stable"))
        rnd += 1
    order = order[:frames]
    return [base[i] for i in order], order


@dataclass
class FrameResult:
    index: int
    iters: int
    converged: bool
    value: float
    issued: float
    done: float = 0.0


@dataclass
class VideoStats:
    frames: int
    lanes: int
    wall_s: float
    fps: float
    p50_ms: float
    p99_ms: float
    mean_iters: float
    gcell_per_s: float
    results: list = field(default_factory=list, repr=False)


class _Lane:
    def __init__(self, torch, device, ny, nx, desc, ws_bytes):
        self.stream = torch.cuda.Stream(device)
        self.img = torch.empty((ny, nx), dtype=torch.uint8, device=device)
        self.mask = torch.empty((ny, nx), dtype=torch.uint8, device=device)
        self.u = torch.empty((ny, nx), dtype=torch.float32, device=device)
        self.out = torch.empty((ny, nx), dtype=torch.uint8, device=device)
        self.ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=device)
        self.ws_ptr = self.ws.data_ptr() + ((-self.ws.data_ptr()) % 256)
        self.ws_bytes = ws_bytes
        self.desc = desc
        self.handle = None
        self.pending = None       # (FrameResult, event) of the frame in flight


@dataclass
class ImageStats:
    images: int
    lanes: int
    wall_s: float
    images_per_s: float
    gbytes_per_s: float          # image bytes in and out per second, end to end


def sobel_stream(images_host, out_host, *, lanes: int = 3, device=None) -> ImageStats:
    """pipe(read, sobel, write) of Sec. 4.2 over pinned uint8 host images of
    one shape: each image is copied in, filtered and copied out on the stream
    of its lane, `lanes` images in flight so copies overlap the filter;
    written in input order."""
    import torch
    dev = torch.device(device or "cuda")
    shape = tuple(images_host[0].shape)
    streams = [torch.cuda.Stream(dev) for _ in range(lanes)]
    bufs = [(torch.empty(shape, dtype=torch.uint8, device=dev), torch.empty(shape, dtype=torch.uint8, device=dev))
            for _ in range(lanes)]
    events = [None] * lanes
    n = len(images_host)
    t0 = time.perf_counter()
    for f in range(n):
        k = f % lanes
        if events[k] is not None:
            events[k].synchronize()            # image f - lanes written
        s, (din, dout) = streams[k], bufs[k]
        with torch.cuda.stream(s):
            din.copy_(images_host[f], non_blocking=True)
        slr.slr_sobel(din.data_ptr(), dout.data_ptr(), shape[1], shape[0], s.cuda_stream)
        with torch.cuda.stream(s):
            out_host[f].copy_(dout, non_blocking=True)
        events[k] = torch.cuda.Event()
        events[k].record(s)
    for f in range(n, n + lanes):
        if events[f % lanes] is not None:
            events[f % lanes].synchronize()
    wall = time.perf_counter() - t0
    return ImageStats(images=n, lanes=lanes, wall_s=wall, images_per_s=n / wall,
                      gbytes_per_s=2.0 * n * shape[0] * shape[1] / wall / 1e9)


class VideoPipeline:
    """pipe(read, detect, ofarm(restore), write) for frames of one size."""

    def __init__(self, ny: int, nx: int, *, lanes: int = 2, wmax: int = 7, tol: float = 1e-3, cap: int = 5000,
                 math: int = 0, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.ny, self.nx = ny, nx
        self.wmax, self.cap = wmax, cap
        sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        # each lane's persistent launch takes its share of the co-resident CTAs
        # (4 restoration CTAs fit an SM), so the lanes run side by side
        grid = 0 if lanes == 1 else max(1, 4 * sms // lanes)
        desc = slr.slr_desc_init(slr.SLR_RESTORE8, nx, ny, 1, storage=slr.SLR_F32, tol=tol, math=math,
                                 grid_ctas=grid)
        ws = slr.slr_workspace_size(desc)
        self.lanes = [_Lane(torch, self.device, ny, nx, desc, ws) for _ in range(lanes)]

    def _issue(self, lane: _Lane, f: int, frame_host, out_host, t0: float) -> None:
        torch = self.torch
        s = lane.stream
        with torch.cuda.stream(s):
            lane.img.copy_(frame_host, non_blocking=True)
        slr.slr_detect_noise(lane.img.data_ptr(), lane.mask.data_ptr(), lane.u.data_ptr(), self.nx, self.ny,
                             self.wmax, s.cuda_stream)
        lane.handle = slr.slr_create(lane.desc, lane.u.data_ptr(), lane.mask.data_ptr(), lane.ws_ptr,
                                     lane.ws_bytes, s.cuda_stream)
        slr.slr_run_until(lane.handle, self.cap)
        slr.slr_state_to_frame(lane.u.data_ptr(), lane.out.data_ptr(), self.nx * self.ny, s.cuda_stream)
        with torch.cuda.stream(s):
            out_host.copy_(lane.out, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(s)
        lane.pending = (FrameResult(f, 0, False, 0.0, time.perf_counter() - t0), ev)

    def _retire(self, lane: _Lane, t0: float) -> FrameResult:
        r, ev = lane.pending
        ev.synchronize()
        st, value, iters, conv, _ = slr.slr_reduce_value(lane.handle, check=False)
        if st < 0:
            raise slr.SlrError(st, slr.slr_last_error(lane.handle))
        slr.slr_destroy(lane.handle)
        lane.handle = None
        lane.pending = None
        r.iters, r.converged, r.value, r.done = iters, conv, value, time.perf_counter() - t0
        return r

    def run(self, frames_host, out_host) -> VideoStats:
        """Restore pinned uint8 host frames into pinned uint8 host outputs (same
        shapes), frames available from the start; returns the stream's stats
        with the per-frame results in input order."""
        n = len(frames_host)
        W = len(self.lanes)
        done = []
        t0 = time.perf_counter()
        for f in range(n):
            lane = self.lanes[f % W]
            if lane.pending is not None:           # frame f - W: the oldest in flight
                done.append(self._retire(lane, t0))
            self._issue(lane, f, frames_host[f], out_host[f], t0)
        for k in range(n, n + W):                  # the last frames, still in order
            lane = self.lanes[k % W]
            if lane.pending is not None:
                done.append(self._retire(lane, t0))
        wall = time.perf_counter() - t0
        assert [r.index for r in done] == list(range(n))
        lat = np.array([(r.done - r.issued) * 1e3 for r in done]) if done else np.zeros(1)
        iters = np.array([r.iters for r in done], dtype=np.float64) if done else np.zeros(1)
        return VideoStats(frames=n, lanes=W, wall_s=wall, fps=n / wall, p50_ms=float(np.percentile(lat, 50)),
                          p99_ms=float(np.percentile(lat, 99)), mean_iters=float(iters.mean()),
                          gcell_per_s=float(iters.sum()) * self.nx * self.ny / wall / 1e9, results=done)

    def close(self) -> None:
        for lane in self.lanes:
            if lane.pending is not None:
                lane.pending[1].synchronize()
            if lane.handle:
                slr.slr_destroy(lane.handle)
                lane.handle = None
