"""Host logic of the serving loop, no GPU: the Poisson request stream, the
size buckets, device-memory footprints and which requests take the solo lane."""
import math

import numpy as np
import pytest


def test_bucket_sides_are_log_spaced_multiples_of_8():
    from paper_1609_04567_gb300 import serve
    sides = serve.bucket_sides(256, 4096, 8)
    assert sides[0] == 256 and sides[-1] == 4096 and len(sides) == 8
    assert all(s % 8 == 0 for s in sides)
    ratios = [b / a for a, b in zip(sides, sides[1:])]
    assert max(ratios) / min(ratios) < 1.05           # equal steps in log size


def test_request_stream_is_poisson_and_reproducible():
    from paper_1609_04567_gb300 import serve
    a = serve.make_requests(20.0, 500.0, seed=7)
    b = serve.make_requests(20.0, 500.0, seed=7)
    assert [(r.kind, r.side, r.arrival) for r in a] == [(r.kind, r.side, r.arrival) for r in b]
    n = len(a)
    assert abs(n - 10000) < 4 * math.sqrt(10000)       # Poisson count within 4 sigma
    gaps = np.diff([r.arrival for r in a])
    assert np.all(gaps >= 0) and abs(gaps.mean() - 1 / 500.0) < 0.05 / 500.0
    # exponential gaps: coefficient of variation 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05
    share = sum(r.kind == serve.KIND_DENOISE for r in a) / n
    assert abs(share - 0.5) < 0.02
    dsides = set(serve.bucket_sides(256, 4096, 8))
    ssides = set(serve.bucket_sides(64, 2048, 8))
    assert {r.side for r in a if r.kind == serve.KIND_DENOISE} == dsides
    assert {r.side for r in a if r.kind == serve.KIND_SOLVE} == ssides


def test_footprints_count_state_aux_and_scratch():
    from paper_1609_04567_gb300 import serve
    assert serve.footprint(serve.KIND_DENOISE, 100) == 100 * 100 * 9       # f32 state, u8 mask, f32 scratch
    assert serve.footprint(serve.KIND_SOLVE, 100) == 100 * 100 * 24        # f64 state, f, scratch


@pytest.mark.parametrize("solo_cells", [None, 1024 * 1024, 1])
def test_solo_lane_rule(solo_cells):
    from paper_1609_04567_gb300 import serve
    srv = object.__new__(serve.Server)                  # the rule needs no GPU state
    srv.solo_cells = solo_cells
    big = serve.Request(0, serve.KIND_DENOISE, 2048, 0.0)
    small = serve.Request(1, serve.KIND_DENOISE, 512, 0.0)
    solve = serve.Request(2, serve.KIND_SOLVE, 2048, 0.0)
    assert srv.is_solo(big) == (solo_cells is not None)
    assert srv.is_solo(small) == (solo_cells == 1)
    assert not srv.is_solo(solve)                       # solves stay in the batch


@pytest.mark.parametrize("light_solo,in_lane,expect", [(0, 0, False), (4, 0, True), (4, 3, True), (4, 4, False),
                                                       (1, 1, False)])
def test_light_load_routing(light_solo, in_lane, expect):
    # any request takes the solo lane while it holds fewer than light_solo
    # jobs; large denoise jobs take it whatever the lane holds
    from paper_1609_04567_gb300 import serve
    srv = object.__new__(serve.Server)                  # the rule needs no GPU state
    srv.solo_cells, srv.light_solo = 1024 * 1024, light_solo
    srv.solo = {i: None for i in range(in_lane)}
    small = serve.Request(1, serve.KIND_SOLVE, 64, 0.0)
    big = serve.Request(2, serve.KIND_DENOISE, 2048, 0.0)
    assert srv.takes_solo(small) == expect
    assert srv.takes_solo(big)


def test_video_streams_are_seeded_permutations():
    # every round of a stream deals each distinct frame once; the same seed
    # gives the same stream
    from paper_1609_04567_gb300 import video
    frames, order = video.make_video(24, 40, 10, distinct=4)
    frames2, order2 = video.make_video(24, 40, 10, distinct=4)
    assert order == order2 and all((a == b).all() for a, b in zip(frames, frames2))
    assert sorted(order[:4]) == [0, 1, 2, 3] and sorted(order[4:8]) == [0, 1, 2, 3]
    assert len(frames) == 10 and frames[0].dtype.name == "uint8"
    for k, i in enumerate(order):
        assert (frames[k] == frames[order.index(i)]).all()


def test_random_images_are_seeded_and_uniform():
    import numpy as np
    from paper_1609_04567_gb300 import inputs
    a = inputs.random_image(64, 96, seed=3)
    assert (a == inputs.random_image(64, 96, seed=3)).all() and not (a == inputs.random_image(64, 96, seed=4)).all()
    counts = np.bincount(a.reshape(-1), minlength=256)
    assert counts.min() > 0 and abs(a.mean() - 127.5) < 3


class _FakeResult:
    status, iters, converged, value = 0, 7, True, 0.5


def _fake_device(monkeypatch, service_s):
    """Stand-ins for the CUDA stream, device tensors and the solver, so that
    the queue's host logic runs on the CPU; every solve takes service_s."""
    import contextlib
    import time as _time
    import torch
    from paper_1609_04567_gb300 import serve

    class FakeSolver:
        def __init__(self, stencil, u, aux, stream=None, **fields):
            assert {"tol", "loop"} <= set(fields)

        def run(self, n):
            _time.sleep(service_s)

        def result(self, check=True):
            return _FakeResult()

        def close(self):
            pass

    real_empty = torch.empty
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: type("S", (), {"cuda_stream": 0})())
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch, "empty", lambda shape, dtype=None, device=None: real_empty(shape, dtype=dtype))
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    monkeypatch.setattr(serve.slr, "Solver", FakeSolver)


def test_queue_alone_serves_in_arrival_order_and_keeps_up_when_it_can(monkeypatch):
    from paper_1609_04567_gb300 import serve
    _fake_device(monkeypatch, 0.001)
    reqs = serve.make_requests(0.3, 100.0, seed=5, denoise_sides=(32, 64), solve_sides=(16, 32), buckets=3)
    st = serve.serve_fifo(reqs, loop=serve.slr.SLR_LOOP_HOST, warmup_s=0.05, device="cpu")
    assert st.completed == len(reqs) and st.max_in_flight == 1 and st.measured > 0
    order = sorted(reqs, key=lambda r: r.arrival)
    for a, b in zip(order, order[1:]):
        assert a.finished <= b.admitted                   # one at a time, in arrival order
    assert all(r.admitted >= r.arrival and r.iters == 7 for r in reqs)
    assert 1.0 <= st.p50_ms < 50.0                       # about one service time


def test_queue_alone_that_falls_behind_reports_no_latency_sample(monkeypatch):
    import math
    from paper_1609_04567_gb300 import serve
    _fake_device(monkeypatch, 0.02)                     # 50 requests/s against 400/s offered
    reqs = serve.make_requests(0.5, 400.0, seed=6, denoise_sides=(32, 64), solve_sides=(16, 32), buckets=3)
    st = serve.serve_fifo(reqs, loop=serve.slr.SLR_LOOP_HOST, warmup_s=0.2, time_limit_s=0.1, device="cpu")
    assert 0 < st.completed < len(reqs) and st.max_queue > 1
    assert st.measured == 0 and math.isnan(st.p50_ms) and math.isnan(st.p99_ms)
