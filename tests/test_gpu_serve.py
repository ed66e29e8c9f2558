"""Continuous-batching serving loop: requests that arrive while others run are
admitted into the resident batch as memory and slots free up; every result
must equal the result of the same request solved alone."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def solve_alone(slr, r, server):
    host_u, host_aux = server.pool.get(r.kind, r.side)
    u = host_u.clone().cuda()
    aux = host_aux.clone().cuda()
    stencil = slr.SLR_RESTORE8 if r.kind == "denoise" else slr.SLR_J2D5
    s = slr.Solver(stencil, u, aux, tol=server.tol[r.kind])
    s.run(server.cap)
    res = s.result()
    s.close()
    return u, res


@pytest.mark.parametrize("solo_cells,light_solo,rate", [(None, 0, 300.0), (128 * 128, 0, 300.0), (None, 1, 3000.0)])
def test_results_alone_equal_results_in_the_mix(gpu, solo_cells, light_solo, rate):
    # solo_cells = 128^2: the denoise jobs of 128^2 pixels and more take the
    # solo lane; light_solo = 1: any request does while the lane is empty (at
    # 3000 requests/s the lane is busy often enough for the batch to get work)
    from paper_1609_04567_gb300 import serve
    reqs = serve.make_requests(0.4, rate, seed=3, denoise_sides=(32, 256), solve_sides=(16, 128), buckets=5)
    assert len(reqs) > 60
    srv = serve.Server(max_slots=64, step_sweeps=8, solo_cells=solo_cells, light_solo=light_solo)
    n_solo = sum(srv.is_solo(r) for r in reqs)
    assert (n_solo > 5) == (solo_cells is not None)
    stats = srv.serve(reqs, keep_results=True)
    assert stats.completed == len(reqs)
    assert stats.max_in_flight > 1                     # work really overlapped
    lanes = [r.lane for r in srv.done]
    if solo_cells is None and light_solo == 0:
        assert set(lanes) == {"batch"}
    else:
        assert lanes.count("solo") > 5 and lanes.count("batch") > 5
    done = {r.rid: r for r in srv.done}
    picks = list(done.values())[::37] + [r for r in done.values() if r.lane == "solo"][:6] + \
        [r for r in done.values() if r.lane == "batch"][:6]
    for r in picks:
        u_alone, res = solve_alone(gpu, r, srv)
        assert (r.iters, r.converged) == (res.iters, res.converged)
        assert torch.equal(r.tensors[0], u_alone)
        assert r.value == res.value
    srv.close()


def test_admission_respects_the_memory_budget(gpu):
    from paper_1609_04567_gb300 import serve
    reqs = serve.make_requests(0.2, 400.0, seed=4, denoise_sides=(64, 256), solve_sides=(32, 128), buckets=4)
    budget = 2 * serve.footprint("denoise", 256)
    srv = serve.Server(max_slots=32, step_sweeps=16, budget_bytes=budget)
    peak = 0
    orig = srv.admit

    def watched(r, now):
        nonlocal peak
        ok = orig(r, now)
        peak = max(peak, srv.in_use)
        return ok
    srv.admit = watched
    stats = srv.serve(reqs)
    assert stats.completed == len(reqs)
    assert 0 < peak <= budget
    assert stats.p99_ms >= stats.p50_ms > 0
    srv.close()


@pytest.mark.parametrize("loop", ["host", "persistent"])
def test_queue_alone_gives_each_request_its_solo_result(gpu, loop):
    # the plain comparator of the serving loop: one request at a time
    from types import SimpleNamespace
    from paper_1609_04567_gb300 import serve
    reqs = serve.make_requests(0.1, 300.0, seed=5, denoise_sides=(32, 256), solve_sides=(16, 128), buckets=5)
    assert len(reqs) > 10
    lp = gpu.SLR_LOOP_HOST if loop == "host" else gpu.SLR_LOOP_PERSISTENT
    st = serve.serve_fifo(reqs, loop=lp)
    assert st.completed == len(reqs) and st.max_in_flight == 1
    ref = SimpleNamespace(pool=serve.InputPool(), tol={"denoise": 1e-3, "solve": 1e-6}, cap=5000)
    for r in reqs:
        assert r.finished >= r.admitted >= r.arrival
        _, res = solve_alone(gpu, r, ref)
        assert (r.iters, r.converged, r.value) == (res.iters, res.converged, res.value), (r.kind, r.side)
