"""Parity of the CUDA restoration loop (Sec. 4.3 restoration phase) with the
oracle through the C ABI: bit-identical in EXACT math, within 1e-5 relative
(iterations within 1) in FAST math."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def restore_case(slr, orc, ny, nx, tol=1e-3, max_iters=5000, math=0, loop=None, seed=1, **extra):
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(ny, nx, seed=seed)
    mask = inputs.noise_mask(frame)
    u = torch.from_numpy(frame.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    fields = dict(tol=tol, math=math, **extra)
    if loop is not None:
        fields["loop"] = loop
    s = slr.Solver(slr.SLR_RESTORE8, u, m, **fields)
    s.run(max_iters)
    r = s.result()
    s.close()
    out = u.cpu().numpy()
    ref, rr = orc.restore8(frame.astype(np.float32), mask, tol=tol, max_iters=max_iters)
    return out, r, ref, rr


@pytest.mark.parametrize("ny,nx", [(256, 256), (300, 517), (1, 1), (2, 9), (37, 1),
                                   (48, 80), (33, 16), (1, 16), (100, 1040), (65, 208), (2, 64)])
def test_exact_matches_oracle(gpu, orc, ny, nx):
    out, r, ref, rr = restore_case(gpu, orc, ny, nx)
    assert r.iters == rr.iters and r.converged == rr.converged and r.count == rr.count
    assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))
    assert r.value == rr.value


def test_host_loop_matches_oracle(gpu, orc):
    out, r, ref, rr = restore_case(gpu, orc, 200, 300, loop=gpu.SLR_LOOP_HOST)
    assert r.iters == rr.iters and np.array_equal(out.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("ny,nx", [(512, 512), (300, 517)])
def test_fast_math_within_tolerance(gpu, orc, ny, nx):
    out, r, ref, rr = restore_case(gpu, orc, ny, nx, math=gpu.SLR_MATH_FAST)
    assert abs(r.iters - rr.iters) <= 1
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) <= 1e-5


# ---- temporal-blocked path (k sweeps per pass over 64 x 64 tiles with an
# 8-pixel halo); widths that are not a multiple of 16 run on padded copies of
# the mask, widths that are not a multiple of 4 on padded copies of the state
# too ----

@pytest.mark.parametrize("k", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("ny,nx", [(256, 256), (300, 528), (65, 208), (1, 16), (2, 64), (130, 144),
                                   (200, 1040), (64, 64), (9, 32),
                                   (40, 2760), (100, 136), (70, 130), (67, 131), (300, 517), (5, 3), (1, 1)])
def test_temporal_blocked_matches_oracle(gpu, orc, ny, nx, k):
    out, r, ref, rr = restore_case(gpu, orc, ny, nx, temporal_k=k)
    assert (r.iters, r.converged, r.count, r.value) == (rr.iters, rr.converged, rr.count, rr.value)
    assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("k", [2, 4, 8])
@pytest.mark.parametrize("cap", [1, 3, 5, 9])
@pytest.mark.parametrize("nx", [272, 270])
def test_temporal_blocked_cap_inside_a_pass_then_resume(gpu, orc, k, cap, nx):
    # a cap that ends inside a pass runs only the sweeps left; a later run
    # with a higher cap resumes from the state in u and equals a straight run
    # (270: the state goes through padded copies, in and out, on each run)
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(150, nx, seed=4)
    mask = inputs.noise_mask(frame)
    u = torch.from_numpy(frame.astype(np.float32)).cuda()
    s = gpu.Solver(gpu.SLR_RESTORE8, u, torch.from_numpy(mask).cuda(), tol=1e-3, temporal_k=k)
    s.run(cap)
    r1 = s.result(check=False)
    mid = u.cpu().numpy()
    ref1, rr1 = orc.restore8(frame.astype(np.float32), mask, tol=1e-3, max_iters=cap)
    assert (r1.iters, r1.converged, r1.value) == (rr1.iters, rr1.converged, rr1.value)
    assert np.array_equal(mid.view(np.uint32), ref1.view(np.uint32))
    s.run(5000)
    r2 = s.result()
    s.close()
    ref2, rr2 = orc.restore8(frame.astype(np.float32), mask, tol=1e-3, max_iters=5000)
    assert (r2.iters, r2.converged, r2.value, r2.count) == (rr2.iters, rr2.converged, rr2.value, rr2.count)
    assert np.array_equal(u.cpu().numpy().view(np.uint32), ref2.view(np.uint32))


@pytest.mark.parametrize("tol", [1e-1, 1e-2, 3e-3])
def test_temporal_blocked_stops_at_the_first_sweep_below_tol(gpu, orc, tol):
    # coarse tolerances stop inside the first or second 8-sweep pass
    out, r, ref, rr = restore_case(gpu, orc, 192, 320, tol=tol, temporal_k=8, seed=7)
    assert rr.converged and (r.iters, r.value) == (rr.iters, rr.value)
    assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))


def test_temporal_blocked_all_noisy_and_no_noisy_pixels(gpu, orc):
    # every pixel noisy (the list holds the whole tile), and none (the mean is 0: one sweep)
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(96, 160, seed=2)
    for mask in (np.ones_like(frame), np.zeros_like(frame)):
        u = torch.from_numpy(frame.astype(np.float32)).cuda()
        s = gpu.Solver(gpu.SLR_RESTORE8, u, torch.from_numpy(mask).cuda(), tol=1e-3, temporal_k=4)
        s.run(300)
        r = s.result(check=False)
        s.close()
        ref, rr = orc.restore8(frame.astype(np.float32), mask, tol=1e-3, max_iters=300)
        assert (r.iters, r.converged, r.value, r.count) == (rr.iters, rr.converged, rr.value, rr.count)
        assert np.array_equal(u.cpu().numpy().view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("k", [2, 8])
def test_temporal_blocked_fast_math_within_tolerance(gpu, orc, k):
    out, r, ref, rr = restore_case(gpu, orc, 300, 528, math=gpu.SLR_MATH_FAST, temporal_k=k)
    assert abs(r.iters - rr.iters) <= 1
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) <= 1e-5


@pytest.mark.slow
def test_full_size_4096_sample(gpu, orc):
    # the restoration configuration (4096 x 4096, 50% salt-and-pepper) in the
    # benchmark's launch configuration, for the sweeps the oracle runs in seconds
    out, r, ref, rr = restore_case(gpu, orc, 4096, 4096, tol=0.0, max_iters=3)
    assert r.iters == rr.iters == 3
    assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))
    assert r.value == rr.value


def test_exact_weight_arithmetic_matches_ieee_for_every_input(gpu):
    # the EXACT sweeps' 1/sqrt with two roundings against __frcp_rn(__fsqrt_rn(x)),
    # all 2^31 non-negative binary32 inputs, on the device
    mismatches, checked = gpu.slr_check_exact_math()
    assert checked == 1 << 31
    assert mismatches == [0, 0, 0]


@pytest.mark.parametrize("scale,alpha", [(2.0 ** 55, 100.0), (1.0, 1e-35), (2.0 ** -70, 1e-30)])
def test_temporal_blocked_outside_the_unchecked_range(gpu, orc, scale, alpha):
    # states above 2^60 in magnitude (some tiles take the weights' checked
    # route), an alpha below 2^-100 (every tile does), tiny states: still bit
    # for bit the oracle
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(150, 208, seed=12)
    mask = inputs.noise_mask(frame)
    u0 = (frame.astype(np.float64) * scale).astype(np.float32)
    u = torch.from_numpy(u0).cuda()
    s = gpu.Solver(gpu.SLR_RESTORE8, u, torch.from_numpy(mask).cuda(), tol=0.0, alpha=alpha, temporal_k=8)
    s.run(12)
    r = s.result(check=False)
    s.close()
    ref, rr = orc.restore8(u0, mask, alpha=alpha, tol=0.0, max_iters=12)
    assert (r.iters, r.value, r.count) == (rr.iters, rr.value, rr.count)
    assert np.array_equal(u.cpu().numpy().view(np.uint32), ref.view(np.uint32))
