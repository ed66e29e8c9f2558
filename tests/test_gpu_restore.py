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
