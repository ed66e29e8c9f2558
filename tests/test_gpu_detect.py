"""Parity of the CUDA adaptive median noise detector (the detection phase of
the Sec. 4.3 two-phase restoration) with the oracle through the C ABI: the
mask is integer work and must be bit-identical; and the two phases composed
(detect, then restore with the detected mask) against the oracle's
composition."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def detect(slr, img, wmax):
    return slr.detect_noise(torch.from_numpy(np.ascontiguousarray(img)).cuda(), wmax=wmax).cpu().numpy()


@pytest.mark.parametrize("ny,nx", [(1, 1), (1, 7), (9, 1), (37, 53), (96, 128), (257, 129), (8, 32), (9, 33)])
@pytest.mark.parametrize("wmax", [3, 7, 15])
def test_matches_oracle(gpu, orc, ny, nx, wmax):
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(ny, nx, seed=11)
    assert np.array_equal(detect(gpu, frame, wmax), orc.amf_detect(frame, wmax=wmax))


@pytest.mark.parametrize("p", [0.1, 0.3, 0.8, 0.95])
@pytest.mark.parametrize("wmax", [5, 9, 11, 13])
def test_noise_levels(gpu, orc, p, wmax):
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(120, 200, seed=5, p_noise=p)
    assert np.array_equal(detect(gpu, frame, wmax), orc.amf_detect(frame, wmax=wmax))


def test_structured_images(gpu, orc):
    img = np.array([[10, 20, 30], [40, 250, 60], [70, 80, 90]], dtype=np.uint8)
    assert detect(gpu, img, 3).tolist() == [[1, 0, 0], [0, 1, 0], [0, 0, 0]]
    ramp = np.tile(np.arange(40, 100, dtype=np.uint8), (40, 1))
    ramp[5, 6], ramp[17, 33] = 255, 0
    assert np.array_equal(detect(gpu, ramp, 5), orc.amf_detect(ramp, wmax=5))
    assert not detect(gpu, np.full((33, 47), 255, dtype=np.uint8), 7).any()


@pytest.mark.parametrize("ny,nx", [(480, 640), (720, 1280)])
def test_video_frame_sizes(gpu, orc, ny, nx):
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(ny, nx, seed=3)
    assert np.array_equal(detect(gpu, frame, 7), orc.amf_detect(frame, wmax=7))


def test_two_phases_composed(gpu, orc):
    # detect on the GPU, restore on the GPU with that mask: equal to the oracle's
    # detection followed by the oracle's restoration (EXACT math)
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(150, 230, seed=8)
    img = torch.from_numpy(frame).cuda()
    u = torch.empty(img.shape, dtype=torch.float32, device="cuda")
    mask = gpu.detect_noise(img, state=u, wmax=7)
    s = gpu.Solver(gpu.SLR_RESTORE8, u, mask, tol=1e-3)
    s.run(5000)
    r = s.result()
    s.close()
    m_ref = orc.amf_detect(frame, wmax=7)
    ref, rr = orc.restore8(frame.astype(np.float32), m_ref, tol=1e-3, max_iters=5000)
    assert np.array_equal(mask.cpu().numpy(), m_ref)
    assert (r.iters, r.converged, r.value) == (rr.iters, rr.converged, rr.value)
    assert np.array_equal(u.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    # the write stage: nearest integer, ties to even, clamped
    assert np.array_equal(gpu.state_to_frame(u).cpu().numpy(), np.clip(np.rint(ref), 0, 255).astype(np.uint8))


def test_state_to_frame_rounding(gpu):
    v = np.array([-3.0, -0.5, 0.49, 0.5, 1.5, 2.5, 127.5, 254.5, 254.51, 255.4, 300.0, np.inf, -np.inf],
                 dtype=np.float32)
    out = gpu.state_to_frame(torch.from_numpy(v).cuda()).cpu().numpy()
    assert out.tolist() == [0, 0, 0, 0, 2, 2, 128, 254, 255, 255, 255, 255, 0]


def test_rejects_bad_arguments(gpu):
    img = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(img)
    for w in (1, 2, 4, 17):
        with pytest.raises(gpu.SlrError, match="wmax"):
            gpu.slr_detect_noise(img.data_ptr(), out.data_ptr(), 0, 16, 16, w)
    with pytest.raises(gpu.SlrError, match="overlap"):
        gpu.slr_detect_noise(img.data_ptr(), img.data_ptr() + 8, 0, 16, 16, 7)
    with pytest.raises(gpu.SlrError, match="device pointers"):
        gpu.slr_detect_noise(0, out.data_ptr(), 0, 16, 16, 7)
