"""The video restoration stream pipe(read, detect, ofarm(restore), write) of
Sec. 4.3: frames come out in input order whatever their iteration counts,
every frame equals the same frame restored alone, and a frame equals the
oracle's detection, restoration and rounding."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def alone(gpu, frame):
    img = torch.from_numpy(frame).cuda()
    u = torch.empty(img.shape, dtype=torch.float32, device="cuda")
    mask = gpu.detect_noise(img, state=u, wmax=7)
    s = gpu.Solver(gpu.SLR_RESTORE8, u, mask, tol=1e-3)
    s.run(5000)
    r = s.result()
    s.close()
    return gpu.state_to_frame(u).cpu().numpy(), r


@pytest.mark.parametrize("lanes", [1, 3])
def test_ordered_and_equal_to_each_frame_alone(gpu, lanes):
    from paper_1609_04567_gb300 import video
    frames, order = video.make_video(72, 136, 10, distinct=4, p_noise=0.5)
    # one frame with little noise: it finishes in fewer sweeps than the others
    frames[3] = video.make_video(72, 136, 1, distinct=1, seed=99, p_noise=0.05)[0][0]
    host_in = [torch.from_numpy(f).pin_memory() for f in frames]
    host_out = [torch.empty((72, 136), dtype=torch.uint8).pin_memory() for _ in frames]
    p = video.VideoPipeline(72, 136, lanes=lanes)
    stats = p.run(host_in, host_out)
    p.close()
    assert stats.frames == 10 and [r.index for r in stats.results] == list(range(10))
    iters = [r.iters for r in stats.results]
    assert iters[3] < min(iters[k] for k in range(10) if k != 3)
    for k, f in enumerate(frames):
        ref, r = alone(gpu, f)
        assert np.array_equal(host_out[k].numpy(), ref)
        assert (stats.results[k].iters, stats.results[k].value) == (r.iters, r.value)


def test_frame_equals_the_oracle_chain(gpu, orc):
    from paper_1609_04567_gb300 import video
    frames, _ = video.make_video(64, 96, 3, distinct=3)
    host_in = [torch.from_numpy(f).pin_memory() for f in frames]
    host_out = [torch.empty((64, 96), dtype=torch.uint8).pin_memory() for _ in frames]
    p = video.VideoPipeline(64, 96, lanes=2)
    p.run(host_in, host_out)
    p.close()
    for k in range(3):
        m = orc.amf_detect(frames[k], wmax=7)
        ref, _ = orc.restore8(frames[k].astype(np.float32), m, tol=1e-3, max_iters=5000)
        assert np.array_equal(host_out[k].numpy(), np.clip(np.rint(ref), 0, 255).astype(np.uint8))
