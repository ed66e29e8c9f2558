"""Parity of the CUDA Sobel edge detector (Sec. 4.2: one stencil sweep, no
reduce) with the oracle through the C ABI: integer work, bit-identical
output; and the image stream pipe(read, sobel, write) writes every image in
input order, equal to the image filtered alone."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def sobel(gpu, img):
    return gpu.sobel(torch.from_numpy(np.ascontiguousarray(img)).cuda()).cpu().numpy()


@pytest.mark.parametrize("ny,nx", [(1, 1), (2, 2), (3, 3), (1, 40), (40, 1), (3, 17), (17, 3), (5, 512),
                                   (33, 528), (64, 700), (300, 1037), (129, 1024), (7, 8192)])
def test_random_images_match_oracle(gpu, orc, ny, nx):
    from paper_1609_04567_gb300 import inputs
    img = inputs.random_image(ny, nx, seed=ny * 1000 + nx)
    assert np.array_equal(sobel(gpu, img), orc.sobel(img))


@pytest.mark.parametrize("ny,nx", [(512, 512), (480, 640), (257, 1000)])
def test_smooth_and_noisy_images(gpu, orc, ny, nx):
    from paper_1609_04567_gb300 import inputs
    for img in (inputs.smooth_image(ny, nx, seed=3), inputs.noisy_frame(ny, nx, seed=4)[0]):
        assert np.array_equal(sobel(gpu, img), orc.sobel(img))


def test_structured_images(gpu, orc):
    y, x = np.mgrid[0:40, 0:90]
    for img in ((3 * x + 4 * y).astype(np.uint8), np.where(x < 45, 10, 200).astype(np.uint8),
                np.full((40, 90), 255, dtype=np.uint8)):
        assert np.array_equal(sobel(gpu, img), orc.sobel(img))


def test_unaligned_rows_and_pointers(gpu, orc):
    # a row pitch of 16-byte groups read at a one-byte offset takes the byte path
    from paper_1609_04567_gb300 import inputs
    img = inputs.random_image(50, 256, seed=9)
    buf = torch.zeros(50 * 256 + 16, dtype=torch.uint8, device="cuda")
    buf[1:1 + 50 * 256] = torch.from_numpy(img.reshape(-1)).cuda()
    out = torch.zeros(50 * 256 + 16, dtype=torch.uint8, device="cuda")
    gpu.slr_sobel(buf.data_ptr() + 1, out.data_ptr() + 3, 256, 50)
    assert np.array_equal(out[3:3 + 50 * 256].cpu().numpy().reshape(50, 256), orc.sobel(img))


def test_image_stream_in_order(gpu):
    from paper_1609_04567_gb300 import inputs, video
    imgs = [inputs.random_image(96, 160, seed=s) for s in range(7)]
    host_in = [torch.from_numpy(a).pin_memory() for a in imgs]
    host_out = [torch.empty((96, 160), dtype=torch.uint8).pin_memory() for _ in imgs]
    st = video.sobel_stream(host_in, host_out, lanes=3)
    assert st.images == 7
    for a, o in zip(imgs, host_out):
        assert np.array_equal(o.numpy(), sobel(gpu, a))


def test_integer_square_root_is_exact(gpu):
    # every value Gx^2 + Gy^2 can take
    mismatches, checked = gpu.slr_check_exact_isqrt()
    assert (mismatches, checked) == (0, 1 << 22)


def test_large_random_image(gpu, orc):
    # millions of gradient pairs across the whole magnitude range
    from paper_1609_04567_gb300 import inputs
    img = inputs.random_image(2048, 2048, seed=21)
    assert np.array_equal(sobel(gpu, img), orc.sobel(img))


def test_rejects_bad_arguments(gpu):
    img = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(gpu.SlrError, match="overlap"):
        gpu.slr_sobel(img.data_ptr(), img.data_ptr() + 5, 16, 16)
    with pytest.raises(gpu.SlrError, match="device pointers"):
        gpu.slr_sobel(img.data_ptr(), 0, 16, 16)


@pytest.mark.slow
def test_full_size_16384(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    img = inputs.smooth_image(4096, 4096, seed=2)
    big = np.tile(img, (4, 4))
    assert np.array_equal(sobel(gpu, big), orc.sobel(big))
