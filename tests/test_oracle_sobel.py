"""Pins of the oracle's Sobel edge detector (Sec. 4.2; Euclidean magnitude of
the two 3x3 gradients, floor, clamped to 255, border 0): a worked example,
closed forms on steps and ramps (including a Pythagorean ramp whose magnitude
is an exact integer).  CPU only."""
import numpy as np
import pytest

import oracle


def test_worked_example_3x3():
    # Gx = (3 - 1) + 2 (6 - 4) + (10 - 7) = 9, Gy = (7 - 1) + 2 (8 - 2) + (10 - 3) = 25,
    # sqrt(81 + 625) = 26.57...; the border is 0
    img = np.array([[1, 2, 3], [4, 5, 6], [7, 8, 10]], dtype=np.uint8)
    assert oracle.sobel(img).tolist() == [[0, 0, 0], [0, 26, 0], [0, 0, 0]]


@pytest.mark.parametrize("v", [0, 99, 255])
def test_constant_image_has_no_edges(v):
    assert not oracle.sobel(np.full((7, 9), v, dtype=np.uint8)).any()


@pytest.mark.parametrize("a,b,expect", [(10, 30, 80), (200, 180, 80), (0, 100, 255), (50, 51, 4)])
def test_vertical_step(a, b, expect):
    # a step between columns 5 and 6: |Gx| = 4 |b - a| in columns 5 and 6
    img = np.full((8, 12), a, dtype=np.uint8)
    img[:, 6:] = b
    out = oracle.sobel(img)
    want = np.zeros_like(out)
    want[1:-1, 5:7] = expect
    assert np.array_equal(out, want)


def test_horizontal_step():
    img = np.full((10, 7), 40, dtype=np.uint8)
    img[4:, :] = 70
    out = oracle.sobel(img)
    want = np.zeros_like(out)
    want[3:5, 1:-1] = 120
    assert np.array_equal(out, want)


@pytest.mark.parametrize("sx,sy,expect", [(1, 0, 8), (0, 2, 16), (1, 1, 11), (3, 4, 40), (5, 12, 104)])
def test_ramps(sx, sy, expect):
    # z = sx x + sy y: Gx = 8 sx, Gy = 8 sy inside; floor(sqrt(64 (sx^2 + sy^2)))
    y, x = np.mgrid[0:9, 0:11]
    img = (sx * x + sy * y).astype(np.uint8)
    out = oracle.sobel(img)
    assert (out[1:-1, 1:-1] == expect).all() and not out[0].any() and not out[:, 0].any()
    assert not out[-1].any() and not out[:, -1].any()


@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (2, 2), (3, 1)])
def test_images_without_interior(shape):
    assert not oracle.sobel(np.full(shape, 77, dtype=np.uint8)).any()
