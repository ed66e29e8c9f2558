"""Pins of the oracle's adaptive median noise detector (the detection phase
of the Sec. 4.3 two-phase restoration; textbook adaptive median filter, lower
median, windows clipped to the image).  Worked examples computed by hand,
closed forms on structured images, and the detection of the generator's own
salt-and-pepper noise.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1609_04567_gb300 import inputs


def test_worked_example_3x3():
    # every window sorted by hand: the corner (0, 0) sees {10, 20, 40, 250}
    # (lower median 20: 10 is the window's minimum, replaced), the centre
    # sees all nine (median 60: 250 is the maximum, replaced); every other
    # pixel lies strictly between its window's extremes
    img = np.array([[10, 20, 30], [40, 250, 60], [70, 80, 90]], dtype=np.uint8)
    assert oracle.amf_detect(img, wmax=3).tolist() == [[1, 0, 0], [0, 1, 0], [0, 0, 0]]


@pytest.mark.parametrize("v", [0, 1, 37, 254, 255])
def test_constant_image_has_no_noise(v):
    img = np.full((9, 13), v, dtype=np.uint8)
    assert not oracle.amf_detect(img, wmax=7).any()


def test_ramp_flags_only_its_extreme_columns():
    # strictly increasing along x: an interior pixel is its window's median,
    # strictly between the extremes; the first and last columns are their
    # windows' minimum and maximum
    img = np.tile(np.arange(20, 84, dtype=np.uint8), (30, 1))
    m = oracle.amf_detect(img, wmax=7)
    expect = np.zeros_like(m)
    expect[:, 0] = expect[:, -1] = 1
    assert np.array_equal(m, expect)


def test_isolated_impulses_on_a_ramp():
    img = np.tile(np.arange(40, 100, dtype=np.uint8), (40, 1))
    expect = np.zeros(img.shape, dtype=np.uint8)
    expect[:, 0] = expect[:, -1] = 1
    for k, (i, j) in enumerate([(5, 6), (5, 20), (17, 33), (30, 12), (34, 50)]):
        img[i, j] = 255 if k % 2 == 0 else 0
        expect[i, j] = 1
    assert np.array_equal(oracle.amf_detect(img, wmax=5), expect)


def test_no_qualifying_window_outputs_the_median():
    # a 100 amid 255s: every window's median is its maximum, so the filter
    # outputs the median (255) and only the centre differs from it
    img = np.full((5, 5), 255, dtype=np.uint8)
    img[2, 2] = 100
    for w in (3, 5):
        m = oracle.amf_detect(img, wmax=w)
        assert m[2, 2] == 1 and m.sum() == 1


def test_window_grows_until_the_median_is_not_an_extreme():
    # the centre and five of its neighbours are 255: the 3 x 3 median is 255
    # (no decision, the filter outputs it: the centre is kept), the 5 x 5
    # median is a ramp value, so with wmax 5 the centre is replaced
    i, j = np.mgrid[0:7, 0:7]
    img = (20 + 7 * i + j).astype(np.uint8)
    for (a, b) in [(3, 3), (2, 2), (2, 3), (2, 4), (3, 2), (3, 4)]:
        img[a, b] = 255
    assert oracle.amf_detect(img, wmax=3)[3, 3] == 0
    assert oracle.amf_detect(img, wmax=5)[3, 3] == 1


@pytest.mark.parametrize("shape,p", [((96, 128), 0.5), ((257, 129), 0.3), ((120, 160), 0.5)])
def test_detects_the_generators_salt_and_pepper(shape, p):
    # the generator's noisy pixels (0 or 255 on a clean image in [20, 235])
    # are found; clean pixels flagged are the few that are their window's
    # minimum or maximum
    frame, clean = inputs.noisy_frame(*shape, seed=7, p_noise=p)
    truth = frame != clean
    m = oracle.amf_detect(frame, wmax=7).astype(bool)
    assert (m & truth).sum() >= 0.9995 * truth.sum()
    assert (m & ~truth).sum() <= 0.02 * (~truth).sum()


def test_rejects_even_or_small_windows():
    img = np.zeros((4, 4), dtype=np.uint8)
    for w in (1, 2, 4):
        with pytest.raises(ValueError):
            oracle.amf_detect(img, wmax=w)
