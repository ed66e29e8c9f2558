"""Pins for the oracle's restoration loop (Sec. 4.3 restoration phase).

The update reads the regularisation as minimising sum phi(u_i - u_j) over the
8 neighbours with phi(t) = sqrt(alpha + t^2) (alpha = 100); its Jacobi
fixed-point form weights each neighbour by w_j = phi'(t)/t = 1/sqrt(alpha+t^2).
Pins: a value worked out by hand, invariants (noise-free pixels untouched, a
constant image is a fixed point, a single noisy pixel heals to its
surroundings), transposition symmetry, the first-order optimality condition of
the functional at the returned state, and the mean-|change| reduce against a
brute-force sum.
"""
import math

import numpy as np
import pytest


def test_worked_example_two_level_neighbourhood(orc):
    # centre u = 0 (noisy), the four upper/left neighbours 0, the others 10.
    # w(0) = 1/sqrt(100) = 1/10, w(10) = 1/sqrt(200) = 1/(10 sqrt 2):
    # u' = 4*10/(10 sqrt2) / (4/10 + 4/(10 sqrt2)) = 10 / (1 + sqrt 2).
    u = np.array([[0, 0, 0], [0, 0, 10], [10, 10, 10]], dtype=np.float32)
    m = np.zeros((3, 3), dtype=np.uint8)
    m[1, 1] = 1
    out, r = orc.restore8(u, m, tol=0.0, max_iters=1)
    assert out[1, 1] == pytest.approx(10.0 / (1.0 + math.sqrt(2.0)), rel=2e-7)
    assert r.count == 1
    assert r.value == pytest.approx(10.0 / (1.0 + math.sqrt(2.0)), rel=1e-6)


def test_unmasked_pixels_bitwise_untouched(orc):
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(48, 40, seed=9)
    mask = inputs.noise_mask(frame)
    u0 = frame.astype(np.float32)
    out, r = orc.restore8(u0, mask, tol=1e-3, max_iters=200)
    keep = mask == 0
    assert np.array_equal(out[keep].view(np.uint32), u0[keep].view(np.uint32))
    assert r.count == int(mask.sum())


def test_constant_image_is_fixed_point(orc):
    u = np.full((9, 11), 77.0, dtype=np.float32)
    m = np.ones((9, 11), dtype=np.uint8)
    out, r = orc.restore8(u, m, tol=1e-3, max_iters=10)
    # a fixed point in exact arithmetic; in binary32 the weighted sum of eight
    # equal values may land one or two ulps away
    assert r.iters == 1 and r.converged and r.value < 2e-5
    assert np.max(np.abs(out - u)) <= 2 * np.spacing(np.float32(77.0))


@pytest.mark.parametrize("pos", [(4, 5), (0, 0), (0, 5), (8, 10)])
def test_single_noisy_pixel_heals_to_surroundings(orc, pos):
    # interior (8 neighbours), corner (3) and edge (5): out-of-range neighbours
    # are left out, so all equal neighbours give back the constant
    u = np.full((9, 11), 123.0, dtype=np.float32)
    u[pos] = 255.0
    m = np.zeros((9, 11), dtype=np.uint8)
    m[pos] = 1
    out, r = orc.restore8(u, m, tol=1e-3, max_iters=10)
    assert out[pos] == pytest.approx(123.0, abs=1e-4)
    assert r.converged and r.iters == 2


def test_transpose_symmetry(orc):
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(30, 30, seed=4)
    mask = inputs.noise_mask(frame)
    a, ra = orc.restore8(frame.astype(np.float32), mask, tol=0.0, max_iters=20)
    b, rb = orc.restore8(frame.T.astype(np.float32), mask.T.copy(), tol=0.0, max_iters=20)
    # the sums run in a different order after transposition: equal to rounding
    assert np.max(np.abs(a - b.T)) < 1e-3


def test_returned_state_is_stationary_point_of_functional(orc):
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(16, 16, seed=12)
    mask = inputs.noise_mask(frame)
    # binary32 rounding keeps single pixels moving by an ulp or so (~1e-5 at
    # values near 100), so the loop is run to a mean change of 2e-5
    out, r = orc.restore8(frame.astype(np.float32), mask, tol=2e-5, max_iters=20000)
    assert r.converged
    u = out.astype(np.float64)
    ny, nx = u.shape
    worst = 0.0
    # d/du_i of sum_j phi(u_i - u_j) = sum_j (u_i - u_j)/sqrt(100 + (u_i-u_j)^2),
    # evaluated by central differences of phi itself, not through the weights
    phi = lambda t: np.sqrt(100.0 + t * t)
    for i in range(ny):
        for j in range(nx):
            if not mask[i, j]:
                continue
            g = 0.0
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    y, x = i + di, j + dj
                    if (di or dj) and 0 <= y < ny and 0 <= x < nx:
                        t = u[i, j] - u[y, x]
                        g += (phi(t + 1e-4) - phi(t - 1e-4)) / 2e-4
            worst = max(worst, abs(g))
    # gradient = (u_i - u'_i) * sum_j w_j with sum_j w_j <= 0.8
    assert worst < 1e-3


@pytest.mark.parametrize("scale,before", [(1.0, 0), (1.0, 25), (1.0 / 512, 3)])
def test_mean_abs_change_reduce_matches_brute_force(orc, scale, before):
    # With pixel values of 20 .. 235 every binary32 change is a multiple of
    # 2^-17; a state scaled below 1/2 has changes with bits under 2^-24,
    # where truncating and rounding to 2^-24 differ.
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(64, 64, seed=21)
    mask = inputs.noise_mask(frame)
    u0 = (frame.astype(np.float64) * scale).astype(np.float32)
    if before:
        u0, _ = orc.restore8(u0, mask, tol=0.0, max_iters=before)
    out, r = orc.restore8(u0, mask, tol=0.0, max_iters=1)
    delta = np.abs(out.astype(np.float32) - u0.astype(np.float32)).astype(np.float64)[mask == 1]
    if scale < 1.0:
        assert np.mean(np.floor(delta * 2 ** 24) != delta * 2 ** 24) > 0.5
    # the reduce truncates each change to 2^-24 before the integer sum
    assert r.value == pytest.approx(delta.mean(), abs=2.0 ** -24)
    assert r.value == np.floor(delta * 2 ** 24).sum() / 2 ** 24 / delta.size


def test_empty_mask_stops_after_one_sweep(orc):
    u = np.arange(20, dtype=np.float32).reshape(4, 5)
    out, r = orc.restore8(u, np.zeros((4, 5), np.uint8), tol=1e-3, max_iters=9)
    assert r.iters == 1 and r.converged and r.value == 0.0 and r.count == 0
    assert np.array_equal(out, u)
