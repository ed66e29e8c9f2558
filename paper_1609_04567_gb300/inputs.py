"""Seeded synthetic inputs for the Loop-of-stencil-reduce workloads.

This module holds only random-number generation and input shaping; none of the
method's arithmetic.  Both the CUDA path's tests/benchmarks and the oracle's
tests take their inputs from here, so the two sides see identical bytes.

Randomness is the SplitMix64 generator (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) used in counter form:
item i of stream s under seed S is mix64(key(S, s) + (i + 1) * GAMMA), with
key(S, s) = mix64(S ^ ((s + 1) * 0xD1B54A32D192ED03)).  A uniform double in
[0, 1) is (x >> 11) * 2^-53; U[-1, 1] is 2u - 1 (exact).

Workload shapes (the paper's datasets are not available, so these stand in):
  * Helmholtz right-hand side f ~ U[-1, 1] (Sec. 4.1 solver), u0 = 0;
  * Game of Life cells alive with probability 0.3;
  * restoration frames (Sec. 4.3): a smooth image, the sum of 8 random 2D
    Gaussians min-max scaled to [20, 235] and rounded to uint8, with 50% of the
    pixels replaced by salt-and-pepper noise (0 or 255 on a fair coin), so the
    noisy-pixel mask is exactly value in {0, 255}.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20160915
GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_KEYMUL = 0xD1B54A32D192ED03
_MASK64 = (1 << 64) - 1

# named streams, so that different inputs under one seed are independent
STREAM_F = 1
STREAM_LIFE = 2
STREAM_IMAGE_PARAMS = 3
STREAM_NOISE = 4
STREAM_BATCH_SIDES = 5
STREAM_ARRIVALS = 6
STREAM_PIXELS = 7               # uniformly random uint8 images
STREAM_BATCH_F0 = 1000          # per-instance right-hand sides start here


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _mix64_int(z: int) -> int:
    z &= _MASK64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & _MASK64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & _MASK64
    z ^= z >> 31
    return z


def stream_key(seed: int, stream: int) -> int:
    return _mix64_int((seed ^ (((stream + 1) * _KEYMUL) & _MASK64)) & _MASK64)


def raw_u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Items start .. start+count-1 of a stream as uint64."""
    key = np.uint64(stream_key(seed, stream))
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + idx * GAMMA)


def uniform01(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    x = raw_u64(seed, stream, start, count)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _chunked(count: int, fn, dtype, chunk: int = 1 << 24) -> np.ndarray:
    out = np.empty(count, dtype=dtype)
    for s in range(0, count, chunk):
        n = min(chunk, count - s)
        out[s:s + n] = fn(s, n)
    return out


def helmholtz_rhs(shape, seed: int = DEFAULT_SEED, stream: int = STREAM_F) -> np.ndarray:
    """f ~ U[-1, 1] as float64, C order, of the given shape ((ny, nx) or (nz, ny, nx))."""
    count = int(np.prod(shape))
    f = _chunked(count, lambda s, n: 2.0 * uniform01(seed, stream, n, s) - 1.0, np.float64)
    return f.reshape(shape)


def life_cells(ny: int, nx: int, seed: int = DEFAULT_SEED, p_alive: float = 0.3) -> np.ndarray:
    """uint8 cells in {0, 1}, alive with probability p_alive."""
    count = ny * nx
    cells = _chunked(count, lambda s, n: (uniform01(seed, STREAM_LIFE, n, s) < p_alive)
                     .astype(np.uint8), np.uint8)
    return cells.reshape(ny, nx)


def smooth_image(ny: int, nx: int, seed: int = DEFAULT_SEED, n_gauss: int = 8) -> np.ndarray:
    """uint8 image in [20, 235]: sum of n_gauss random Gaussians (centre
    U[0,N)^2, width U[N/16, N/4], amplitude U[-1,1]), min-max scaled, rounded."""
    p = uniform01(seed, STREAM_IMAGE_PARAMS, 5 * n_gauss).reshape(n_gauss, 5)
    n = float(max(nx, ny))
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    img = np.zeros((ny, nx), dtype=np.float64)
    for g in range(n_gauss):
        cx, cy = p[g, 0] * nx, p[g, 1] * ny
        sg = n / 16.0 + p[g, 2] * (n / 4.0 - n / 16.0)
        amp = 2.0 * p[g, 3] - 1.0
        gx = np.exp(-((x - cx) ** 2) / (2.0 * sg * sg))
        gy = np.exp(-((y - cy) ** 2) / (2.0 * sg * sg))
        img += amp * (gy * gx)
    lo, hi = float(img.min()), float(img.max())
    scale = 215.0 / (hi - lo) if hi > lo else 0.0
    out = np.rint(20.0 + (img - lo) * scale)
    return np.clip(out, 20, 235).astype(np.uint8)


def noisy_frame(ny: int, nx: int, seed: int = DEFAULT_SEED, p_noise: float = 0.5):
    """A restoration input: returns (noisy uint8 frame, clean uint8 image).

    Each pixel is noisy with probability p_noise; a noisy pixel is 0 or 255 on
    a fair coin (bit 0 of its random word)."""
    clean = smooth_image(ny, nx, seed)
    r = raw_u64(seed, STREAM_NOISE, 0, ny * nx).reshape(ny, nx)
    u = (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    noisy = u < p_noise
    salt = (r & np.uint64(1)).astype(bool)
    frame = clean.copy()
    frame[noisy & salt] = 255
    frame[noisy & ~salt] = 0
    return frame, clean


def random_image(ny: int, nx: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """uint8 image with every pixel uniform in [0, 255] (the low byte of its
    random word)."""
    return (raw_u64(seed, STREAM_PIXELS, 0, ny * nx) & np.uint64(0xFF)).astype(np.uint8).reshape(ny, nx)


def noise_mask(frame: np.ndarray) -> np.ndarray:
    """The detection rule that stands in for the adaptive median filter: a pixel
    is noisy when its value is 0 or 255."""
    return ((frame == 0) | (frame == 255)).astype(np.uint8)


def batch_sides(count: int, lo: int = 64, hi: int = 1024, seed: int = DEFAULT_SEED,
                stream: int = STREAM_BATCH_SIDES) -> np.ndarray:
    """Grid sides log-uniform in [lo, hi]: round(exp(U[ln lo, ln hi]))."""
    u = uniform01(seed, stream, count)
    return np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def exp_gaps(count: int, rate: float, seed: int = DEFAULT_SEED,
             stream: int = STREAM_ARRIVALS) -> np.ndarray:
    """Poisson-process inter-arrival gaps (seconds) with the given mean rate."""
    u = uniform01(seed, stream, count)
    return -np.log1p(-u) / rate


def batch_grid_rhs(i: int, side: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Right-hand side of 2D grid i of the batched workload (its own stream)."""
    return helmholtz_rhs((side, side), seed=seed, stream=STREAM_BATCH_F0 + i)


def batch_cube_rhs(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Right-hand side of the batched workload's n^3 grid, (nz, ny, nx)."""
    return helmholtz_rhs((n * n * n,), seed=seed, stream=STREAM_BATCH_F0 + 999).reshape(n, n, n)
