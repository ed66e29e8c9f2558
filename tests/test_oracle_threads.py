"""The oracle's threaded build (-fopenmp: the rows of each sweep shared among
host threads) returns bit for bit what the single-threaded build returns, on
every solver: the same state, iteration count, reduced value and count.  It is
the build the benchmark times on all host cores, and the one the full-size
GPU parity tests use to finish in seconds.  CPU only."""
import numpy as np
import pytest

from paper_1609_04567_gb300 import inputs


def both(orc, fn, *args, **kw):
    one = fn(*args, **kw)
    with orc.threads(4) as n:
        many = fn(*args, **kw)
    return one, many, n


def same(one, many):
    (a, ra), (b, rb) = one, many
    assert a.dtype == b.dtype and np.array_equal(a.view(np.uint8), b.view(np.uint8))
    assert ra == rb


@pytest.fixture(scope="module")
def omp(orc):
    if not orc.omp_available():
        pytest.skip("gcc without -fopenmp")
    return orc


@pytest.mark.parametrize("storage", [None, "f32", "bf16", "f16"])
@pytest.mark.parametrize("wrap", [False, True])
def test_j2d5_threads_agree(omp, storage, wrap):
    f = inputs.helmholtz_rhs((61, 45), seed=3)
    if storage is not None:
        f = omp.round_storage(f.astype(np.float32), storage)
    one, many, n = both(omp, omp.j2d5, np.zeros_like(f), f, tol=1e-6, max_iters=300, storage=storage, wrap=wrap,
                        ghost=0.25)
    assert n > 1
    same(one, many)


@pytest.mark.parametrize("storage", [None, "f32", "bf16"])
def test_j3d7_threads_agree(omp, storage):
    f = inputs.helmholtz_rhs((7, 19, 23), seed=4)
    if storage is not None:
        f = omp.round_storage(f.astype(np.float32), storage)
    one, many, _ = both(omp, omp.j3d7, np.zeros_like(f), f, tol=1e-7, max_iters=200, storage=storage)
    same(one, many)


@pytest.mark.parametrize("wrap", [False, True])
def test_life_threads_agree(omp, wrap):
    cells = inputs.life_cells(57, 64, seed=9)
    one, many, _ = both(omp, omp.life, cells, wrap=wrap, max_gens=120)
    same(one, many)


def test_restore8_threads_agree(omp):
    frame, _ = inputs.noisy_frame(53, 64, seed=6)
    mask = inputs.noise_mask(frame)
    one, many, _ = both(omp, omp.restore8, frame.astype(np.float32), mask, tol=1e-3, max_iters=5000)
    same(one, many)


def test_defect_correction_threads_agree(omp):
    f = inputs.helmholtz_rhs((40, 36), seed=8)
    one, many, _ = both(omp, omp.j2d5_dc, np.zeros_like(f), f, tol=1e-10, k_in=20, max_outer=500)
    same(one, many)


def test_outside_the_block_one_thread_again(omp):
    with omp.threads(3) as n:
        assert n == 3
    # the single-threaded build is back in use
    f = inputs.helmholtz_rhs((16, 16), seed=1)
    u, r = omp.j2d5(np.zeros_like(f), f, tol=1e-6)
    assert r.converged and np.isfinite(u).all()
