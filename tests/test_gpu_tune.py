"""The autotuner and the launch choices it searches.

Grid size, Life's generations per pass, the restoration's tiling and the loop
driver must not change any result: every setting is checked bit-exact against
the oracle.  The tuner must leave the caller's state untouched, return a
choice no slower than the library default it timed, cache it under the exact
shape and the shape's power-of-two bucket, and hand it to later slr_create
calls whose fields are left to the library."""
import numpy as np
import pytest
import torch

from test_gpu_jacobi import jacobi_case
from test_gpu_life import life_case
from test_gpu_restore import restore_case

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def empty_cache(gpu):
    gpu.slr_tune_clear()
    yield
    gpu.slr_tune_clear()


# ---- launch choices leave results unchanged ---------------------------------

@pytest.mark.parametrize("grid", [1, 3, 7, 100000])
def test_jacobi_any_grid_size_is_bit_exact(gpu, orc, grid):
    jacobi_case(gpu, orc, (130, 200), grid_ctas=grid)


@pytest.mark.parametrize("grid", [1, 5])
def test_j3d7_bf16_any_grid_size_is_bit_exact(gpu, orc, grid):
    jacobi_case(gpu, orc, (9, 20, 33), storage="bf16", grid_ctas=grid)


@pytest.mark.parametrize("k,grid", [(6, 1), (6, 5), (12, 17), (1, 3), (0, 2)])
def test_life_any_grid_size_is_bit_exact(gpu, orc, k, grid):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(520, 1024, seed=k * 31 + grid)
    life_case(gpu, orc, cells, True, 70, gpu.SLR_LOOP_PERSISTENT, temporal_k=k, grid_ctas=grid)


@pytest.mark.parametrize("tiling,grid", [(2, 1), (2, 9), (1, 5), (1, 0), (2, 0)])
def test_restore_tiling_and_grid_size_are_bit_exact(gpu, orc, tiling, grid):
    out, r, ref, rr = restore_case(gpu, orc, 200, 256, tiling=tiling, grid_ctas=grid)
    assert r.iters == rr.iters and r.converged == rr.converged and r.count == rr.count
    assert np.array_equal(out.view(np.uint32), ref.view(np.uint32)) and r.value == rr.value


@pytest.mark.parametrize("k,grid", [(2, 1), (4, 7), (8, 152), (8, 0), (3, 600)])
def test_restore_temporal_k_and_grid_size_are_bit_exact(gpu, orc, k, grid):
    out, r, ref, rr = restore_case(gpu, orc, 200, 256, temporal_k=k, grid_ctas=grid)
    assert (r.iters, r.converged, r.count, r.value) == (rr.iters, rr.converged, rr.count, rr.value)
    assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("grid", [2, 11])
def test_defect_correction_any_grid_size_is_bit_exact(gpu, orc, grid):
    from paper_1609_04567_gb300 import inputs
    f = inputs.helmholtz_rhs((48, 40), seed=5)
    u = torch.zeros((48, 40), dtype=torch.float64, device="cuda")
    s = gpu.Solver(gpu.SLR_J2D5, u, torch.from_numpy(f).cuda(), tol=1e-10, defect_correction=1,
                   inner_sweeps=20, grid_ctas=grid)
    s.run(1000)
    r = s.result()
    s.close()
    ref, rr = orc.j2d5_dc(np.zeros((48, 40)), f, tol=1e-10, k_in=20, max_outer=1000)
    assert (r.iters, r.converged, r.value) == (rr.iters, rr.converged, rr.value)
    assert np.array_equal(u.cpu().numpy().view(np.uint64), ref.view(np.uint64))


# ---- the tuner ----------------------------------------------------------------

def check_choice(gpu, r, stencil):
    assert r["loop"] in (gpu.SLR_LOOP_HOST, gpu.SLR_LOOP_PERSISTENT)
    assert r["grid_ctas"] >= 0 and r["trials"] >= 2
    assert 0.0 < r["ms_per_iter"] <= r["default_ms_per_iter"]
    if stencil == gpu.SLR_LIFE:
        assert 1 <= r["temporal_k"] <= 32
    if stencil == gpu.SLR_RESTORE8:
        assert r["tiling"] in (gpu.SLR_TILING_NONE, gpu.SLR_TILING_TMA)
        assert 1 <= r["temporal_k"] <= 8


def test_tune_life_reads_only_and_later_solves_stay_exact(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(512, 1024, seed=77)
    u = torch.from_numpy(cells).cuda()
    r = gpu.tune(gpu.SLR_LIFE, u, trial_iters=48)
    assert np.array_equal(u.cpu().numpy(), cells)
    check_choice(gpu, r, gpu.SLR_LIFE)
    d = gpu.slr_desc_init(gpu.SLR_LIFE, 1024, 512, 1)
    got = gpu.slr_tune_lookup(d).as_dict()
    assert got == r
    life_case(gpu, orc, cells, True, 90, gpu.SLR_LOOP_AUTO)


def test_tune_helmholtz_256_fp64(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    f = torch.from_numpy(inputs.helmholtz_rhs((256, 256), seed=1)).cuda()
    u = torch.zeros((256, 256), dtype=torch.float64, device="cuda")
    r = gpu.tune(gpu.SLR_J2D5, u, f, trial_iters=32)
    assert torch.count_nonzero(u).item() == 0
    check_choice(gpu, r, gpu.SLR_J2D5)
    assert jacobi_case(gpu, orc, (256, 256)).converged


def test_tune_restore(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(256, 256, seed=1)
    mask = torch.from_numpy(inputs.noise_mask(frame)).cuda()
    u = torch.from_numpy(frame.astype(np.float32)).cuda()
    r = gpu.tune(gpu.SLR_RESTORE8, u, mask, trial_iters=16)
    assert np.array_equal(u.cpu().numpy(), frame.astype(np.float32))
    check_choice(gpu, r, gpu.SLR_RESTORE8)
    out, res, ref, rr = restore_case(gpu, orc, 256, 256)
    assert res.iters == rr.iters and np.array_equal(out.view(np.uint32), ref.view(np.uint32))


def test_tune_defect_correction_keeps_the_device_loop(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    f = torch.from_numpy(inputs.helmholtz_rhs((64, 64), seed=2)).cuda()
    u = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    r = gpu.tune(gpu.SLR_J2D5, u, f, trial_iters=2, defect_correction=1, inner_sweeps=10)
    assert r["loop"] == gpu.SLR_LOOP_PERSISTENT
    check_choice(gpu, r, gpu.SLR_J2D5)


def test_explicit_fields_are_held_fixed(gpu):
    from paper_1609_04567_gb300 import inputs
    u = torch.from_numpy(inputs.life_cells(256, 512, seed=4)).cuda()
    r = gpu.tune(gpu.SLR_LIFE, u, trial_iters=24, loop=gpu.SLR_LOOP_PERSISTENT, temporal_k=4, grid_ctas=19)
    assert (r["loop"], r["temporal_k"], r["grid_ctas"]) == (gpu.SLR_LOOP_PERSISTENT, 4, 19)
    assert r["trials"] == 1 and r["ms_per_iter"] == r["default_ms_per_iter"]


def test_bucket_lookup_and_clear(gpu):
    from paper_1609_04567_gb300 import inputs
    u = torch.from_numpy(inputs.life_cells(512, 1024, seed=9)).cuda()
    r = gpu.tune(gpu.SLR_LIFE, u, trial_iters=16)
    near = gpu.slr_desc_init(gpu.SLR_LIFE, 1100, 600, 1)          # same floor(log2) extents
    assert gpu.slr_tune_lookup(near).as_dict() == r
    assert gpu.slr_tune_lookup(gpu.slr_desc_init(gpu.SLR_LIFE, 1024, 256, 1)) is None
    assert gpu.slr_tune_lookup(gpu.slr_desc_init(gpu.SLR_LIFE, 1024, 512, 1, boundary=gpu.SLR_DIRICHLET)) is None
    gpu.slr_tune_clear()
    assert gpu.slr_tune_lookup(near) is None
