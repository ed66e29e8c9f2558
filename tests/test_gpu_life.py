"""Parity of the CUDA Game of Life loop with the oracle (bit-exact state, same
iteration count, live count and stop reason), through the C ABI."""
import numpy as np
import pytest
import torch

from conftest import run_solver

pytestmark = pytest.mark.gpu


def life_case(slr, orc, cells, wrap, gens, loop, **extra):
    from paper_1609_04567_gb300 import slr as S
    u = torch.from_numpy(cells).cuda()
    out, r = run_solver(slr, S.SLR_LIFE, u, None, gens,
                        boundary=S.SLR_WRAP if wrap else S.SLR_DIRICHLET, loop=loop, **extra)
    ref, rr = orc.life(cells, wrap=wrap, max_gens=gens)
    assert np.array_equal(out, ref)
    assert (r.iters, r.count, r.converged) == (rr.iters, rr.count, rr.converged)
    assert r.status == (0 if rr.converged else 1)


@pytest.mark.parametrize("ny,nx", [(300, 1040), (257, 512), (8, 16), (70, 2048 + 32)])
@pytest.mark.parametrize("wrap", [True, False])
def test_fast_path_matches_oracle(gpu, orc, ny, nx, wrap):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(ny, nx, seed=ny * 7 + nx)
    life_case(gpu, orc, cells, wrap, 60, gpu.SLR_LOOP_PERSISTENT)


@pytest.mark.parametrize("ny,nx", [(33, 17), (1, 1), (1, 50), (50, 1), (5, 3), (129, 1000)])
@pytest.mark.parametrize("wrap", [True, False])
def test_generic_path_matches_oracle(gpu, orc, ny, nx, wrap):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(ny, nx, seed=ny + 3 * nx)
    life_case(gpu, orc, cells, wrap, 40, gpu.SLR_LOOP_PERSISTENT)


@pytest.mark.parametrize("ny,nx", [(256, 512), (33, 17)])
def test_host_loop_matches_oracle(gpu, orc, ny, nx):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(ny, nx, seed=11)
    life_case(gpu, orc, cells, True, 30, gpu.SLR_LOOP_HOST)


def test_still_life_stops_after_one_generation(gpu, orc):
    cells = np.zeros((64, 64), np.uint8)
    cells[10:12, 20:22] = 1
    life_case(gpu, orc, cells, True, 100, gpu.SLR_LOOP_PERSISTENT)
    u = torch.from_numpy(cells).cuda()
    _, r = run_solver(gpu, gpu.SLR_LIFE, u, None, 100)
    assert r.iters == 1 and r.converged and r.count == 4


def test_nonbinary_cells_read_as_alive(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(64, 128, seed=3) * np.uint8(200)
    cells[0, :7] = 7
    u = torch.from_numpy(cells).cuda()
    out, r = run_solver(gpu, gpu.SLR_LIFE, u, None, 10)
    ref, rr = orc.life((cells != 0).astype(np.uint8), wrap=True, max_gens=10)
    assert np.array_equal(out, ref) and r.count == rr.count


def test_resume_equals_straight_run(gpu):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(256, 1024, seed=9)
    a = torch.from_numpy(cells).cuda()
    s = gpu.Solver(gpu.SLR_LIFE, a)
    s.run(25)
    r1 = s.result()
    s.run(70)
    r2 = s.result()
    b = torch.from_numpy(cells).cuda()
    _, r3 = run_solver(gpu, gpu.SLR_LIFE, b, None, 70)
    assert r1.iters == 25 and r2.iters == 70 == r3.iters
    assert torch.equal(a, b) and r2.count == r3.count


@pytest.mark.slow
def test_full_size_8192_matches_oracle_sample(gpu, orc):
    # the benchmark workload (8192 x 8192 torus) in the benchmark's launch
    # configuration, against the oracle for as many generations as it runs in
    # seconds
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(8192, 8192)
    life_case(gpu, orc, cells, True, 4, gpu.SLR_LOOP_PERSISTENT)


@pytest.mark.slow
def test_full_size_2000_generations_properties(gpu):
    # at full length no oracle run fits; the torus symmetries must hold at any
    # size: shifting or transposing the input shifts/transposes the output,
    # the reduced live count is the population, and 1000 + 1000 == 2000
    from paper_1609_04567_gb300 import inputs
    cells = torch.from_numpy(inputs.life_cells(8192, 8192)).cuda()
    base = cells.clone()
    s = gpu.Solver(gpu.SLR_LIFE, base)
    s.run(2000)
    r = s.result()
    s.close()
    assert r.iters == 2000 and not r.converged
    assert r.count == int(base.sum().item())
    sh = torch.roll(cells, shifts=(37, 1000), dims=(0, 1)).contiguous()
    _, rs = run_solver(gpu, gpu.SLR_LIFE, sh, None, 2000)
    assert torch.equal(sh, torch.roll(base, shifts=(37, 1000), dims=(0, 1)))
    tr = cells.t().contiguous()
    _, rt = run_solver(gpu, gpu.SLR_LIFE, tr, None, 2000)
    assert torch.equal(tr, base.t())
    half = cells.clone()
    s = gpu.Solver(gpu.SLR_LIFE, half)
    s.run(1000)
    s.run(2000)
    rh = s.result()
    s.close()
    assert torch.equal(half, base) and rh.count == r.count == rs.count == rt.count


# ---- temporal-blocked path (K generations per pass over a bit-packed grid) ----
# It serves widths that are multiples of 32; tiles own 1024 columns and
# 482 - 2K rows (several tiles in y from ny = 1000).

@pytest.mark.parametrize("ny,nx,wrap", [
    (256, 1024, True), (96, 2176, True), (32, 128, True), (480, 3072, True), (64, 1152, True),
    (257, 1024, True), (1, 32, True), (7, 96, True), (450, 2048, True),
    (257, 512, False), (70, 2080, False), (500, 1056, False), (33, 32, False), (1, 64, False),
    (1000, 1024, True), (1000, 1056, False),
])
@pytest.mark.parametrize("k", [2, 7, 16, 32])
def test_temporal_blocked_matches_oracle(gpu, orc, ny, nx, wrap, k):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(ny, nx, seed=ny + nx + k)
    u = torch.from_numpy(cells).cuda()
    out, r = run_solver(gpu, gpu.SLR_LIFE, u, None, 45,
                        boundary=gpu.SLR_WRAP if wrap else gpu.SLR_DIRICHLET, temporal_k=k)
    ref, rr = orc.life(cells, wrap=wrap, max_gens=45)
    assert np.array_equal(out, ref)
    assert (r.iters, r.count, r.converged) == (rr.iters, rr.count, rr.converged)


@pytest.mark.parametrize("k", [4, 16])
def test_temporal_blocked_stops_inside_a_pass(gpu, orc, k):
    # a blinker and a block that fade into a still state after a few
    # generations: the stop generation falls inside a K-generation pass
    cells = np.zeros((256, 1024), np.uint8)
    cells[100:102, 300:302] = 1                       # block: still
    cells[10, 10:13] = 1                              # blinker next to ...
    cells[11, 13] = 1                                 # ... a cell that perturbs it
    u = torch.from_numpy(cells).cuda()
    out, r = run_solver(gpu, gpu.SLR_LIFE, u, None, 500, temporal_k=k)
    ref, rr = orc.life(cells, wrap=True, max_gens=500)
    assert np.array_equal(out, ref)
    assert (r.iters, r.count, r.converged) == (rr.iters, rr.count, rr.converged)


def test_temporal_blocked_resume_and_cap(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(512, 2048, seed=77)
    a = torch.from_numpy(cells).cuda()
    s = gpu.Solver(gpu.SLR_LIFE, a, temporal_k=16)
    s.run(13)
    r1 = s.result()
    s.run(61)
    r2 = s.result()
    s.close()
    ref, rr = orc.life(cells, wrap=True, max_gens=61)
    assert r1.iters == 13 and r2.iters == 61 == rr.iters
    assert np.array_equal(a.cpu().numpy(), ref) and r2.count == rr.count
