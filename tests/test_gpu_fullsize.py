"""Full-size configurations against the oracle, bit for bit, for their whole
run or a large part of it, in the launch configuration the benchmark times.

The oracle's threaded build (the rows of each sweep shared among all host
cores; the same values as the single-threaded build, checked on CPU) makes
these runs fit in seconds to a minute:

  * the 8192 x 8192 Game of Life torus for 100 generations (four passes of
    the temporal-blocked kernel's default 25 generations per pass), and a
    dead torus with a pattern that dies out after 130 generations, so the
    per-pass still-state logic stops the run inside its sixth pass;
  * the 4096 x 4096 restoration (50% salt-and-pepper) to convergence;
  * the batched workload (512 2D Helmholtz grids with sides log-uniform in
    [64, 1024] plus one 512^3 grid, bfloat16 storage, tol 1e-6, cap 5000) run
    as one batch, with 32 of its grids (every 16th, so the sample follows the
    side distribution) and the 3D grid compared with the oracle.

For every bfloat16 result of the batch sample the error against the FP64
oracle is stated: max |u - u64| / max |u64| with u64 the FP64 oracle's iterate
after the same number of sweeps (the storage precision's own error), and
against the FP64 oracle run to the same tolerance (which may stop at another
sweep).  Rounding every stored value to bfloat16 adds at most 2^-8 relative
per sweep, so after n sweeps the first error is bounded a priori by about
2n * 2^-8 (input rounding included); one sweep stays below 1e-2."""
import os

import numpy as np
import pytest
import torch

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CORES = os.cpu_count() or 1


def _place(grid, pattern, y, x):
    rows = pattern.strip("\n").split("\n")
    for dy, row in enumerate(rows):
        for dx, ch in enumerate(row):
            grid[y + dy, x + dx] = 1 if ch == "#" else 0


DIEHARD = """
......#.
##......
.#...###
"""
BLOCK = """
##
##
"""


def test_life_8192_torus_100_generations_vs_oracle(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(8192, 8192)
    u = torch.from_numpy(cells).cuda()
    s = gpu.Solver(gpu.SLR_LIFE, u)           # library defaults: 25 generations per pass here
    s.run(100)
    r = s.result()
    s.close()
    with orc.threads(CORES):
        ref, rr = orc.life(cells, wrap=True, max_gens=100)
    assert np.array_equal(u.cpu().numpy(), ref)
    assert (r.iters, r.count, r.converged, r.value) == (rr.iters, rr.count, rr.converged, rr.value) == \
        (100, rr.count, False, float(rr.count))


def test_life_8192_torus_stills_inside_a_pass_vs_oracle(gpu, orc):
    cells = np.zeros((8192, 8192), dtype=np.uint8)
    _place(cells, DIEHARD, 4000, 4000)
    for y, x in [(100, 100), (7000, 300), (2000, 8100), (8190, 5000), (6000, 6000)]:
        _place(cells, BLOCK, y, x)              # (2000, 8100) and (8190, 5000) sit near the wrap seams
    u = torch.from_numpy(cells).cuda()
    s = gpu.Solver(gpu.SLR_LIFE, u)
    s.run(2000)
    r = s.result()
    s.close()
    with orc.threads(CORES):
        ref, rr = orc.life(cells, wrap=True, max_gens=2000)
    assert rr.converged and rr.count == 20 and 125 < rr.iters <= 150   # inside the sixth 25-generation pass
    assert np.array_equal(u.cpu().numpy(), ref)
    assert (r.iters, r.count, r.converged) == (rr.iters, rr.count, rr.converged)


def test_restore_4096_to_convergence_vs_oracle(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(4096, 4096)
    mask = inputs.noise_mask(frame)
    u = torch.from_numpy(frame.astype(np.float32)).cuda()
    s = gpu.Solver(gpu.SLR_RESTORE8, u, torch.from_numpy(mask).cuda(), tol=1e-3)
    s.run(5000)
    r = s.result()
    s.close()
    with orc.threads(CORES):
        ref, rr = orc.restore8(frame.astype(np.float32), mask, tol=1e-3, max_iters=5000)
    assert rr.converged and rr.iters > 20
    assert np.array_equal(u.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    assert (r.iters, r.value, r.count, r.converged) == (rr.iters, rr.value, rr.count, rr.converged)


def _bf16(a64):
    return torch.from_numpy(np.ascontiguousarray(a64).astype(np.float32)).to(torch.bfloat16)


def test_batch_workload_sample_vs_oracle_with_fp64_errors(gpu, orc, record_property):
    from paper_1609_04567_gb300 import inputs
    sides = [int(x) for x in inputs.batch_sides(512)]
    grids = []
    for i, sd in enumerate(sides):
        f = _bf16(inputs.batch_grid_rhs(i, sd)).cuda()
        grids.append((f, torch.zeros_like(f)))
    f3 = _bf16(inputs.batch_cube_rhs(512)).cuda()
    grids.append((f3, torch.zeros_like(f3)))
    b = gpu.Batch(len(grids) + 1)
    slots = [b.add(gpu.SLR_J3D7 if u.dim() == 3 else gpu.SLR_J2D5, u, f, 5000, tol=1e-6) for f, u in grids]
    b.run(100000)
    _, running = b.poll()
    assert running == 0
    sample = list(range(0, 512, 16)) + [512]
    rows = []
    for i in sample:
        f, u = grids[i]
        r = b.result(slots[i])
        got = u.float().cpu().numpy()
        f_or = f.float().cpu().numpy()
        f64 = inputs.batch_cube_rhs(512) if i == 512 else inputs.batch_grid_rhs(i, sides[i])
        fn = orc.j3d7 if i == 512 else orc.j2d5
        with orc.threads(CORES if i == 512 or sides[i] >= 512 else 1):
            ref, rr = fn(np.zeros_like(f_or), f_or, tol=1e-6, max_iters=5000, storage="bf16")
            assert np.array_equal(got, ref), f"grid {i}"
            assert (r.iters, r.converged, r.value) == (rr.iters, rr.converged, rr.value), f"grid {i}"
            # the FP64 oracle on the unrounded f: after the same sweeps, and run to the same tolerance
            same, _ = fn(np.zeros_like(f64), f64, tol=0.0, max_iters=r.iters)
            own, ro = fn(np.zeros_like(f64), f64, tol=1e-6, max_iters=5000)
        g = got.astype(np.float64)
        e_same = float(np.max(np.abs(g - same)) / np.max(np.abs(same)))
        e_own = float(np.max(np.abs(g - own)) / np.max(np.abs(own)))
        rows.append((i, "512^3" if i == 512 else f"{sides[i]}^2", r.iters, r.converged, ro.iters, e_same, e_own))
        assert e_same <= 2.0 * r.iters * 2.0 ** -8 * 1.01, rows[-1]
        if r.iters == 1:
            assert e_same <= 1e-2, rows[-1]
    b.close()
    record_property("bf16_fp64_errors", rows)
    print("\ngrid  size  sweeps  converged  fp64_sweeps  err_same_sweeps  err_vs_fp64_at_tol")
    for row in rows:
        print("%4d %7s %6d %6s %8d %12.3e %12.3e" % row)
