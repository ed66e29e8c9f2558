"""Temporal-blocked 2D Jacobi (k sweeps per HBM pass, binary32 arithmetic with
binary32 / bfloat16 / binary16 storage, Dirichlet ghost 0) against the oracle:
bit-identical states, equal iteration counts and reduced values, for fixed
sweep counts over grids of several ragged tiles and for solves that stop in
the middle of a pass (the pass is recomputed up to the stopping sweep)."""
import numpy as np
import pytest
import torch

from test_gpu_jacobi import jacobi_case

pytestmark = pytest.mark.gpu

# tiles hold 240 owned columns by 96 (4-byte storage) or 208 (2-byte storage)
# owned rows: these shapes have ragged tiles in both directions, several tiles
# per axis, and grids smaller than one tile
SHAPES = [((300, 520), "f32"), ((470, 500), "bf16"), ((230, 250), "f16"), ((97, 241), "f32"),
          ((209, 480), "bf16"), ((1, 4), "f32"), ((3, 8), "bf16"), ((2, 8), "f16"), ((193, 16), "f32")]


@pytest.mark.parametrize("shape,storage", SHAPES)
@pytest.mark.parametrize("k", [8, 3])
def test_fixed_sweeps_bit_exact(gpu, orc, shape, storage, k):
    # 23 sweeps: whole passes and a shorter last one
    r = jacobi_case(gpu, orc, shape, storage=storage, tol=0.0, max_iters=23, temporal_k=k)
    assert r.iters == 23 and not r.converged


@pytest.mark.parametrize("k", [2, 5, 7, 8, 32])
def test_every_k(gpu, orc, k):
    # k above the halo width runs the most sweeps a pass can take
    jacobi_case(gpu, orc, (250, 490), storage="f32", tol=0.0, max_iters=17, temporal_k=k)


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("shape", [(96, 80), (256, 256), (130, 500)])
def test_convergence_stops_mid_pass(gpu, orc, storage, shape):
    # the stopping sweep falls inside a pass: state, value and count must be
    # those of the one-sweep loop
    r = jacobi_case(gpu, orc, shape, storage=storage, tol=1e-6, max_iters=3000, temporal_k=8)
    assert r.converged or storage != "f32"


@pytest.mark.parametrize("tol", [1e-3, 1e-4, 3e-5])
def test_stop_at_each_position_in_the_pass(gpu, orc, tol):
    # different tolerances put the stopping sweep at different places in a pass
    r = jacobi_case(gpu, orc, (200, 312), storage="f32", tol=tol, max_iters=3000, temporal_k=8)
    assert r.converged


def test_first_sweep_converges(gpu, orc):
    # f = 0 and u = 0: the first sweep changes nothing and stops the loop
    u = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    f = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    s = gpu.Solver(gpu.SLR_J2D5, u, f, tol=1e-9, temporal_k=8)
    s.run(100)
    r = s.result()
    s.close()
    assert (r.iters, r.converged, r.value) == (1, True, 0.0)
    assert not u.any()


def test_cap_and_resume(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    f32 = inputs.helmholtz_rhs((128, 136), seed=4).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    u = torch.zeros((128, 136), dtype=torch.float32, device="cuda")
    s = gpu.Solver(gpu.SLR_J2D5, u, f, tol=1e-6, temporal_k=8)
    s.run(11)
    r1 = s.result(check=False)
    assert r1.iters == 11 and not r1.converged
    s.run(13)
    assert s.result(check=False).iters == 13
    s.run(3000)
    r2 = s.result()
    s.close()
    ref, rr = orc.j2d5(np.zeros((128, 136), dtype=np.float32), f32, tol=1e-6, max_iters=3000, storage="f32")
    assert (r2.iters, r2.converged, r2.value) == (rr.iters, rr.converged, rr.value)
    assert np.array_equal(u.cpu().numpy().view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("storage,kw", [("f32", dict(wrap=True)), ("f64", dict()), ("bf16", dict()),
                                        ("bf16", dict(ghost=0.1))])
def test_requests_it_does_not_apply_to_fall_back(gpu, orc, storage, kw):
    # periodic boundary, binary64 state, 2-byte rows that are not whole 16-byte
    # groups (nx = 36), and a ghost value bfloat16 cannot hold run the
    # one-sweep-per-pass loop
    shape = (40, 36) if storage == "bf16" and not kw else (40, 64)
    jacobi_case(gpu, orc, shape, storage=storage, tol=0.0, max_iters=11, temporal_k=8, **kw)


@pytest.mark.parametrize("storage,ghost", [("f32", 0.25), ("f32", -0.0), ("f32", 1.0 / 3.0), ("bf16", 0.75),
                                           ("f16", -1.5), ("bf16", -0.0)])
@pytest.mark.parametrize("shape", [(130, 500), (33, 40)])
def test_dirichlet_ghost_values(gpu, orc, storage, ghost, shape):
    # the tiles' cells outside the grid hold the ghost value, to convergence
    jacobi_case(gpu, orc, shape, storage=storage, tol=1e-5, max_iters=3000, temporal_k=8, ghost=ghost)


@pytest.mark.parametrize("storage,kw", [("f32", dict(sigma=0.0)), ("bf16", dict(h=0.01, sigma=3.0)),
                                        ("f32", dict(sigma=1e20)), ("f16", dict(sigma=1e20))])
def test_other_constants(gpu, orc, storage, kw):
    # Poisson (sigma 0), another mesh width, and a divisor outside the range of
    # the corrected quotient (every division through the IEEE operation)
    jacobi_case(gpu, orc, (150, 264), storage=storage, tol=0.0, max_iters=19, temporal_k=8, **kw)


@pytest.mark.slow
def test_full_size_2d(gpu, orc):
    # the large single grids of the Jacobi bench: one whole pass and one sweep
    jacobi_case(gpu, orc, (8192, 8192), storage="f32", tol=0.0, max_iters=9, temporal_k=8)
    jacobi_case(gpu, orc, (8192, 8192), storage="bf16", tol=0.0, max_iters=9, temporal_k=8)
    jacobi_case(gpu, orc, (8192, 8192), storage="f16", tol=0.0, max_iters=9, temporal_k=8)
