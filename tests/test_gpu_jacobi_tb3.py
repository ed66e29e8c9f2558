"""Temporal-blocked 3D Jacobi (k <= 4 sweeps per HBM pass, binary32 arithmetic
with binary32 / bfloat16 / binary16 storage, a Dirichlet ghost value) against
the oracle: bit-identical states, equal iteration counts and reduced values,
for fixed sweep counts over grids of several ragged work units (columns of 48
owned x by 24 - 2K owned y cells, chunks of 64 planes) and for solves that
stop in the middle of a pass (the pass is recomputed up to the stopping
sweep)."""
import numpy as np
import pytest
import torch

from test_gpu_jacobi import jacobi_case

pytestmark = pytest.mark.gpu

# (nz, ny, nx): several units along every axis with ragged last ones, chunks
# of 64 planes plus a ragged one, grids smaller than one unit, single planes
SHAPES = [((70, 50, 104), "f32"), ((130, 37, 96), "bf16"), ((65, 21, 200), "f16"), ((9, 40, 52), "f32"),
          ((3, 3, 16), "bf16"), ((1, 1, 8), "f16"), ((1, 30, 100), "f32"), ((129, 8, 48), "bf16"),
          ((40, 1, 4), "f32")]


@pytest.mark.parametrize("shape,storage", SHAPES)
@pytest.mark.parametrize("k", [4, 3, 2])
def test_fixed_sweeps_bit_exact(gpu, orc, shape, storage, k):
    # 11 sweeps: whole passes and a shorter last one
    r = jacobi_case(gpu, orc, shape, storage=storage, tol=0.0, max_iters=11, temporal_k=k)
    assert r.iters == 11 and not r.converged


@pytest.mark.parametrize("k", [2, 4, 5, 32])
def test_every_k(gpu, orc, k):
    # k above the pipeline depth runs the most sweeps a pass can take
    jacobi_case(gpu, orc, (34, 60, 120), storage="f32", tol=0.0, max_iters=13, temporal_k=k)


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("shape", [(24, 24, 24), (40, 30, 64)])
def test_convergence_stops_mid_pass(gpu, orc, storage, shape):
    # the stopping sweep falls inside a pass: state, value and count must be
    # those of the one-sweep loop
    r = jacobi_case(gpu, orc, shape, storage=storage, tol=1e-6, max_iters=3000, temporal_k=4)
    assert r.converged or storage != "f32"


@pytest.mark.parametrize("tol", [1e-3, 3e-4, 1e-4, 3e-5])
def test_stop_at_each_position_in_the_pass(gpu, orc, tol):
    # different tolerances put the stopping sweep at different places in a pass
    r = jacobi_case(gpu, orc, (20, 36, 72), storage="f32", tol=tol, max_iters=3000, temporal_k=4)
    assert r.converged


def test_tuned_choice_matches(gpu, orc):
    # the autotuner times k = 2 and 4 against the default on this grid; whatever it keeps,
    # the solve equals the oracle's
    from paper_1609_04567_gb300 import inputs
    shape = (30, 44, 96)
    f32 = inputs.helmholtz_rhs(shape, seed=1).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    u = torch.zeros(shape, dtype=torch.float32, device="cuda")
    r = gpu.tune(gpu.SLR_J3D7, u, f, tol=1e-5, trial_iters=16)
    assert r["temporal_k"] in (0, 1, 2, 4) and r["trials"] >= 3        # 0: the library default
    s = gpu.Solver(gpu.SLR_J3D7, u, f, tol=1e-5)
    s.run(3000)
    r = s.result()
    s.close()
    ref, rr = orc.j3d7(np.zeros(shape, dtype=np.float32), f32, tol=1e-5, max_iters=3000, storage="f32")
    assert (r.iters, r.converged, r.value) == (rr.iters, rr.converged, rr.value)
    assert np.array_equal(u.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_first_sweep_converges(gpu):
    u = torch.zeros((16, 16, 16), dtype=torch.float32, device="cuda")
    f = torch.zeros((16, 16, 16), dtype=torch.float32, device="cuda")
    s = gpu.Solver(gpu.SLR_J3D7, u, f, tol=1e-9, temporal_k=4)
    s.run(100)
    r = s.result()
    s.close()
    assert (r.iters, r.converged, r.value) == (1, True, 0.0)
    assert not u.any()


@pytest.mark.parametrize("caps", [(1, 2, 3000), (5, 6, 3000), (3, 11, 3000)])
def test_cap_and_resume(gpu, orc, caps):
    # caps that end inside a pass run only the sweeps left; each run resumes
    # from the state in u, and the last equals a straight run
    from paper_1609_04567_gb300 import inputs
    shape = (33, 26, 56)
    f32 = inputs.helmholtz_rhs(shape, seed=4).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    u = torch.zeros(shape, dtype=torch.float32, device="cuda")
    s = gpu.Solver(gpu.SLR_J3D7, u, f, tol=1e-6, temporal_k=4)
    for cap in caps[:-1]:
        s.run(cap)
        r = s.result(check=False)
        assert r.iters == cap and not r.converged
        ref, rr = orc.j3d7(np.zeros(shape, dtype=np.float32), f32, tol=1e-6, max_iters=cap, storage="f32")
        assert r.value == rr.value and np.array_equal(u.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    s.run(caps[-1])
    r2 = s.result()
    s.close()
    ref, rr = orc.j3d7(np.zeros(shape, dtype=np.float32), f32, tol=1e-6, max_iters=caps[-1], storage="f32")
    assert (r2.iters, r2.converged, r2.value) == (rr.iters, rr.converged, rr.value)
    assert np.array_equal(u.cpu().numpy().view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("storage,ghost", [("f32", 0.25), ("f32", -0.0), ("f32", 1.0 / 3.0), ("bf16", 0.75),
                                           ("f16", -1.5), ("bf16", -0.0)])
@pytest.mark.parametrize("shape", [(30, 40, 104), (5, 7, 16)])
def test_dirichlet_ghost_values(gpu, orc, storage, ghost, shape):
    # the planes below 0 and from nz on and the cells outside the grid hold
    # the ghost value at every level of the pass
    jacobi_case(gpu, orc, shape, storage=storage, tol=1e-5, max_iters=3000, temporal_k=4, ghost=ghost)


@pytest.mark.parametrize("storage,kw", [("f32", dict(sigma=0.0)), ("bf16", dict(h=0.01, sigma=3.0)),
                                        ("f32", dict(sigma=1e20)), ("f16", dict(sigma=1e20))])
def test_other_constants(gpu, orc, storage, kw):
    # Poisson (sigma 0), another mesh width, and a divisor outside the range of
    # the corrected quotient (every division through the IEEE operation)
    jacobi_case(gpu, orc, (21, 30, 96), storage=storage, tol=0.0, max_iters=9, temporal_k=4, **kw)


@pytest.mark.parametrize("storage,kw", [("f32", dict(wrap=True)), ("f64", dict()), ("bf16", dict()),
                                        ("bf16", dict(ghost=0.1))])
def test_requests_it_does_not_apply_to_fall_back(gpu, orc, storage, kw):
    # periodic boundary, binary64 state, 2-byte rows that are not whole 16-byte
    # groups (nx = 36), and a ghost value bfloat16 cannot hold run the
    # one-sweep-per-pass loop
    shape = (9, 10, 36) if storage == "bf16" and not kw else (9, 10, 64)
    jacobi_case(gpu, orc, shape, storage=storage, tol=0.0, max_iters=7, temporal_k=4, **kw)


@pytest.mark.slow
def test_full_size_3d_bf16(gpu):
    # the 512^3 bf16 grid of the batch workload: one whole pass of 4 sweeps
    # and one more sweep, against the one-sweep-per-pass loop (its own parity
    # with the oracle at this size is tested elsewhere); the grid is large
    # enough that every unit count and the dynamic hand-out are exercised
    from paper_1609_04567_gb300 import inputs
    n = 512
    f = torch.from_numpy(inputs.batch_cube_rhs(n)).to(torch.bfloat16).cuda()
    outs = []
    for k in (1, 4):
        u = torch.zeros((n, n, n), dtype=torch.bfloat16, device="cuda")
        s = gpu.Solver(gpu.SLR_J3D7, u, f, tol=0.0, temporal_k=k)
        s.run(5)
        r = s.result(check=False)
        s.close()
        outs.append((u, r))
    (u1, r1), (u4, r4) = outs
    assert r1.iters == r4.iters == 5 and r1.value == r4.value
    assert torch.equal(u1.view(torch.int16), u4.view(torch.int16))
