"""FP64 defect correction around FP32 Jacobi inner solves: bit-exact with the
oracle (same operations in the same order), iteration counts equal, and the
returned state's scaled FP64 defect below the tolerance when recomputed by
the oracle."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,k_in,tol", [((12, 12), 20, 1e-10), ((64, 64), 50, 1e-10), ((33, 47), 30, 1e-9),
                                            ((1, 1), 5, 1e-12)])
def test_defect_correction_matches_oracle(gpu, orc, shape, k_in, tol):
    from paper_1609_04567_gb300 import inputs
    f = inputs.helmholtz_rhs(shape, seed=31)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    s = gpu.Solver(gpu.SLR_J2D5, u, torch.from_numpy(f).cuda(), tol=tol, defect_correction=1, inner_sweeps=k_in)
    s.run(100000)
    r = s.result()
    s.close()
    ref, rr = orc.j2d5_dc(np.zeros(shape), f, tol=tol, k_in=k_in, max_outer=100000)
    assert (r.iters, r.converged) == (rr.iters, rr.converged)
    out = u.cpu().numpy()
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))
    assert r.value == rr.value < tol
    assert orc.j2d5_scaled_defect(out, f) < tol


def test_defect_correction_cap_and_resume(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    f = inputs.helmholtz_rhs((40, 40), seed=32)
    u = torch.zeros((40, 40), dtype=torch.float64, device="cuda")
    s = gpu.Solver(gpu.SLR_J2D5, u, torch.from_numpy(f).cuda(), tol=1e-10, defect_correction=1, inner_sweeps=10)
    s.run(3)
    r1 = s.result()
    s.run(100000)
    r2 = s.result()
    s.close()
    ref, rr = orc.j2d5_dc(np.zeros((40, 40)), f, tol=1e-10, k_in=10)
    assert r1.iters == 3 and not r1.converged
    # a resumed run restarts the inner solve from the stored state: the same
    # operations as one straight run
    assert r2.iters == rr.iters and np.array_equal(u.cpu().numpy(), ref)


def test_defect_correction_rejects_other_setups(gpu):
    f = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.SlrError) as e:
        gpu.Solver(gpu.SLR_J2D5, torch.zeros_like(f), f, defect_correction=1)
    assert e.value.status == gpu.SLR_ERR_UNSUPPORTED


@pytest.mark.parametrize("shape,k_in,tol", [((6, 7, 8), 15, 1e-10), ((20, 24, 32), 30, 1e-10),
                                            ((1, 1, 1), 4, 1e-12), ((9, 1, 13), 10, 1e-11)])
def test_defect_correction_3d_matches_oracle(gpu, orc, shape, k_in, tol):
    from paper_1609_04567_gb300 import inputs
    f = inputs.helmholtz_rhs(shape, seed=33)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    s = gpu.Solver(gpu.SLR_J3D7, u, torch.from_numpy(f).cuda(), tol=tol, defect_correction=1, inner_sweeps=k_in)
    s.run(100000)
    r = s.result()
    s.close()
    ref, rr = orc.j3d7_dc(np.zeros(shape), f, tol=tol, k_in=k_in, max_outer=100000)
    assert (r.iters, r.converged) == (rr.iters, rr.converged)
    out = u.cpu().numpy()
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))
    assert r.value == rr.value < tol
    assert orc.j3d7_scaled_defect(out, f) < tol
