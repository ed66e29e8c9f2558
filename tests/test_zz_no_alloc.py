"""The allocation-free Jacobi entry point (slr_run_static).

It is meant for callers that cannot allocate device memory when they need a
solve (for example under a memory budget owned by another framework's
allocator, or in a loop that must not call cudaMalloc/cudaFree because those
synchronise the device).  Its scratch lives in a static device array inside
the library, so these tests check that it gives what the ordinary entry point
gives (slr_create + slr_run_until + slr_reduce_value with a caller workspace)
on two calls in a row -- the second call must not see the first call's
leftovers -- and that grids larger than the array are refused.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def reference_solve(slr, f, **fields):
    u = torch.zeros_like(f)
    s = slr.Solver(slr.SLR_J2D5 if f.dim() == 2 else slr.SLR_J3D7, u, f, **fields)
    s.run(5000)
    r = s.result()
    s.close()
    return u, r


@pytest.mark.parametrize("shape,storage", [((256, 256), torch.float64), ((96, 80), torch.bfloat16),
                                           ((12, 20, 24), torch.float64)])
def test_static_entry_matches_workspace_entry_on_two_calls(gpu, shape, storage):
    from paper_1609_04567_gb300 import inputs
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((101, 202)):
        f64 = inputs.helmholtz_rhs(shape, seed=seed)
        f = torch.from_numpy(f64).to(storage).cuda() if storage != torch.float64 else torch.from_numpy(f64).cuda()
        ref_u, ref = reference_solve(gpu, f, tol=1e-6)
        u = torch.zeros_like(f)
        d = gpu.slr_desc_init(gpu.SLR_J2D5 if len(shape) == 2 else gpu.SLR_J3D7,
                              shape[-1], shape[-2], shape[0] if len(shape) == 3 else 1,
                              storage=gpu.storage_of(storage), tol=1e-6)
        st, value, iters, converged = gpu.slr_run_static(d, u.data_ptr(), f.data_ptr(), 5000, stream.cuda_stream)
        assert st == ref.status and (iters, converged) == (ref.iters, ref.converged), f"call {call}"
        a, b = u.double().cpu().numpy(), ref_u.double().cpu().numpy()
        tol = 1e-12 if storage == torch.float64 else 1e-2
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b)), f"call {call}"
        assert value == pytest.approx(ref.value, rel=tol)


def test_static_entry_rejects_grids_beyond_its_array(gpu):
    # 1024 x 1024 binary64 needs 8 MiB of state, twice what the array holds
    f = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    d = gpu.slr_desc_init(gpu.SLR_J2D5, 1024, 1024, 1)
    st, *_ = gpu.slr_run_static(d, u.data_ptr(), f.data_ptr(), 10, 0, check=False)
    assert st == gpu.SLR_ERR_INVALID_ARG
    msg = gpu.slr_static_last_error()
    assert "SLR_STATIC_STATE_BYTES" in msg and str(gpu.SLR_STATIC_STATE_BYTES) in msg
    life = gpu.slr_desc_init(gpu.SLR_LIFE, 64, 64, 1)
    st, *_ = gpu.slr_run_static(life, u.data_ptr(), f.data_ptr(), 10, 0, check=False)
    assert st == gpu.SLR_ERR_UNSUPPORTED
