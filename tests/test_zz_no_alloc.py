"""The allocation-free Jacobi entry point (slr_run_static).

It is meant for callers that cannot allocate device memory when they need a
solve: code running under a device-memory budget that another framework's
allocator owns, real-time loops that forbid allocation after start-up, or
host threads where cudaMalloc/cudaFree would synchronise the device and stall
other streams.  Its scratch (the second state buffer and the loop's control
block) lives in a static device array inside the library, shared by every
call.

These tests run two calls in a row on different inputs -- the second call
must not see what the first left in the shared array -- and check each call
bit for bit against the oracle (state, iteration count, reduced value) and
against the ordinary entry point (slr_create + slr_run_until +
slr_reduce_value with a caller workspace), within the tolerances the other
Jacobi tests use.  Grids larger than the array are refused.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.bfloat16: 1e-2, torch.float32: 1e-5}
ORACLE_STORAGE = {torch.float64: None, torch.bfloat16: "bf16", torch.float32: "f32"}


def reference_solve(slr, f, **fields):
    u = torch.zeros_like(f)
    s = slr.Solver(slr.SLR_J2D5 if f.dim() == 2 else slr.SLR_J3D7, u, f, **fields)
    s.run(5000)
    r = s.result()
    s.close()
    return u, r


def oracle_solve(orc, f_dev, storage):
    """The oracle's loop on the same (storage-rounded) f, from u = 0."""
    fn = orc.j2d5 if f_dev.dim() == 2 else orc.j3d7
    st = ORACLE_STORAGE[storage]
    if st is None:
        f = f_dev.cpu().numpy()
        return fn(np.zeros_like(f), f, tol=1e-6, max_iters=5000)
    f = f_dev.float().cpu().numpy()
    return fn(np.zeros_like(f), f, tol=1e-6, max_iters=5000, storage=st)


@pytest.mark.parametrize("shape,storage", [((256, 256), torch.float64), ((96, 80), torch.bfloat16),
                                           ((200, 328), torch.float32), ((12, 20, 24), torch.float64)])
def test_static_entry_matches_oracle_and_workspace_entry_on_two_calls(gpu, orc, shape, storage):
    from paper_1609_04567_gb300 import inputs
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((101, 202)):
        f64 = inputs.helmholtz_rhs(shape, seed=seed)
        f = torch.from_numpy(f64).cuda()
        if storage != torch.float64:
            f = f.float().to(storage)
        ref_u, ref = reference_solve(gpu, f, tol=1e-6)
        u = torch.zeros_like(f)
        d = gpu.slr_desc_init(gpu.SLR_J2D5 if len(shape) == 2 else gpu.SLR_J3D7,
                              shape[-1], shape[-2], shape[0] if len(shape) == 3 else 1,
                              storage=gpu.storage_of(storage), tol=1e-6)
        st, value, iters, converged = gpu.slr_run_static(d, u.data_ptr(), f.data_ptr(), 5000, stream.cuda_stream)
        # bit for bit against the oracle: state, iteration count, reduced value
        want, wr = oracle_solve(orc, f, storage)
        got = u.double().cpu().numpy() if storage != torch.float64 else u.cpu().numpy()
        assert np.array_equal(got, want.astype(np.float64) if storage != torch.float64 else want), f"call {call}"
        assert (iters, converged, value) == (wr.iters, wr.converged, wr.value), f"call {call}"
        # and against the workspace entry point within the tolerance the Jacobi tests use
        assert st == ref.status and (iters, converged) == (ref.iters, ref.converged), f"call {call}"
        a, b = u.double().cpu().numpy(), ref_u.double().cpu().numpy()
        assert np.max(np.abs(a - b)) <= TOL[storage] * np.max(np.abs(b)), f"call {call}"
        assert value == pytest.approx(ref.value, rel=TOL[storage])


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
