"""Parity of the CUDA Helmholtz Jacobi loops (2D 5-point, 3D 7-point) with the
oracle through the C ABI.  EXACT math evaluates the oracle's operations in the
oracle's order with IEEE rounding, so the bar is bit-identical states and
equal iteration counts; the stated tolerances (1e-12 relative in FP64, 1e-5 in
FP32, 1e-2 with bfloat16/binary16 storage) are asserted as well."""
import numpy as np
import pytest
import torch

from conftest import run_solver

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-2, "f16": 1e-2}
TORCH = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def rel_err(a, b):
    # in binary64 throughout: an all-zero reference must not divide 0 by a 1e-300 rounded to 0
    return float(np.max(np.abs(a.astype(np.float64) - b.astype(np.float64)))) / max(
        float(np.max(np.abs(b.astype(np.float64)))), 1e-300)


def prepare(f64, storage):
    """f in the storage precision (FP64 -> FP32 (RN) -> storage (RNE)), and the
    same values as the oracle's float64/float32 input."""
    if storage == "f64":
        return torch.from_numpy(f64), f64
    t = torch.from_numpy(f64.astype(np.float32)).to(TORCH[storage])
    return t, t.float().numpy()


def jacobi_case(slr, orc, shape, storage="f64", tol=1e-6, max_iters=5000, wrap=False, ghost=0.0,
                sigma=1.0, h=0.0, loop=None, seed=1, **extra):
    from paper_1609_04567_gb300 import inputs
    f64 = inputs.helmholtz_rhs(shape, seed=seed)
    ft, fo = prepare(f64, storage)
    u = torch.zeros(shape, dtype=TORCH[storage], device="cuda")
    fields = dict(tol=tol, boundary=slr.SLR_WRAP if wrap else slr.SLR_DIRICHLET, ghost=ghost, sigma=sigma, h=h,
                  **extra)
    if loop is not None:
        fields["loop"] = loop
    stencil = slr.SLR_J3D7 if len(shape) == 3 else slr.SLR_J2D5
    s = slr.Solver(stencil, u, ft.cuda(), **fields)
    s.run(max_iters)
    r = s.result()
    s.close()
    out = u.float().cpu().numpy() if storage in ("bf16", "f16") else u.cpu().numpy()
    fn = orc.j3d7 if len(shape) == 3 else orc.j2d5
    ref, rr = fn(np.zeros(shape, dtype=fo.dtype), fo, sigma=sigma, h=h, wrap=wrap, ghost=ghost, tol=tol,
                 max_iters=max_iters, storage=None if storage == "f64" else storage)
    assert r.iters == rr.iters and r.converged == rr.converged
    assert rel_err(out, ref) <= TOL[storage]
    assert np.array_equal(out.view(np.uint64 if out.dtype == np.float64 else np.uint32),
                          ref.view(np.uint64 if ref.dtype == np.float64 else np.uint32))
    assert r.value == rr.value
    return r


def test_helmholtz_256_fp64_to_1e6(gpu, orc):
    # the 2D Helmholtz configuration: 256 x 256 FP64, sigma 1, h = 1/257, tol 1e-6
    r = jacobi_case(gpu, orc, (256, 256))
    assert r.converged


def test_helmholtz_256_fp64_host_loop(gpu, orc):
    jacobi_case(gpu, orc, (256, 256), loop=gpu.SLR_LOOP_HOST)


@pytest.mark.parametrize("shape,kw", [
    ((33, 17), dict(tol=1e-9)),
    ((1, 1), dict(tol=1e-12)),
    ((1, 7), dict(tol=1e-12)),
    ((40, 1), dict(tol=1e-12)),
    ((48, 64), dict(wrap=True, tol=1e-9)),
    ((37, 29), dict(ghost=0.75, tol=1e-9)),
    ((64, 64), dict(sigma=0.0, tol=1e-8)),
    ((50, 90), dict(h=0.01, sigma=3.0, tol=1e-10)),
    ((1100, 300), dict(tol=0.0, max_iters=25)),
])
def test_fp64_edge_cases(gpu, orc, shape, kw):
    jacobi_case(gpu, orc, shape, **kw)


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("shape", [(96, 80), (17, 33)])
def test_storage_precisions(gpu, orc, storage, shape):
    jacobi_case(gpu, orc, shape, storage=storage, tol=1e-6, max_iters=3000)


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_j3d7(gpu, orc, storage):
    jacobi_case(gpu, orc, (12, 20, 24), storage=storage, tol=1e-6, max_iters=2000)


def test_j3d7_wrap_ragged(gpu, orc):
    jacobi_case(gpu, orc, (5, 9, 13), wrap=True, tol=1e-9)


def test_j3d7_host_loop(gpu, orc):
    jacobi_case(gpu, orc, (9, 10, 11), tol=1e-8, loop=gpu.SLR_LOOP_HOST)


def test_cap_and_resume(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    f = torch.from_numpy(inputs.helmholtz_rhs((128, 128), seed=4)).cuda()
    u = torch.zeros((128, 128), dtype=torch.float64, device="cuda")
    s = gpu.Solver(gpu.SLR_J2D5, u, f, tol=1e-7)
    s.run(10)
    r1 = s.result()
    assert r1.iters == 10 and not r1.converged and r1.status == gpu.SLR_NOT_CONVERGED
    s.run(3000)
    r2 = s.result()
    s.close()
    ref, rr = orc.j2d5(np.zeros((128, 128)), f.cpu().numpy(), tol=1e-7, max_iters=3000)
    assert (r2.iters, r2.converged, r2.value) == (rr.iters, rr.converged, rr.value)
    assert np.array_equal(u.cpu().numpy(), ref)


def test_wait_limit_reports_timeout_and_context_survives(gpu, orc):
    # one CTA leaves before the first grid barrier: every other CTA's bounded
    # wait runs out, the run reports SLR_ERR_TIMEOUT, and the next solve on a
    # fresh handle still works
    from paper_1609_04567_gb300 import inputs
    f = torch.from_numpy(inputs.helmholtz_rhs((64, 64), seed=2)).cuda()
    u = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    s = gpu.Solver(gpu.SLR_J2D5, u, f, wait_limit_ns=20_000_000, debug_flags=gpu.SLR_DEBUG_SKIP_ARRIVAL)
    s.run(100)
    st = s.result(check=False).status
    s.close()
    assert st == gpu.SLR_ERR_TIMEOUT
    jacobi_case(gpu, orc, (64, 64))


@pytest.mark.parametrize("d", [4.0 + (1.0 / 257) ** 2, 4.0 + (1.0 / 8193) ** 2, 4.0 + (1.0 / 65) ** 2,
                               6.0 + (1.0 / 513) ** 2, 4.0, 6.0, 3.0, 7.0, 0.1, 3.14159265, 1e-5, 12345.678])
def test_constant_division_matches_ieee(gpu, d):
    # the sweeps' a / d (reciprocal + two corrections) against the IEEE division:
    # every binary32 numerator, 2^26 binary64 numerators
    mismatches, checked = gpu.slr_check_exact_division(d)
    assert checked == [1 << 32, 1 << 26]
    assert mismatches == [0, 0]


# ---- TMA-staged sweeps (Dirichlet ghost +0, rows of whole 16-byte groups) ----
# forced with SLR_TILING_TMA on grids with ragged tiles in x (nx not a multiple
# of 256) and in y (ny not a multiple of the tile's rows), a fixed number of
# sweeps (tol 0), bit-exact against the oracle
@pytest.mark.parametrize("shape,storage", [((300, 520), "f32"), ((96, 1024), "f64"), ((70, 1040), "bf16"),
                                           ((33, 264), "f16"), ((9, 37, 264), "bf16"), ((17, 20, 256), "f32"),
                                           ((5, 9, 128), "f64"), ((4, 3, 520), "f16"), ((1, 1, 8), "bf16")])
def test_tma_path_bit_exact(gpu, orc, shape, storage):
    r = jacobi_case(gpu, orc, shape, storage=storage, tol=0.0, max_iters=23, tiling=gpu.SLR_TILING_TMA)
    assert r.iters == 23 and not r.converged


@pytest.mark.parametrize("kw", [dict(wrap=True), dict(ghost=0.25), dict(ghost=-0.0)])
def test_tma_request_falls_back_where_it_does_not_apply(gpu, orc, kw):
    jacobi_case(gpu, orc, (40, 512), storage="f32", tol=0.0, max_iters=9, tiling=gpu.SLR_TILING_TMA, **kw)


@pytest.mark.parametrize("tiling", [1, 2])
def test_tma_and_register_paths_agree_to_convergence(gpu, orc, tiling):
    # the FP32 form of the 256 x 256 Helmholtz problem, both staging choices
    r = jacobi_case(gpu, orc, (256, 256), storage="f32", tol=1e-6, tiling=tiling)
    assert r.converged


@pytest.mark.slow
def test_full_size_2d_f32_and_3d_bf16_default_path(gpu, orc):
    # the large single grids of the Jacobi bench, a few sweeps, library-chosen staging
    jacobi_case(gpu, orc, (8192, 8192), storage="f32", tol=0.0, max_iters=3)
    jacobi_case(gpu, orc, (512, 512, 512), storage="bf16", tol=0.0, max_iters=2)
