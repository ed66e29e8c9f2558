"""Elemental functions written by the user (the pattern's API of Sec. 3.2,
Fig. 1), compiled at run time: the Helmholtz Jacobi and Life written as user
functions must reproduce the oracle bit for bit (state, value, iterations);
source errors come back with the compiler's log."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

JACOBI = """
__device__ slr_t slr_update(const slr_nbr &u, slr_t f, long long i, long long j, const double *p)
{
    const slr_t s = ((u(-1, 0) + u(1, 0)) + u(0, -1)) + u(0, 1);
    return ((slr_t)p[0] * f + s) / (slr_t)p[1];
}
__device__ double slr_delta(slr_t a, slr_t b) { return (double)fabs(a - b); }
"""

LIFE = """
__device__ slr_t slr_update(const slr_nbr &u, slr_t, long long, long long, const double *)
{
    const slr_t n = u(-1, -1) + u(-1, 0) + u(-1, 1) + u(0, -1) + u(0, 1) + u(1, -1) + u(1, 0) + u(1, 1);
    return (n == 3 || (u(0, 0) == 1 && n == 2)) ? 1 : 0;
}
__device__ double slr_delta(slr_t a, slr_t b) { return a != b ? 1.0 : 0.0; }
"""


def jacobi_constants(nx, sigma=1.0, h=0.0):
    hh = h if h > 0 else 1.0 / (nx + 1)
    h2 = hh * hh
    return h2, 4.0 + sigma * h2


@pytest.mark.parametrize("dtype,wrap,shape", [("f32", False, (48, 64)), ("f32", False, (37, 21)),
                                              ("f64", True, (30, 40)), ("f64", False, (64, 64))])
def test_jacobi_as_user_functions(gpu, orc, dtype, wrap, shape):
    from paper_1609_04567_gb300 import inputs
    f64 = inputs.helmholtz_rhs(shape, seed=6)
    h2, d = jacobi_constants(shape[1])
    if dtype == "f32":
        f = f64.astype(np.float32)
        params = (float(np.float32(h2)), float(np.float32(d)))
        tdt = torch.float32
    else:
        f, params, tdt = f64, (h2, d), torch.float64
    u = torch.zeros(shape, dtype=tdt, device="cuda")
    s = gpu.UserSolver(JACOBI, u, torch.from_numpy(f).cuda(), params=params, boundary=int(wrap), tol=1e-6)
    s.run(5000)
    value, iters, conv = s.result()
    s.close()
    ref, rr = orc.j2d5(np.zeros(shape, dtype=f.dtype), f, wrap=wrap, tol=1e-6, max_iters=5000,
                       storage="f32" if dtype == "f32" else None)
    assert (iters, conv, value) == (rr.iters, rr.converged, rr.value)
    view = np.uint32 if dtype == "f32" else np.uint64
    assert np.array_equal(u.cpu().numpy().view(view), ref.view(view))


def test_life_as_user_functions(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    cells = inputs.life_cells(40, 56, seed=12)
    u = torch.from_numpy(cells.astype(np.float32)).cuda()
    s = gpu.UserSolver(LIFE, u, boundary=1, reduce="sum", tol=0.5)
    s.run(400)
    value, iters, conv = s.result()
    s.close()
    ref, rr = orc.life(cells, wrap=True, max_gens=400)
    assert (iters, conv) == (rr.iters, rr.converged)
    assert np.array_equal(u.cpu().numpy().astype(np.uint8), ref)


def test_resume_and_cached_program(gpu, orc):
    from paper_1609_04567_gb300 import inputs
    f = inputs.helmholtz_rhs((32, 32), seed=2)
    h2, d = jacobi_constants(32)
    u = torch.zeros((32, 32), dtype=torch.float64, device="cuda")
    s = gpu.UserSolver(JACOBI, u, torch.from_numpy(f).cuda(), params=(h2, d), tol=1e-9)
    s.run(7)
    assert s.result()[1] == 7
    s.run(100000)
    value, iters, conv = s.result()
    s.close()
    ref, rr = orc.j2d5(np.zeros((32, 32)), f, tol=1e-9, max_iters=100000)
    assert (iters, value) == (rr.iters, rr.value) and np.array_equal(u.cpu().numpy(), ref)


def test_compile_errors_report_the_log(gpu):
    u = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.SlrError, match="does not compile") as e:
        gpu.UserSolver("__device__ slr_t slr_update(const slr_nbr &u) { return undefined_name; }", u)
    assert "undefined_name" in str(e.value)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_device_and_host_loops_agree(gpu, orc, dtype):
    # the cooperative loop and the host-driven loop give the same state, value
    # and count (max reduce: Jacobi; sum reduce: Life)
    from paper_1609_04567_gb300 import inputs
    f64 = inputs.helmholtz_rhs((70, 90), seed=9)
    h2, d = jacobi_constants(90)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    f = torch.from_numpy(f64).to(tdt).cuda()
    params = (float(np.float32(h2)), float(np.float32(d))) if dtype == "f32" else (h2, d)
    out = []
    for loop in (gpu.SLR_LOOP_PERSISTENT, gpu.SLR_LOOP_HOST):
        u = torch.zeros((70, 90), dtype=tdt, device="cuda")
        s = gpu.UserSolver(JACOBI, u, f, params=params, tol=1e-6, loop=loop)
        s.run(5000)
        out.append((s.result(), u.cpu().numpy()))
        s.close()
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])
    cells = inputs.life_cells(33, 47, seed=4).astype(np.float32)
    res = []
    for loop in (gpu.SLR_LOOP_PERSISTENT, gpu.SLR_LOOP_HOST):
        u = torch.from_numpy(cells).cuda()
        s = gpu.UserSolver(LIFE, u, boundary=1, reduce="sum", tol=0.5, loop=loop)
        s.run(300)
        res.append((s.result(), u.cpu().numpy()))
        s.close()
    assert res[0][0] == res[1][0] and np.array_equal(res[0][1], res[1][1])
