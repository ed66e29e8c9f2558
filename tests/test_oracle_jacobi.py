"""Pins for the oracle's Helmholtz Jacobi solvers (Sec. 4.1 problem, Sec. 3.1 loop).

Nothing here compares the oracle with a retyped copy of itself.  The pins are:
  * discrete sine modes, eigenfunctions of the 5-point (7-point) operator with
    zero Dirichlet ghosts: from u0 = 0 the n-th Jacobi iterate is exactly
    c*(1 - mu^n) v, so the state, the reduced max|change| and the iteration
    count at which the repeat-until test first passes are all closed forms;
  * brute force: the converged loop equals a dense linear solve of the
    discrete system (numpy.linalg.solve) on tiny grids, for Dirichlet ghosts
    of any value, wrap-around and non-square grids;
  * the storage-precision paths: one sweep equals the FP32 sweep rounded by
    torch/numpy's own conversions; every stored value is representable;
  * defect correction: converges to the dense solution to its tolerance.
"""
import math

import numpy as np
import pytest


def sine_mode_2d(n, p, q):
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    return np.outer(np.sin(q * math.pi * x), np.sin(p * math.pi * x)), h


def jacobi_factor(h, sigma, modes):
    """mu and c* of a sine mode: neighbour sum of the mode is 2*sum(cos(p pi h)) v."""
    dim = len(modes)
    d = 2 * dim + sigma * h * h
    mu = 2.0 * sum(math.cos(m * math.pi * h) for m in modes) / d
    lam = (4.0 / (h * h)) * sum(math.sin(m * math.pi * h / 2) ** 2 for m in modes)
    cstar = 1.0 / (lam + sigma)
    return mu, cstar


def predicted_iters(cstar, mu, vmax, tol, cap):
    for n in range(1, cap + 1):
        if abs(cstar) * mu ** (n - 1) * (1 - mu) * vmax < tol:
            return n
    return cap


@pytest.mark.parametrize("n,p,q,sigma", [(31, 1, 1, 1.0), (31, 1, 2, 0.0), (24, 3, 1, 5.0)])
def test_j2d5_sine_mode_closed_form(orc, n, p, q, sigma):
    v, h = sine_mode_2d(n, p, q)
    mu, cstar = jacobi_factor(h, sigma, (p, q))
    for sweeps in (1, 2, 7, 40):
        u, r = orc.j2d5(np.zeros_like(v), v, sigma=sigma, tol=0.0, max_iters=sweeps)
        assert r.iters == sweeps and not r.converged
        expect = cstar * (1 - mu ** sweeps) * v
        assert np.max(np.abs(u - expect)) <= 1e-13 * abs(cstar)
        dmax = abs(cstar) * mu ** (sweeps - 1) * (1 - mu) * np.max(np.abs(v))
        assert r.value == pytest.approx(dmax, rel=1e-9, abs=1e-16)


@pytest.mark.parametrize("tol", [1e-6, 3e-7, 1e-9])
def test_j2d5_iteration_count_closed_form(orc, tol):
    n, p, q, sigma = 31, 1, 1, 1.0
    v, h = sine_mode_2d(n, p, q)
    mu, cstar = jacobi_factor(h, sigma, (p, q))
    expect_n = predicted_iters(cstar, mu, np.max(np.abs(v)), tol, 5000)
    u, r = orc.j2d5(np.zeros_like(v), v, sigma=sigma, tol=tol, max_iters=5000)
    assert r.converged and r.iters == expect_n
    # repeat-until: the test fails one sweep earlier
    u2, r2 = orc.j2d5(np.zeros_like(v), v, sigma=sigma, tol=tol, max_iters=expect_n - 1)
    assert not r2.converged and r2.value >= tol


def test_j2d5_cap_stops_loop(orc):
    v, _ = sine_mode_2d(16, 1, 1)
    _, r = orc.j2d5(np.zeros_like(v), v, tol=1e-30, max_iters=3)
    assert r.iters == 3 and not r.converged


def dense_helmholtz(ny, nx, h, sigma, wrap, ghost, f, dim_d=4.0):
    """Dense matrix of (d u - sum nbrs)/h^2 with the boundary moved to the RHS."""
    n = nx * ny
    A = np.zeros((n, n))
    b = f.reshape(-1).astype(np.float64).copy()
    d = dim_d + sigma * h * h
    for i in range(ny):
        for j in range(nx):
            r = i * nx + j
            A[r, r] += d / (h * h)
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                y, x = i + di, j + dj
                if wrap:
                    A[r, (y % ny) * nx + (x % nx)] -= 1.0 / (h * h)
                elif 0 <= y < ny and 0 <= x < nx:
                    A[r, y * nx + x] -= 1.0 / (h * h)
                else:
                    b[r] += ghost / (h * h)
    return A, b


@pytest.mark.parametrize("ny,nx,h,wrap,ghost,sigma", [
    (8, 8, 0.0, False, 0.0, 1.0),
    (5, 9, 0.1, False, 0.0, 2.0),
    (6, 7, 0.125, True, 0.0, 1.0),
    (8, 8, 0.0, False, 0.75, 1.0),
])
def test_j2d5_brute_force_dense_solve(orc, ny, nx, h, wrap, ghost, sigma):
    from paper_1609_04567_gb300 import inputs
    f = inputs.helmholtz_rhs((ny, nx), seed=7)
    hh = h if h > 0 else 1.0 / (nx + 1)
    A, b = dense_helmholtz(ny, nx, hh, sigma, wrap, ghost, f)
    exact = np.linalg.solve(A, b).reshape(ny, nx)
    u, r = orc.j2d5(np.zeros((ny, nx)), f, sigma=sigma, h=h, wrap=wrap, ghost=ghost,
                    tol=1e-15, max_iters=200000)
    assert r.converged
    # stopping at max|change| < tol leaves an error of at most about
    # tol * rho / (1 - rho), rho the spectral radius of the Jacobi iteration
    jac = np.eye(A.shape[0]) - A / np.diag(A)[:, None]
    rho = np.max(np.abs(np.linalg.eigvals(jac)))
    bound = 2e-15 / (1 - rho) + 1e-13 * np.max(np.abs(exact))
    assert np.max(np.abs(u - exact)) <= bound


def test_j3d7_sine_mode_closed_form(orc):
    n, modes, sigma = 11, (1, 2, 1), 1.0
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    v = (np.sin(modes[2] * math.pi * x)[:, None, None] * np.sin(modes[1] * math.pi * x)[None, :, None]
         * np.sin(modes[0] * math.pi * x)[None, None, :])
    mu, cstar = jacobi_factor(h, sigma, modes)
    for sweeps in (1, 5, 30):
        u, r = orc.j3d7(np.zeros_like(v), v, sigma=sigma, tol=0.0, max_iters=sweeps)
        expect = cstar * (1 - mu ** sweeps) * v
        assert np.max(np.abs(u - expect)) <= 1e-13 * abs(cstar)
        dmax = abs(cstar) * mu ** (sweeps - 1) * (1 - mu) * np.max(np.abs(v))
        assert r.value == pytest.approx(dmax, rel=1e-9)
    expect_n = predicted_iters(cstar, mu, np.max(np.abs(v)), 1e-7, 5000)
    _, r = orc.j3d7(np.zeros_like(v), v, sigma=sigma, tol=1e-7, max_iters=5000)
    assert r.converged and r.iters == expect_n


@pytest.mark.parametrize("nz,ny,nx,h,wrap,ghost,sigma", [
    (3, 4, 5, 0.0, False, 0.0, 1.0),
    (4, 3, 5, 0.25, True, 0.0, 3.0),
    (3, 5, 4, 0.0, False, -0.5, 1.0),
    (5, 3, 3, 0.2, False, 1.25, 0.0),
])
def test_j3d7_brute_force_dense_solve(orc, nz, ny, nx, h, wrap, ghost, sigma):
    from paper_1609_04567_gb300 import inputs
    f = inputs.helmholtz_rhs((nz, ny, nx), seed=11)
    hh = h if h > 0 else 1.0 / (nx + 1)
    n = nx * ny * nz
    A = np.zeros((n, n))
    b = f.reshape(-1).copy()
    for k in range(nz):
        for i in range(ny):
            for j in range(nx):
                r = (k * ny + i) * nx + j
                A[r, r] += (6 + sigma * hh * hh) / (hh * hh)
                for dk, di, dj in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
                    z, y, x = k + dk, i + di, j + dj
                    if wrap:
                        A[r, ((z % nz) * ny + (y % ny)) * nx + (x % nx)] -= 1.0 / (hh * hh)
                    elif 0 <= z < nz and 0 <= y < ny and 0 <= x < nx:
                        A[r, (z * ny + y) * nx + x] -= 1.0 / (hh * hh)
                    else:
                        b[r] += ghost / (hh * hh)
    exact = np.linalg.solve(A, b).reshape(nz, ny, nx)
    u, r = orc.j3d7(np.zeros_like(f), f, sigma=sigma, h=h, wrap=wrap, ghost=ghost, tol=1e-15, max_iters=200000)
    assert r.converged
    jac = np.eye(n) - A / np.diag(A)[:, None]
    rho = np.max(np.abs(np.linalg.eigvals(jac)))
    bound = 2e-15 / (1 - rho) + 1e-13 * np.max(np.abs(exact))
    assert np.max(np.abs(u - exact)) <= bound


def test_j2d5_f32_closed_form(orc):
    n, p, q, sigma = 31, 1, 2, 1.0
    v, h = sine_mode_2d(n, p, q)
    mu, cstar = jacobi_factor(h, sigma, (p, q))
    v32 = v.astype(np.float32)
    u, r = orc.j2d5(np.zeros_like(v32), v32, sigma=sigma, tol=0.0, max_iters=50, storage="f32")
    expect = cstar * (1 - mu ** 50) * v
    assert np.max(np.abs(u - expect)) <= 1e-5 * abs(cstar)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_storage_path_one_sweep_is_rounded_f32_sweep(orc, storage):
    import torch
    from paper_1609_04567_gb300 import inputs
    f64 = inputs.helmholtz_rhs((20, 24), seed=3)
    tdt = torch.bfloat16 if storage == "bf16" else torch.float16
    f_s = torch.from_numpy(f64.astype(np.float32)).to(tdt).float().numpy()
    u0 = torch.from_numpy((0.01 * f64).astype(np.float32)).to(tdt).float().numpy()
    u32, _ = orc.j2d5(u0, f_s, tol=0.0, max_iters=1, storage="f32")
    us, _ = orc.j2d5(u0, f_s, tol=0.0, max_iters=1, storage=storage)
    lib_rounded = torch.from_numpy(u32).to(tdt).float().numpy()
    assert np.array_equal(us.view(np.uint32), lib_rounded.view(np.uint32))


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_storage_path_state_representable_and_bounded(orc, storage):
    import torch
    n = 31
    v, h = sine_mode_2d(n, 1, 1)
    mu, cstar = jacobi_factor(h, 1.0, (1, 1))
    tdt = torch.bfloat16 if storage == "bf16" else torch.float16
    f_s = torch.from_numpy(v.astype(np.float32)).to(tdt).float().numpy()
    u, r = orc.j2d5(np.zeros_like(f_s), f_s, tol=1e-6, max_iters=20000, storage=storage)
    again = torch.from_numpy(u).to(tdt).float().numpy()
    assert np.array_equal(u, again)                       # stored values are representable
    # the loop stops when no stored value moves by tol or more; the state is
    # then a fixed point of the rounded iteration, within the stagnation bound
    # (half an ulp of the state divided by the contraction gap 1 - mu) of c* v
    ulp = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}[storage] * np.max(np.abs(cstar * v))
    bound = ulp / (1 - mu) + 1e-3 * abs(cstar)
    assert r.converged
    assert np.max(np.abs(u - cstar * v)) <= bound


def test_defect_correction_reaches_dense_solution(orc):
    from paper_1609_04567_gb300 import inputs
    ny = nx = 12
    f = inputs.helmholtz_rhs((ny, nx), seed=5)
    h = 1.0 / (nx + 1)
    A, b = dense_helmholtz(ny, nx, h, 1.0, False, 0.0, f)
    exact = np.linalg.solve(A, b).reshape(ny, nx)
    u, r = orc.j2d5_dc(np.zeros((ny, nx)), f, tol=1e-10, k_in=20)
    assert r.converged and r.value < 1e-10
    assert orc.j2d5_scaled_defect(u, f) == pytest.approx(r.value, rel=0, abs=0)
    # the scaled defect bounds the error by rho / (1 - mu) for the slowest mode
    mu, _ = jacobi_factor(h, 1.0, (1, 1))
    assert np.max(np.abs(u - exact)) <= 1e-10 / (1 - mu) * 1.01


def test_scaled_defect_of_zero_state(orc):
    v, h = sine_mode_2d(9, 1, 1)
    d = 4 + h * h
    assert orc.j2d5_scaled_defect(np.zeros_like(v), v) == pytest.approx(h * h * np.max(np.abs(v)) / d, rel=1e-14)


def sine_mode_3d(n, modes):
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    v = (np.sin(modes[2] * math.pi * x)[:, None, None] * np.sin(modes[1] * math.pi * x)[None, :, None]
         * np.sin(modes[0] * math.pi * x)[None, None, :])
    return v, h


def test_j3d7_f32_closed_form(orc):
    n, modes, sigma = 13, (1, 1, 2), 1.0
    v, h = sine_mode_3d(n, modes)
    mu, cstar = jacobi_factor(h, sigma, modes)
    v32 = v.astype(np.float32)
    for sweeps in (1, 20, 60):
        u, r = orc.j3d7(np.zeros_like(v32), v32, sigma=sigma, tol=0.0, max_iters=sweeps, storage="f32")
        expect = cstar * (1 - mu ** sweeps) * v
        assert np.max(np.abs(u - expect)) <= 1e-5 * abs(cstar)
        dmax = abs(cstar) * mu ** (sweeps - 1) * (1 - mu) * np.max(np.abs(v))
        assert r.value == pytest.approx(dmax, rel=1e-3, abs=1e-6 * abs(cstar))


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_j3d7_storage_one_sweep_is_rounded_f32_sweep(orc, storage):
    import torch
    from paper_1609_04567_gb300 import inputs
    f64 = inputs.helmholtz_rhs((6, 7, 9), seed=4)
    tdt = torch.bfloat16 if storage == "bf16" else torch.float16
    f_s = torch.from_numpy(f64.astype(np.float32)).to(tdt).float().numpy()
    u0 = torch.from_numpy((0.01 * f64).astype(np.float32)).to(tdt).float().numpy()
    for wrap in (False, True):
        u32, _ = orc.j3d7(u0, f_s, wrap=wrap, tol=0.0, max_iters=1, storage="f32")
        us, r = orc.j3d7(u0, f_s, wrap=wrap, tol=0.0, max_iters=1, storage=storage)
        lib_rounded = torch.from_numpy(u32).to(tdt).float().numpy()
        assert np.array_equal(us.view(np.uint32), lib_rounded.view(np.uint32))
        # the change is taken between stored values
        assert r.value == float(np.max(np.abs(us - u0)))


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_j3d7_storage_state_representable_and_bounded(orc, storage):
    import torch
    n, modes = 11, (1, 1, 1)
    v, h = sine_mode_3d(n, modes)
    mu, cstar = jacobi_factor(h, 1.0, modes)
    tdt = torch.bfloat16 if storage == "bf16" else torch.float16
    f_s = torch.from_numpy(v.astype(np.float32)).to(tdt).float().numpy()
    u, r = orc.j3d7(np.zeros_like(f_s), f_s, tol=1e-6, max_iters=20000, storage=storage)
    assert np.array_equal(u, torch.from_numpy(u).to(tdt).float().numpy())
    ulp = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}[storage] * np.max(np.abs(cstar * v))
    assert r.converged
    assert np.max(np.abs(u - cstar * v)) <= ulp / (1 - mu) + 1e-3 * abs(cstar)


@pytest.mark.parametrize("dim,wrap,ghost", [(2, False, 0.5), (2, True, 0.0), (3, False, -0.25), (3, True, 0.0)])
def test_f32_paths_reach_the_dense_solution(orc, dim, wrap, ghost):
    # the binary32 loop, run to its stagnation level, against numpy's dense
    # solve of the same discrete system (built here from the operator's
    # definition): the error is bounded by a few binary32 roundings of the
    # state amplified by 1 / (1 - rho)
    from paper_1609_04567_gb300 import inputs
    shape = (7, 6) if dim == 2 else (4, 5, 6)
    sigma, h = 2.0, 0.2
    f = inputs.helmholtz_rhs(shape, seed=9)
    n = f.size
    offs = [(-1, 0), (1, 0), (0, -1), (0, 1)] if dim == 2 else \
        [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    A = np.zeros((n, n))
    b = f.reshape(-1).copy()
    for idx in np.ndindex(shape):
        r = np.ravel_multi_index(idx, shape)
        A[r, r] += (2 * dim + sigma * h * h) / (h * h)
        for o in offs:
            nb = tuple(i + d for i, d in zip(idx, o))
            if wrap:
                A[r, np.ravel_multi_index(tuple(c % s for c, s in zip(nb, shape)), shape)] -= 1.0 / (h * h)
            elif all(0 <= c < s for c, s in zip(nb, shape)):
                A[r, np.ravel_multi_index(nb, shape)] -= 1.0 / (h * h)
            else:
                b[r] += ghost / (h * h)
    exact = np.linalg.solve(A, b).reshape(shape)
    run = orc.j2d5 if dim == 2 else orc.j3d7
    f32 = f.astype(np.float32)
    u, r = run(np.zeros_like(f32), f32, sigma=sigma, h=h, wrap=wrap, ghost=ghost, tol=1e-7, max_iters=100000,
               storage="f32")
    jac = np.eye(n) - A / np.diag(A)[:, None]
    rho = np.max(np.abs(np.linalg.eigvals(jac)))
    scale = np.max(np.abs(exact))
    assert np.max(np.abs(u - exact)) <= (1e-7 + 8 * 2.0 ** -24 * scale) / (1 - rho) + 2e-7 * scale


def test_defect_correction_steps(orc):
    # The correction loop step by step against the oracle's binary32 Jacobi
    # path (pinned above) and the operator built from its definition:
    #   correction 1 from u = 0: r = f exactly, so u1 is K binary32 sweeps of
    #   A e = f from e = 0, widened to binary64 -- bit for bit;
    #   correction 2: u2 = u1 + K binary32 sweeps of A e = r1 from e = 0,
    #   r1 = f - A u1 in binary64 (numpy's order here: equal up to rounding).
    from paper_1609_04567_gb300 import inputs
    ny, nx, K = 10, 12, 7
    f = inputs.helmholtz_rhs((ny, nx), seed=8)
    z64, z32 = np.zeros((ny, nx)), np.zeros((ny, nx), dtype=np.float32)
    u1, r1 = orc.j2d5_dc(z64, f, tol=0.0, k_in=K, max_outer=1)
    s1, _ = orc.j2d5(z32, f.astype(np.float32), tol=0.0, max_iters=K, storage="f32")
    assert np.array_equal(u1, s1.astype(np.float64))
    assert r1.iters == 1 and not r1.converged
    assert r1.value == orc.j2d5_scaled_defect(u1, f)
    h = 1.0 / (nx + 1)
    A, b = dense_helmholtz(ny, nx, h, 1.0, False, 0.0, f)
    res1 = (b - A @ u1.reshape(-1)).reshape(ny, nx)
    e2, _ = orc.j2d5(z32, res1.astype(np.float32), tol=0.0, max_iters=K, storage="f32")
    u2, r2 = orc.j2d5_dc(z64, f, tol=0.0, k_in=K, max_outer=2)
    assert r2.iters == 2
    assert np.max(np.abs(u2 - (u1 + e2.astype(np.float64)))) <= 1e-6 * np.max(np.abs(e2))
    # the scaled defect it reports is the change the next FP64 Jacobi sweep makes
    nxt, rj = orc.j2d5(u2, f, tol=0.0, max_iters=1)
    assert r2.value == pytest.approx(rj.value, rel=1e-9)


def dense_helmholtz_3d(nz, ny, nx, h, sigma, f):
    """Dense matrix of the 3D operator ((6 + sigma h^2) u - sum of 6 nbrs) / h^2, ghost 0."""
    n = nx * ny * nz
    A = np.zeros((n, n))
    for k in range(nz):
        for i in range(ny):
            for j in range(nx):
                r = (k * ny + i) * nx + j
                A[r, r] += (6 + sigma * h * h) / (h * h)
                for dk, di, dj in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
                    z, y, x = k + dk, i + di, j + dj
                    if 0 <= z < nz and 0 <= y < ny and 0 <= x < nx:
                        A[r, (z * ny + y) * nx + x] -= 1.0 / (h * h)
    return A, f.reshape(-1).astype(np.float64).copy()


def test_defect_correction_3d_reaches_dense_solution(orc):
    from paper_1609_04567_gb300 import inputs
    nz, ny, nx = 5, 6, 7
    f = inputs.helmholtz_rhs((nz, ny, nx), seed=15)
    h = 1.0 / (nx + 1)
    A, b = dense_helmholtz_3d(nz, ny, nx, h, 1.0, f)
    exact = np.linalg.solve(A, b).reshape(nz, ny, nx)
    u, r = orc.j3d7_dc(np.zeros((nz, ny, nx)), f, tol=1e-10, k_in=15)
    assert r.converged and r.value < 1e-10
    assert orc.j3d7_scaled_defect(u, f) == r.value
    jac = np.eye(A.shape[0]) - A / np.diag(A)[:, None]
    rho = np.max(np.abs(np.linalg.eigvals(jac)))
    assert np.max(np.abs(u - exact)) <= 1e-10 / (1 - rho) * 1.01


def test_scaled_defect_3d_of_zero_state(orc):
    from paper_1609_04567_gb300 import inputs
    f = inputs.helmholtz_rhs((4, 5, 6), seed=2)
    h = 1.0 / 7
    d = 6 + h * h
    assert orc.j3d7_scaled_defect(np.zeros_like(f), f) == pytest.approx(h * h * np.max(np.abs(f)) / d, rel=1e-14)


def test_defect_correction_3d_steps(orc):
    # as the 2D steps: correction 1 from u = 0 is K binary32 3D sweeps of
    # A e = f, widened, bit for bit; correction 2 adds K sweeps of A e = r1;
    # the reported value is the change of the next FP64 3D Jacobi sweep
    from paper_1609_04567_gb300 import inputs
    nz, ny, nx, K = 4, 5, 6, 6
    f = inputs.helmholtz_rhs((nz, ny, nx), seed=9)
    z64, z32 = np.zeros((nz, ny, nx)), np.zeros((nz, ny, nx), dtype=np.float32)
    u1, r1 = orc.j3d7_dc(z64, f, tol=0.0, k_in=K, max_outer=1)
    s1, _ = orc.j3d7(z32, f.astype(np.float32), tol=0.0, max_iters=K, storage="f32")
    assert np.array_equal(u1, s1.astype(np.float64))
    assert r1.iters == 1 and r1.value == orc.j3d7_scaled_defect(u1, f)
    h = 1.0 / (nx + 1)
    A, b = dense_helmholtz_3d(nz, ny, nx, h, 1.0, f)
    res1 = (b - A @ u1.reshape(-1)).reshape(nz, ny, nx)
    e2, _ = orc.j3d7(z32, res1.astype(np.float32), tol=0.0, max_iters=K, storage="f32")
    u2, r2 = orc.j3d7_dc(z64, f, tol=0.0, k_in=K, max_outer=2)
    assert np.max(np.abs(u2 - (u1 + e2.astype(np.float64)))) <= 1e-6 * np.max(np.abs(e2))
    _, rj = orc.j3d7(u2, f, tol=0.0, max_iters=1)
    assert r2.value == pytest.approx(rj.value, rel=1e-9)
