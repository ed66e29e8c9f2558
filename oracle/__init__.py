"""Plain CPU oracle for the Loop-of-stencil-reduce hot path (arXiv 1609.04567).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only callers.
The CUDA library neither imports nor links anything from here, and this module
imports nothing from the CUDA package.

The arithmetic lives in ``slr_oracle.c`` (plain C, no fused multiply-add); this
module compiles it with gcc on first use and marshals numpy arrays through
ctypes.  Every function returns ``(state, Result)`` and never modifies its
inputs.

Parity status: every solver here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, known patterns, brute force, library
rounding); none is "parity unpinned".

Threads: the same C file also builds with ``-fopenmp`` (``liboracle_omp.so``),
which shares the rows of each sweep among host threads and leaves every value
unchanged (the reduces are a maximum, an integer sum and an or).  Inside
``with threads(n):`` the solvers run that build on n threads; outside it they
run the single-threaded build.  ``tests/test_oracle_threads.py`` checks that
both builds agree bit for bit.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_libs = {}
_omp_threads = 0          # > 0 inside `with threads(n)`: solvers use the OpenMP build

STORAGE = {"f32": 0, "bf16": 1, "f16": 2}


class _CResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("value", ctypes.c_double),
                ("converged", ctypes.c_int32), ("changed", ctypes.c_int32),
                ("count", ctypes.c_uint64)]


class _CBlock(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("row0", ctypes.c_int64), ("lo", ctypes.c_int64), ("hi", ctypes.c_int64),
                ("own_lo", ctypes.c_int64), ("own_hi", ctypes.c_int64)]


class _CPartial(ctypes.Structure):
    _fields_ = [("maxbits", ctypes.c_uint64), ("sum", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("changed", ctypes.c_uint64)]


@dataclass
class Result:
    iters: int
    value: float
    converged: bool
    changed: bool
    count: int


def build(force: bool = False) -> str:
    """Compile ``slr_oracle.c`` into ``liboracle.so`` next to it (gcc, -O2,
    -ffp-contract=off), and the threaded build ``liboracle_omp.so`` when gcc
    accepts -fopenmp.  Returns the path of the single-threaded object."""
    _compile(_LIB, [], force)
    try:
        _compile(_LIB_OMP, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass                                  # no OpenMP here: threads() runs one thread
    return _LIB


def _compile(lib: str, extra, force: bool) -> str:
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(_SRC):
        return lib
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-Wno-unknown-pragmas",
           "-fPIC", "-shared"] + list(extra) + ["-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd, stderr=subprocess.DEVNULL if extra else None)
    os.replace(tmp, lib)
    return lib


def omp_available() -> bool:
    """Whether the threaded build exists (gcc with -fopenmp)."""
    build()
    return os.path.exists(_LIB_OMP) and os.path.getmtime(_LIB_OMP) >= os.path.getmtime(_SRC)


@contextlib.contextmanager
def threads(n: int):
    """Run the solvers on n host threads (the OpenMP build) inside the block;
    yields the thread count actually used (1 without OpenMP)."""
    global _omp_threads
    saved = _omp_threads
    used = 1
    if n > 1 and omp_available():
        used = int(_load(True).orc_set_threads(int(n)))
        _omp_threads = used
    try:
        yield used
    finally:
        _omp_threads = saved


def _load(omp=None):
    if omp is None:
        omp = _omp_threads > 0
    if omp in _libs:
        return _libs[omp]
    build()
    lib = ctypes.CDLL(_LIB_OMP if omp else _LIB)
    P = ctypes.c_void_p
    i64, f64, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    R = ctypes.POINTER(_CResult)
    lib.orc_j2d5_f64.argtypes = [P, P, i64, i64, f64, f64, i32, f64, f64, i64, R]
    lib.orc_j2d5_f32.argtypes = [P, P, i64, i64, f64, f64, i32, ctypes.c_float, i32, f64, i64, R]
    lib.orc_j3d7_f64.argtypes = [P, P, i64, i64, i64, f64, f64, i32, f64, f64, i64, R]
    lib.orc_j3d7_f32.argtypes = [P, P, i64, i64, i64, f64, f64, i32, ctypes.c_float, i32, f64, i64, R]
    lib.orc_life.argtypes = [P, i64, i64, i32, i64, R]
    lib.orc_restore8.argtypes = [P, P, i64, i64, ctypes.c_float, f64, i64, R]
    lib.orc_j2d5_dc.argtypes = [P, P, i64, i64, f64, f64, f64, i64, i64, R]
    lib.orc_amf_detect.argtypes = [P, P, i64, i64, i32]
    lib.orc_amf_detect.restype = i32
    lib.orc_sobel.argtypes = [P, P, i64, i64]
    lib.orc_sobel.restype = i32
    lib.orc_j2d5_scaled_defect.argtypes = [P, P, i64, i64, f64, f64]
    lib.orc_j2d5_scaled_defect.restype = f64
    lib.orc_j3d7_dc.argtypes = [P, P, i64, i64, i64, f64, f64, f64, i64, i64, R]
    lib.orc_j3d7_dc.restype = i32
    lib.orc_j3d7_scaled_defect.argtypes = [P, P, i64, i64, i64, f64, f64]
    lib.orc_j3d7_scaled_defect.restype = f64
    for name in ("orc_j2d5_f64", "orc_j2d5_f32", "orc_j3d7_f64", "orc_j3d7_f32",
                 "orc_life", "orc_restore8", "orc_j2d5_dc"):
        getattr(lib, name).restype = i32
    lib.orc_f32_to_bf16.argtypes = [ctypes.c_float]
    lib.orc_f32_to_bf16.restype = ctypes.c_uint16
    lib.orc_f32_to_f16.argtypes = [ctypes.c_float]
    lib.orc_f32_to_f16.restype = ctypes.c_uint16
    lib.orc_round_storage.argtypes = [ctypes.c_float, i32]
    lib.orc_round_storage.restype = ctypes.c_float
    for name in ("orc_f32_to_bf16_array", "orc_f32_to_f16_array", "orc_f16_to_f32_array"):
        getattr(lib, name).argtypes = [P, P, i64]
        getattr(lib, name).restype = None
    lib.orc_round_storage_array.argtypes = [P, P, i64, i32]
    lib.orc_round_storage_array.restype = None
    lib.orc_set_threads.argtypes = [i32]
    lib.orc_set_threads.restype = i32
    B, PT = ctypes.POINTER(_CBlock), ctypes.POINTER(_CPartial)
    f32 = ctypes.c_float
    lib.orc_j2d5_block_f64.argtypes = [P, P, P, i64, i64, B, f64, f64, i32, f64, PT]
    lib.orc_j2d5_block_f32.argtypes = [P, P, P, i64, i64, B, f64, f64, i32, f32, i32, PT]
    lib.orc_j3d7_block_f64.argtypes = [P, P, P, i64, i64, i64, B, f64, f64, i32, f64, PT]
    lib.orc_j3d7_block_f32.argtypes = [P, P, P, i64, i64, i64, B, f64, f64, i32, f32, i32, PT]
    lib.orc_life_block.argtypes = [P, P, i64, i64, B, i32, PT]
    lib.orc_restore8_block.argtypes = [P, P, P, i64, i64, B, f32, PT]
    for name in ("orc_j2d5_block_f64", "orc_j2d5_block_f32", "orc_j3d7_block_f64", "orc_j3d7_block_f32",
                 "orc_life_block", "orc_restore8_block"):
        getattr(lib, name).restype = i32
    _libs[omp] = lib
    return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _res(r: _CResult) -> Result:
    return Result(int(r.iters), float(r.value), bool(r.converged), bool(r.changed), int(r.count))


def _check(rc: int, name: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {name} failed with code {rc}")


def j2d5(u0, f, *, sigma=1.0, h=0.0, wrap=False, ghost=0.0, tol=1e-6, max_iters=5000,
         storage=None):
    """2D 5-point Helmholtz Jacobi loop (Sec. 4.1 solver, Sec. 3.1 loop).

    ``storage=None`` runs in FP64 on float64 arrays; ``storage`` in
    {"f32","bf16","f16"} runs FP32 arithmetic with the state rounded to that
    precision after every update (arrays given as float32 holding values
    representable in the storage precision)."""
    lib = _load()
    r = _CResult()
    if storage is None:
        u = np.array(u0, dtype=np.float64, order="C", copy=True)
        ff = np.ascontiguousarray(f, dtype=np.float64)
        ny, nx = u.shape
        _check(lib.orc_j2d5_f64(_ptr(u), _ptr(ff), nx, ny, sigma, h, int(wrap), ghost,
                                tol, max_iters, ctypes.byref(r)), "j2d5_f64")
    else:
        u = np.array(u0, dtype=np.float32, order="C", copy=True)
        ff = np.ascontiguousarray(f, dtype=np.float32)
        ny, nx = u.shape
        _check(lib.orc_j2d5_f32(_ptr(u), _ptr(ff), nx, ny, sigma, h, int(wrap), ghost,
                                STORAGE[storage], tol, max_iters, ctypes.byref(r)), "j2d5_f32")
    return u, _res(r)


def j3d7(u0, f, *, sigma=1.0, h=0.0, wrap=False, ghost=0.0, tol=1e-6, max_iters=5000,
         storage=None):
    """3D 7-point Helmholtz Jacobi loop; arrays are (nz, ny, nx), x contiguous."""
    lib = _load()
    r = _CResult()
    if storage is None:
        u = np.array(u0, dtype=np.float64, order="C", copy=True)
        ff = np.ascontiguousarray(f, dtype=np.float64)
        nz, ny, nx = u.shape
        _check(lib.orc_j3d7_f64(_ptr(u), _ptr(ff), nx, ny, nz, sigma, h, int(wrap), ghost,
                                tol, max_iters, ctypes.byref(r)), "j3d7_f64")
    else:
        u = np.array(u0, dtype=np.float32, order="C", copy=True)
        ff = np.ascontiguousarray(f, dtype=np.float32)
        nz, ny, nx = u.shape
        _check(lib.orc_j3d7_f32(_ptr(u), _ptr(ff), nx, ny, nz, sigma, h, int(wrap), ghost,
                                STORAGE[storage], tol, max_iters, ctypes.byref(r)), "j3d7_f32")
    return u, _res(r)


def life(cells, *, wrap=True, max_gens=2000):
    """Game of Life B3/S23 loop (Fig. 1 elemental function); uint8 cells."""
    lib = _load()
    r = _CResult()
    a = np.array(cells, dtype=np.uint8, order="C", copy=True)
    ny, nx = a.shape
    _check(lib.orc_life(_ptr(a), nx, ny, int(wrap), max_gens, ctypes.byref(r)), "life")
    return a, _res(r)


def restore8(u0, mask, *, alpha=100.0, tol=1e-3, max_iters=5000):
    """Restoration loop of the Sec. 4.3 denoiser on float32 state and a uint8
    noisy-pixel mask."""
    lib = _load()
    r = _CResult()
    u = np.array(u0, dtype=np.float32, order="C", copy=True)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    ny, nx = u.shape
    _check(lib.orc_restore8(_ptr(u), _ptr(m), nx, ny, alpha, tol, max_iters,
                            ctypes.byref(r)), "restore8")
    return u, _res(r)


def amf_detect(img, *, wmax=7) -> np.ndarray:
    """Adaptive median noise detector (the detection phase of the Sec. 4.3
    denoiser) on a uint8 image: a uint8 mask, 1 where the filter with windows
    3 x 3 .. wmax x wmax replaces the pixel."""
    lib = _load()
    a = np.ascontiguousarray(img, dtype=np.uint8)
    ny, nx = a.shape
    m = np.zeros((ny, nx), dtype=np.uint8)
    _check(lib.orc_amf_detect(_ptr(a), _ptr(m), nx, ny, int(wmax)), "amf_detect")
    return m


def sobel(img) -> np.ndarray:
    """Sobel edge magnitude (Sec. 4.2) of a uint8 image: min(255,
    floor(sqrt(Gx^2 + Gy^2))) inside, 0 on the border."""
    lib = _load()
    a = np.ascontiguousarray(img, dtype=np.uint8)
    ny, nx = a.shape
    out = np.zeros((ny, nx), dtype=np.uint8)
    _check(lib.orc_sobel(_ptr(a), _ptr(out), nx, ny), "sobel")
    return out


def j2d5_dc(u0, f, *, sigma=1.0, h=0.0, tol=1e-10, k_in=50, max_outer=100000):
    """FP64 defect correction with FP32 Jacobi inner solves (ghost 0)."""
    lib = _load()
    r = _CResult()
    u = np.array(u0, dtype=np.float64, order="C", copy=True)
    ff = np.ascontiguousarray(f, dtype=np.float64)
    ny, nx = u.shape
    _check(lib.orc_j2d5_dc(_ptr(u), _ptr(ff), nx, ny, sigma, h, tol, k_in, max_outer,
                           ctypes.byref(r)), "j2d5_dc")
    return u, _res(r)


def j3d7_dc(u0, f, *, sigma=1.0, h=0.0, tol=1e-10, k_in=50, max_outer=100000):
    """FP64 defect correction with FP32 Jacobi inner solves, 3D 7-point
    operator (ghost 0); arrays are (nz, ny, nx)."""
    lib = _load()
    r = _CResult()
    u = np.array(u0, dtype=np.float64, order="C", copy=True)
    ff = np.ascontiguousarray(f, dtype=np.float64)
    nz, ny, nx = u.shape
    _check(lib.orc_j3d7_dc(_ptr(u), _ptr(ff), nx, ny, nz, sigma, h, tol, k_in, max_outer, ctypes.byref(r)),
           "j3d7_dc")
    return u, _res(r)


def j3d7_scaled_defect(u, f, *, sigma=1.0, h=0.0) -> float:
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64)
    ff = np.ascontiguousarray(f, dtype=np.float64)
    nz, ny, nx = uu.shape
    return float(lib.orc_j3d7_scaled_defect(_ptr(uu), _ptr(ff), nx, ny, nz, sigma, h))


def j2d5_scaled_defect(u, f, *, sigma=1.0, h=0.0) -> float:
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64)
    ff = np.ascontiguousarray(f, dtype=np.float64)
    ny, nx = uu.shape
    return float(lib.orc_j2d5_scaled_defect(_ptr(uu), _ptr(ff), nx, ny, sigma, h))


def f32_to_bf16_bits(x: float) -> int:
    return int(_load().orc_f32_to_bf16(ctypes.c_float(x)))


def f32_to_f16_bits(x: float) -> int:
    return int(_load().orc_f32_to_f16(ctypes.c_float(x)))


def round_storage(a, storage: str) -> np.ndarray:
    """Round a float32 array to the storage precision and back with the
    oracle's own bit-level routine (round to nearest even)."""
    lib = _load()
    x = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty_like(x)
    lib.orc_round_storage_array(_ptr(x), _ptr(out), x.size, STORAGE[storage])
    return out


def f32_to_bf16_array(a) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    lib.orc_f32_to_bf16_array(_ptr(x), _ptr(out), x.size)
    return out


def f32_to_f16_array(a) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    lib.orc_f32_to_f16_array(_ptr(x), _ptr(out), x.size)
    return out


def f16_bits_to_f32_array(a) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(a, dtype=np.uint16)
    out = np.empty(x.shape, dtype=np.float32)
    lib.orc_f16_to_f32_array(_ptr(x), _ptr(out), x.size)
    return out


def block_sweep(stencil: str, src, dst, aux, *, rows: int, row0: int, lo: int, hi: int, own_lo: int, own_hi: int,
                nx: int, ny: int, nz: int = 1, sigma=1.0, h=0.0, wrap=False, ghost=0.0, storage=None,
                alpha=100.0):
    """One sweep of a row block (3D: a slab of z-planes) of a larger grid:
    rows [lo, hi) of the block array dst receive the update of src, the
    change is reduced over rows [own_lo, own_hi); block row r is grid row
    row0 + r.  src, dst, aux are C-ordered numpy arrays of the block
    (rows x nx, or rows x ny x nx); nx, ny (nz) are the grid's extents.
    ``stencil`` is "j2d5", "j3d7", "life" or "restore8".  Returns a dict with
    maxbits, sum, count and changed."""
    lib = _load()
    b = _CBlock(rows, row0, lo, hi, own_lo, own_hi)
    out = _CPartial()

    def P(a):
        return None if a is None else _ptr(a)
    if stencil == "j2d5":
        if storage is None:
            rc = lib.orc_j2d5_block_f64(P(src), P(dst), P(aux), nx, ny, ctypes.byref(b), sigma, h, int(wrap), ghost,
                                        ctypes.byref(out))
        else:
            rc = lib.orc_j2d5_block_f32(P(src), P(dst), P(aux), nx, ny, ctypes.byref(b), sigma, h, int(wrap), ghost,
                                        STORAGE[storage], ctypes.byref(out))
    elif stencil == "j3d7":
        if storage is None:
            rc = lib.orc_j3d7_block_f64(P(src), P(dst), P(aux), nx, ny, nz, ctypes.byref(b), sigma, h, int(wrap),
                                        ghost, ctypes.byref(out))
        else:
            rc = lib.orc_j3d7_block_f32(P(src), P(dst), P(aux), nx, ny, nz, ctypes.byref(b), sigma, h, int(wrap),
                                        ghost, STORAGE[storage], ctypes.byref(out))
    elif stencil == "life":
        rc = lib.orc_life_block(P(src), P(dst), nx, ny, ctypes.byref(b), int(wrap), ctypes.byref(out))
    elif stencil == "restore8":
        rc = lib.orc_restore8_block(P(src), P(dst), P(aux), nx, ny, ctypes.byref(b), alpha, ctypes.byref(out))
    else:
        raise ValueError(stencil)
    _check(rc, "block_sweep")
    return {"maxbits": int(out.maxbits), "sum": int(out.sum), "count": int(out.count), "changed": int(out.changed)}
