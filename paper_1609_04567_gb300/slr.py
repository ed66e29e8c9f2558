"""Thin ctypes binding of libslr.so (include/slr.h), plus a torch-tensor wrapper.

The functions ``slr_*`` below carry the C names and only marshal arguments:
device pointers are passed as integers (``tensor.data_ptr()``), the stream as
``torch.cuda.Stream.cuda_stream``.  Every sweep, reduce and test runs in the
CUDA library; there is no CPU path.  If ``libslr.so`` is missing or cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libslr.so")

# enums of slr.h
SLR_OK, SLR_NOT_CONVERGED = 0, 1
SLR_ERR_INVALID_ARG, SLR_ERR_WORKSPACE, SLR_ERR_CUDA, SLR_ERR_TIMEOUT, SLR_ERR_UNSUPPORTED = -1, -2, -3, -4, -5
SLR_J2D5, SLR_J3D7, SLR_LIFE, SLR_RESTORE8 = 0, 1, 2, 3
SLR_DIRICHLET, SLR_WRAP = 0, 1
SLR_RED_MAX_ABS_DELTA, SLR_RED_MEAN_ABS_DELTA_MASKED, SLR_RED_LIVE_COUNT = 0, 1, 2
SLR_U8, SLR_BF16, SLR_F16, SLR_F32, SLR_F64 = 0, 1, 2, 3, 4
SLR_LOOP_AUTO, SLR_LOOP_HOST, SLR_LOOP_PERSISTENT = 0, 1, 2
SLR_MATH_EXACT, SLR_MATH_FAST = 0, 1
SLR_TILING_AUTO, SLR_TILING_NONE, SLR_TILING_TMA = 0, 1, 2
SLR_DEBUG_SKIP_ARRIVAL = 1

STATUS_NAMES = {0: "SLR_OK", 1: "SLR_NOT_CONVERGED", -1: "SLR_ERR_INVALID_ARG", -2: "SLR_ERR_WORKSPACE",
                -3: "SLR_ERR_CUDA", -4: "SLR_ERR_TIMEOUT", -5: "SLR_ERR_UNSUPPORTED"}


class slr_desc(ctypes.Structure):
    _fields_ = [
        ("stencil", ctypes.c_int32), ("storage", ctypes.c_int32), ("reduce", ctypes.c_int32),
        ("boundary", ctypes.c_int32),
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
        ("ghost", ctypes.c_double), ("tol", ctypes.c_double), ("sigma", ctypes.c_double),
        ("h", ctypes.c_double), ("alpha", ctypes.c_float),
        ("loop", ctypes.c_int32), ("math", ctypes.c_int32), ("temporal_k", ctypes.c_int32),
        ("wait_limit_ns", ctypes.c_int64), ("debug_flags", ctypes.c_int32),
        ("defect_correction", ctypes.c_int32), ("inner_sweeps", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
        ("tiling", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class slr_tune_result(ctypes.Structure):
    _fields_ = [
        ("loop", ctypes.c_int32), ("temporal_k", ctypes.c_int32), ("tiling", ctypes.c_int32),
        ("grid_ctas", ctypes.c_int32), ("trials", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("ms_per_iter", ctypes.c_double), ("default_ms_per_iter", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class slr_user_desc(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int32), ("boundary", ctypes.c_int32), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
        ("ghost", ctypes.c_double), ("tol", ctypes.c_double), ("reduce", ctypes.c_int32),
        ("loop", ctypes.c_int32), ("params", ctypes.c_double * 8),
    ]


SLR_USER_MAX, SLR_USER_SUM = 0, 1


class slr_block(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("row0", ctypes.c_int64), ("lo", ctypes.c_int64), ("hi", ctypes.c_int64),
                ("own_lo", ctypes.c_int64), ("own_hi", ctypes.c_int64)]


class slr_partial(ctypes.Structure):
    _fields_ = [("maxbits", ctypes.c_uint64), ("sum", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("changed", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

EXPORTS = ["slr_desc_init", "slr_workspace_size", "slr_create", "slr_run_until", "slr_reduce_value",
           "slr_destroy", "slr_last_error", "slr_version", "slr_run_static", "slr_static_last_error",
           "slr_batch_workspace_size", "slr_batch_scratch_size", "slr_batch_create", "slr_batch_add",
           "slr_batch_run", "slr_batch_poll", "slr_batch_result", "slr_batch_remove", "slr_batch_destroy",
           "slr_batch_last_error", "slr_tune_scratch_size", "slr_tune", "slr_tune_lookup", "slr_tune_clear",
           "slr_tune_last_error", "slr_check_exact_math", "slr_check_exact_division", "slr_detect_noise",
           "slr_state_to_frame", "slr_sobel", "slr_check_exact_isqrt", "slr_user_workspace_size",
           "slr_user_create", "slr_user_run_until", "slr_user_reduce_value", "slr_user_destroy",
           "slr_user_last_error", "slr_block_sweep", "slr_measure_logic_rate"]
SLR_STATIC_STATE_BYTES = 4 << 20

_lib = None


class SlrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libslr.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a)")
    import torch  # noqa: F401  -- loads the CUDA runtime the library shares with torch
    lib = ctypes.CDLL(path)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    D = ctypes.POINTER(slr_desc)
    lib.slr_desc_init.argtypes = [D, i32, i64, i64, i64]
    lib.slr_desc_init.restype = None
    lib.slr_workspace_size.argtypes = [D]
    lib.slr_workspace_size.restype = ctypes.c_size_t
    lib.slr_create.argtypes = [D, P, P, P, ctypes.c_size_t, P, ctypes.POINTER(P)]
    lib.slr_create.restype = i32
    lib.slr_run_until.argtypes = [P, i64]
    lib.slr_run_until.restype = i32
    lib.slr_reduce_value.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                     ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint64)]
    lib.slr_reduce_value.restype = i32
    lib.slr_destroy.argtypes = [P]
    lib.slr_destroy.restype = i32
    lib.slr_last_error.argtypes = [P]
    lib.slr_last_error.restype = ctypes.c_char_p
    lib.slr_version.argtypes = []
    lib.slr_version.restype = ctypes.c_char_p
    lib.slr_run_static.argtypes = [D, P, P, i64, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                   ctypes.POINTER(i32)]
    lib.slr_run_static.restype = i32
    lib.slr_static_last_error.argtypes = []
    lib.slr_static_last_error.restype = ctypes.c_char_p
    lib.slr_batch_workspace_size.argtypes = [i32]
    lib.slr_batch_workspace_size.restype = ctypes.c_size_t
    lib.slr_batch_scratch_size.argtypes = [D]
    lib.slr_batch_scratch_size.restype = ctypes.c_size_t
    lib.slr_batch_create.argtypes = [i32, P, ctypes.c_size_t, P, ctypes.POINTER(P)]
    lib.slr_batch_create.restype = i32
    lib.slr_batch_add.argtypes = [P, D, P, P, P, i64, ctypes.POINTER(i32)]
    lib.slr_batch_add.restype = i32
    lib.slr_batch_run.argtypes = [P, i64]
    lib.slr_batch_run.restype = i32
    lib.slr_batch_poll.argtypes = [P, ctypes.POINTER(i32), i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.slr_batch_poll.restype = i32
    lib.slr_batch_result.argtypes = [P, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                     ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint64)]
    lib.slr_batch_result.restype = i32
    lib.slr_batch_remove.argtypes = [P, i32]
    lib.slr_batch_remove.restype = i32
    lib.slr_batch_destroy.argtypes = [P]
    lib.slr_batch_destroy.restype = i32
    lib.slr_batch_last_error.argtypes = [P]
    lib.slr_batch_last_error.restype = ctypes.c_char_p
    R = ctypes.POINTER(slr_tune_result)
    lib.slr_tune_scratch_size.argtypes = [D]
    lib.slr_tune_scratch_size.restype = ctypes.c_size_t
    lib.slr_tune.argtypes = [D, P, P, P, ctypes.c_size_t, P, i64, R]
    lib.slr_tune.restype = i32
    lib.slr_tune_lookup.argtypes = [D, R]
    lib.slr_tune_lookup.restype = i32
    lib.slr_tune_clear.argtypes = []
    lib.slr_tune_clear.restype = None
    lib.slr_tune_last_error.argtypes = []
    lib.slr_tune_last_error.restype = ctypes.c_char_p
    lib.slr_check_exact_math.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), P]
    lib.slr_check_exact_math.restype = i32
    lib.slr_check_exact_division.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.POINTER(ctypes.c_uint64), P]
    lib.slr_check_exact_division.restype = i32
    lib.slr_detect_noise.argtypes = [P, P, P, i64, i64, i32, P]
    lib.slr_detect_noise.restype = i32
    lib.slr_state_to_frame.argtypes = [P, P, i64, P]
    lib.slr_state_to_frame.restype = i32
    lib.slr_sobel.argtypes = [P, P, i64, i64, P]
    lib.slr_sobel.restype = i32
    lib.slr_check_exact_isqrt.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), P]
    lib.slr_check_exact_isqrt.restype = i32
    UD = ctypes.POINTER(slr_user_desc)
    lib.slr_user_workspace_size.argtypes = [UD]
    lib.slr_user_workspace_size.restype = ctypes.c_size_t
    lib.slr_user_create.argtypes = [UD, ctypes.c_char_p, P, P, P, ctypes.c_size_t, P, ctypes.POINTER(P)]
    lib.slr_user_create.restype = i32
    lib.slr_user_run_until.argtypes = [P, i64]
    lib.slr_user_run_until.restype = i32
    lib.slr_user_reduce_value.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                          ctypes.POINTER(i32)]
    lib.slr_user_reduce_value.restype = i32
    lib.slr_user_destroy.argtypes = [P]
    lib.slr_user_destroy.restype = i32
    lib.slr_user_last_error.argtypes = [P]
    lib.slr_user_last_error.restype = ctypes.c_char_p
    lib.slr_block_sweep.argtypes = [D, ctypes.POINTER(slr_block), P, P, P, P, P]
    lib.slr_block_sweep.restype = i32
    lib.slr_measure_logic_rate.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), P]
    lib.slr_measure_logic_rate.restype = i32
    _lib = lib
    return lib


# ---- the C calls, one to one ----------------------------------------------

def slr_desc_init(stencil: int, nx: int, ny: int, nz: int = 1, **fields) -> slr_desc:
    d = slr_desc()
    load().slr_desc_init(ctypes.byref(d), stencil, nx, ny, nz)
    for k, v in fields.items():
        setattr(d, k, v)
    return d


def slr_workspace_size(d: slr_desc) -> int:
    return int(load().slr_workspace_size(ctypes.byref(d)))


def slr_create(d: slr_desc, u_ptr: int, aux_ptr: int, ws_ptr: int, ws_bytes: int, stream: int) -> int:
    h = ctypes.c_void_p()
    st = load().slr_create(ctypes.byref(d), u_ptr or None, aux_ptr or None, ws_ptr or None, ws_bytes,
                           stream or None, ctypes.byref(h))
    if st != SLR_OK:
        raise SlrError(st, slr_last_error(None))
    return h.value


def slr_run_until(h: int, max_iters: int) -> int:
    st = load().slr_run_until(h, max_iters)
    if st < 0:
        raise SlrError(st, slr_last_error(h))
    return st


def slr_reduce_value(h: int, check: bool = True):
    """Returns (status, value, iters, converged, count)."""
    v, it, c, n = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_uint64()
    st = load().slr_reduce_value(h, ctypes.byref(v), ctypes.byref(it), ctypes.byref(c), ctypes.byref(n))
    if check and st < 0:
        raise SlrError(st, slr_last_error(h))
    return st, v.value, it.value, bool(c.value), n.value


def slr_destroy(h: int) -> int:
    return load().slr_destroy(h)


def slr_last_error(h) -> str:
    return load().slr_last_error(h).decode()


def slr_version() -> str:
    return load().slr_version().decode()


def slr_measure_logic_rate(stream: int = 0):
    """Measured logic-pipe throughput: (thread logic operations per second, kernel ms)."""
    r, t = ctypes.c_double(), ctypes.c_double()
    st = load().slr_measure_logic_rate(ctypes.byref(r), ctypes.byref(t), stream or None)
    if st != SLR_OK:
        raise SlrError(st, "logic-rate kernel failed")
    return r.value, t.value


def slr_block_sweep(d: slr_desc, b: slr_block, src_ptr: int, dst_ptr: int, aux_ptr: int, partial_ptr: int,
                    stream: int, check: bool = True) -> int:
    """One sweep of a row block (device step of the 1:n split); the partial
    reduce goes to the device slr_partial at partial_ptr."""
    st = load().slr_block_sweep(ctypes.byref(d), ctypes.byref(b), src_ptr or None, dst_ptr or None, aux_ptr or None,
                                partial_ptr or None, stream or None)
    if check and st < 0:
        raise SlrError(st, slr_last_error(None))
    return st


def slr_run_static(d: slr_desc, u_ptr: int, f_ptr: int, max_iters: int, stream: int, check: bool = True):
    """The allocation-free Jacobi solve; returns (status, value, iters, converged)."""
    v, it, c = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int32()
    st = load().slr_run_static(ctypes.byref(d), u_ptr or None, f_ptr or None, max_iters, stream or None,
                               ctypes.byref(v), ctypes.byref(it), ctypes.byref(c))
    if check and st < 0:
        raise SlrError(st, slr_static_last_error())
    return st, v.value, it.value, bool(c.value)


def slr_static_last_error() -> str:
    return load().slr_static_last_error().decode()


def _bcheck(st: int, b) -> int:
    if st < 0:
        raise SlrError(st, load().slr_batch_last_error(b).decode())
    return st


def slr_batch_workspace_size(max_instances: int) -> int:
    return int(load().slr_batch_workspace_size(max_instances))


def slr_batch_scratch_size(d: slr_desc) -> int:
    return int(load().slr_batch_scratch_size(ctypes.byref(d)))


def slr_batch_create(max_instances: int, ws_ptr: int, ws_bytes: int, stream: int) -> int:
    h = ctypes.c_void_p()
    _bcheck(load().slr_batch_create(max_instances, ws_ptr or None, ws_bytes, stream or None, ctypes.byref(h)), None)
    return h.value


def slr_batch_add(b: int, d: slr_desc, u_ptr: int, aux_ptr: int, scratch_ptr: int, max_iters: int) -> int:
    slot = ctypes.c_int32()
    _bcheck(load().slr_batch_add(b, ctypes.byref(d), u_ptr or None, aux_ptr or None, scratch_ptr or None,
                                 max_iters, ctypes.byref(slot)), b)
    return slot.value


def slr_batch_run(b: int, sweeps: int) -> int:
    return _bcheck(load().slr_batch_run(b, sweeps), b)


def slr_batch_poll(b: int, max_finished: int = 4096):
    """Returns (finished slots, number still running)."""
    arr = (ctypes.c_int32 * max_finished)()
    nf, nr = ctypes.c_int32(), ctypes.c_int32()
    _bcheck(load().slr_batch_poll(b, arr, max_finished, ctypes.byref(nf), ctypes.byref(nr)), b)
    return [arr[i] for i in range(nf.value)], nr.value


def slr_batch_result(b: int, slot: int):
    """Returns (status, value, iters, converged, count)."""
    v, it, c, n = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_uint64()
    st = _bcheck(load().slr_batch_result(b, slot, ctypes.byref(v), ctypes.byref(it), ctypes.byref(c),
                                         ctypes.byref(n)), b)
    return st, v.value, it.value, bool(c.value), n.value


def slr_batch_remove(b: int, slot: int) -> int:
    return _bcheck(load().slr_batch_remove(b, slot), b)


def slr_batch_destroy(b: int) -> int:
    return load().slr_batch_destroy(b)


def slr_batch_last_error(b) -> str:
    return load().slr_batch_last_error(b).decode()


def slr_tune_scratch_size(d: slr_desc) -> int:
    return int(load().slr_tune_scratch_size(ctypes.byref(d)))


def slr_tune(d: slr_desc, u_ptr: int, aux_ptr: int, scratch_ptr: int, scratch_bytes: int, stream: int,
             trial_iters: int = 0) -> slr_tune_result:
    r = slr_tune_result()
    st = load().slr_tune(ctypes.byref(d), u_ptr or None, aux_ptr or None, scratch_ptr or None, scratch_bytes,
                         stream or None, trial_iters, ctypes.byref(r))
    if st != SLR_OK:
        raise SlrError(st, slr_tune_last_error())
    return r


def slr_tune_lookup(d: slr_desc):
    """The cached choice for d, or None."""
    r = slr_tune_result()
    return r if load().slr_tune_lookup(ctypes.byref(d), ctypes.byref(r)) else None


def slr_tune_clear() -> None:
    load().slr_tune_clear()


def slr_tune_last_error() -> str:
    return load().slr_tune_last_error().decode()


def slr_check_exact_math(stream: int = 0):
    """Returns (mismatches of the three checks, inputs checked)."""
    mm = (ctypes.c_uint64 * 3)()
    n = ctypes.c_uint64()
    st = load().slr_check_exact_math(mm, ctypes.byref(n), stream or None)
    if st != SLR_OK:
        raise SlrError(st, "exact-math self-check failed to run")
    return list(mm), n.value


def slr_check_exact_division(d: float, stream: int = 0):
    """Returns ([mismatches binary32, binary64], [numerators checked binary32, binary64])."""
    mm, n = (ctypes.c_uint64 * 2)(), (ctypes.c_uint64 * 2)()
    st = load().slr_check_exact_division(d, mm, n, stream or None)
    if st != SLR_OK:
        raise SlrError(st, "division self-check refused or failed")
    return list(mm), list(n)


def slr_detect_noise(img_ptr: int, mask_ptr: int, state_ptr: int, nx: int, ny: int, wmax: int = 7,
                     stream: int = 0) -> int:
    """Adaptive median noise detection of a device uint8 image into a device
    uint8 mask, and the image as binary32 into `state_ptr` unless 0 (enqueued
    on `stream`)."""
    st = load().slr_detect_noise(img_ptr or None, mask_ptr or None, state_ptr or None, nx, ny, wmax,
                                 stream or None)
    if st != SLR_OK:
        raise SlrError(st, slr_last_error(None))
    return st


def slr_state_to_frame(state_ptr: int, img_ptr: int, n: int, stream: int = 0) -> int:
    st = load().slr_state_to_frame(state_ptr or None, img_ptr or None, n, stream or None)
    if st != SLR_OK:
        raise SlrError(st, slr_last_error(None))
    return st


def slr_sobel(img_ptr: int, out_ptr: int, nx: int, ny: int, stream: int = 0) -> int:
    st = load().slr_sobel(img_ptr or None, out_ptr or None, nx, ny, stream or None)
    if st != SLR_OK:
        raise SlrError(st, slr_last_error(None))
    return st


def sobel(img, out=None, *, stream=None):
    """Sobel edge magnitude (Sec. 4.2) of a uint8 CUDA image tensor."""
    import torch
    if not img.is_cuda or img.dtype != torch.uint8 or img.dim() != 2 or not img.is_contiguous():
        raise ValueError("img must be a contiguous 2D uint8 CUDA tensor")
    if out is None:
        out = torch.empty_like(img)
    st = stream if stream is not None else torch.cuda.current_stream(img.device)
    ny, nx = img.shape
    slr_sobel(img.data_ptr(), out.data_ptr(), nx, ny, st.cuda_stream)
    return out


def detect_noise(img, mask=None, state=None, *, wmax: int = 7, stream=None):
    """The noisy-pixel mask of a uint8 CUDA image tensor (the detection phase
    of the two-phase restoration); `mask` (uint8, same shape) is filled and
    returned, allocated when None; `state` (float32, same shape), when given,
    receives the image as the restoration's initial state."""
    import torch
    if not img.is_cuda or img.dtype != torch.uint8 or img.dim() != 2 or not img.is_contiguous():
        raise ValueError("img must be a contiguous 2D uint8 CUDA tensor")
    if mask is None:
        mask = torch.empty_like(img)
    if state is not None and (state.dtype != torch.float32 or state.shape != img.shape or not state.is_contiguous()):
        raise ValueError("state must be a contiguous float32 tensor shaped like img")
    st = stream if stream is not None else torch.cuda.current_stream(img.device)
    ny, nx = img.shape
    slr_detect_noise(img.data_ptr(), mask.data_ptr(), state.data_ptr() if state is not None else 0, nx, ny, wmax,
                     st.cuda_stream)
    return mask


def state_to_frame(state, img=None, *, stream=None):
    """A restored float32 CUDA state as a uint8 frame (nearest, ties to even,
    clamped to [0, 255])."""
    import torch
    if not state.is_cuda or state.dtype != torch.float32 or not state.is_contiguous():
        raise ValueError("state must be a contiguous float32 CUDA tensor")
    if img is None:
        img = torch.empty(state.shape, dtype=torch.uint8, device=state.device)
    st = stream if stream is not None else torch.cuda.current_stream(state.device)
    slr_state_to_frame(state.data_ptr(), img.data_ptr(), state.numel(), st.cuda_stream)
    return img


def slr_check_exact_isqrt(stream: int = 0):
    """Returns (mismatches, values checked) of the Sobel magnitude's integer square root."""
    mm, n = ctypes.c_uint64(), ctypes.c_uint64()
    st = load().slr_check_exact_isqrt(ctypes.byref(mm), ctypes.byref(n), stream or None)
    if st != SLR_OK:
        raise SlrError(st, "integer square root self-check failed")
    return mm.value, n.value


class UserSolver:
    """A loop-of-stencil-reduce over elemental functions given as CUDA C++
    source (compiled at run time; see slr_user_create in slr.h):
    ``slr_update(u, aux, i, j, p)`` gives an item's new value from its
    neighbours ``u(di, dj)``, ``slr_delta(new, old)`` its contribution to the
    reduce (``reduce`` "max" or "sum"), the loop stops when the reduced value
    is below ``tol``.  ``u`` (float32 or float64, 2D, contiguous CUDA) is
    updated in place; ``aux`` (same dtype and shape) or None."""

    def __init__(self, source: str, u, aux=None, *, params=(), boundary: int = 0, ghost: float = 0.0,
                 reduce: str = "max", tol: float = 1e-6, loop: int = 0, stream=None):
        import torch
        if not u.is_cuda or u.dim() != 2 or not u.is_contiguous() or u.dtype not in (torch.float32, torch.float64):
            raise ValueError("u must be a contiguous 2D float32 or float64 CUDA tensor")
        if aux is not None and (aux.dtype != u.dtype or aux.shape != u.shape or not aux.is_contiguous()):
            raise ValueError("aux must match u's dtype and shape")
        if len(params) > 8:
            raise ValueError("at most 8 params")
        d = slr_user_desc()
        d.dtype = SLR_F32 if u.dtype == torch.float32 else SLR_F64
        d.boundary, d.ny, d.nx = boundary, u.shape[0], u.shape[1]
        d.ghost, d.tol = ghost, tol
        d.reduce = {"max": SLR_USER_MAX, "sum": SLR_USER_SUM}[reduce]
        d.loop = loop
        for k, v in enumerate(params):
            d.params[k] = v
        self.desc = d
        self.stream = stream if stream is not None else torch.cuda.current_stream(u.device)
        lib = load()
        ws = lib.slr_user_workspace_size(ctypes.byref(d))
        if ws == 0:
            raise SlrError(SLR_ERR_INVALID_ARG, "invalid user descriptor")
        self.ws = torch.empty(ws + 256, dtype=torch.uint8, device=u.device)
        off = (-self.ws.data_ptr()) % 256
        self.u, self.aux = u, aux
        h = ctypes.c_void_p()
        st = lib.slr_user_create(ctypes.byref(d), source.encode(), u.data_ptr(),
                                 aux.data_ptr() if aux is not None else None, self.ws.data_ptr() + off, ws,
                                 self.stream.cuda_stream, ctypes.byref(h))
        if st != SLR_OK:
            raise SlrError(st, lib.slr_user_last_error(None).decode())
        self.handle = h.value

    def run(self, max_iters: int) -> int:
        lib = load()
        st = lib.slr_user_run_until(self.handle, max_iters)
        if st < 0:
            raise SlrError(st, lib.slr_user_last_error(self.handle).decode())
        return st

    def result(self):
        """(value, iters, converged) of the last iteration."""
        v, it, c = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int32()
        load().slr_user_reduce_value(self.handle, ctypes.byref(v), ctypes.byref(it), ctypes.byref(c))
        return v.value, it.value, bool(c.value)

    def close(self):
        if getattr(self, "handle", None):
            load().slr_user_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune(stencil: int, u, aux=None, *, stream=None, trial_iters: int = 0, **fields) -> dict:
    """Autotune the launch choices for a problem shaped like ``u`` on its
    own data (u and aux are only read); later Solvers of the same shape pick
    the choice up.  Returns the choice as a dict."""
    import torch
    shape = tuple(u.shape)
    nz, ny, nx = (1,) * (3 - len(shape)) + shape
    d = slr_desc_init(stencil, nx, ny, nz, storage=storage_of(u.dtype), **fields)
    stream = stream if stream is not None else torch.cuda.current_stream(u.device)
    nbytes = slr_tune_scratch_size(d)
    if nbytes == 0:
        slr_tune(d, u.data_ptr(), aux.data_ptr() if aux is not None else 0, 0, 0, stream.cuda_stream)
        raise SlrError(SLR_ERR_INVALID_ARG, "invalid descriptor")
    scratch = torch.empty(nbytes + 256, dtype=torch.uint8, device=u.device)
    off = (-scratch.data_ptr()) % 256
    r = slr_tune(d, u.data_ptr(), aux.data_ptr() if aux is not None else 0, scratch.data_ptr() + off, nbytes,
                 stream.cuda_stream, trial_iters)
    return r.as_dict()


class Batch:
    """A resident batch of instances over torch tensors (the library's
    batched persistent launch).  ``add`` allocates the instance's scratch with
    torch and keeps references until ``remove``."""

    def __init__(self, max_instances: int, *, device=None, stream=None):
        import torch
        self.device = torch.device(device or "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ws = slr_batch_workspace_size(max_instances)
        if ws == 0:
            raise SlrError(SLR_ERR_INVALID_ARG, "max_instances out of range")
        self.ws = torch.empty(ws + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.handle = slr_batch_create(max_instances, self.ws.data_ptr() + off, ws, self.stream.cuda_stream)
        self.held = {}

    def add(self, stencil: int, u, aux, max_iters: int, **fields) -> int:
        import torch
        shape = tuple(u.shape)
        nz, ny, nx = (1,) * (3 - len(shape)) + shape
        d = slr_desc_init(stencil, nx, ny, nz, storage=storage_of(u.dtype), **fields)
        nbytes = slr_batch_scratch_size(d)
        if nbytes == 0:
            raise SlrError(SLR_ERR_INVALID_ARG, "descriptor not accepted for batches")
        scratch = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        slot = slr_batch_add(self.handle, d, u.data_ptr(), aux.data_ptr(), scratch.data_ptr(), max_iters)
        self.held[slot] = (u, aux, scratch)
        return slot

    def run(self, sweeps: int) -> None:
        slr_batch_run(self.handle, sweeps)

    def poll(self):
        return slr_batch_poll(self.handle)

    def result(self, slot: int) -> Result:
        return Result(*slr_batch_result(self.handle, slot))

    def remove(self, slot: int) -> None:
        slr_batch_remove(self.handle, slot)
        self.held.pop(slot, None)

    def close(self) -> None:
        if getattr(self, "handle", None):
            slr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- torch wrapper ----------------------------------------------------------

@dataclass
class Result:
    status: int
    value: float
    iters: int
    converged: bool
    count: int


_TORCH_STORAGE = None


def storage_of(dtype) -> int:
    import torch
    global _TORCH_STORAGE
    if _TORCH_STORAGE is None:
        _TORCH_STORAGE = {torch.uint8: SLR_U8, torch.bfloat16: SLR_BF16, torch.float16: SLR_F16,
                          torch.float32: SLR_F32, torch.float64: SLR_F64}
    return _TORCH_STORAGE[dtype]


class Solver:
    """One loop-of-stencil-reduce instance over caller-owned torch tensors.

    ``u`` (state, in/out) and ``aux`` (f or mask) are CUDA tensors; the
    workspace is allocated here with torch (the library itself never
    allocates).  ``run(max_iters)`` enqueues the loop on ``stream``;
    ``result()`` waits and reads the reduced value."""

    def __init__(self, stencil: int, u, aux=None, *, stream=None, **fields):
        import torch
        if not u.is_cuda or not u.is_contiguous():
            raise ValueError("u must be a contiguous CUDA tensor")
        shape = tuple(u.shape)
        nz, ny, nx = (1,) * (3 - len(shape)) + shape
        self.desc = slr_desc_init(stencil, nx, ny, nz, storage=storage_of(u.dtype), **fields)
        self.stream = stream if stream is not None else torch.cuda.current_stream(u.device)
        ws = slr_workspace_size(self.desc)
        if ws == 0:
            # the library's own checks name the problem (invalid or unsupported)
            slr_create(self.desc, u.data_ptr(), aux.data_ptr() if aux is not None else 0, 0, 0,
                       self.stream.cuda_stream)
            raise SlrError(SLR_ERR_INVALID_ARG, "invalid descriptor")
        self.ws = torch.empty(ws + 256, dtype=torch.uint8, device=u.device)
        off = (-self.ws.data_ptr()) % 256
        self.u, self.aux = u, aux
        self.handle = slr_create(self.desc, u.data_ptr(), aux.data_ptr() if aux is not None else 0,
                                 self.ws.data_ptr() + off, ws, self.stream.cuda_stream)

    def run(self, max_iters: int) -> int:
        return slr_run_until(self.handle, max_iters)

    def result(self, check: bool = True) -> Result:
        return Result(*slr_reduce_value(self.handle, check))

    def close(self):
        if getattr(self, "handle", None):
            slr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
