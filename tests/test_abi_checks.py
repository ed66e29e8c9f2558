"""Argument checks of the C ABI that run before any CUDA call.

Every call below is refused by the library's own validation, so nothing is
launched and no pointer is dereferenced (the pointers are made-up integers);
the tests need no GPU.  They pin the documented error behaviour of
include/slr.h: the status, and a message that names the problem."""
import ctypes

import pytest

FAKE_U, FAKE_AUX, FAKE_WS = 0x100000, 0x900000, 0x2000000


@pytest.fixture(scope="module")
def slr():
    from paper_1609_04567_gb300 import build, slr as binding
    build.build()
    binding.load()
    return binding


def test_detection_refuses_bad_arguments(slr):
    cases = [
        (dict(img=0), "device pointers"),
        (dict(nx=0), "[1, 2^31)"),
        (dict(wmax=4), "odd"),
        (dict(wmax=1), "odd"),
        (dict(wmax=17), "odd"),
        (dict(mask=FAKE_U + 100), "overlap"),                  # mask inside the image
        (dict(state=FAKE_AUX - 8), "overlap"),                 # state runs into the mask
        (dict(state=FAKE_WS + 2), "4-byte aligned"),
        (dict(ny=65536 * 8 + 1), "rows"),                      # more row blocks than a grid holds
    ]
    for change, words in cases:
        a = dict(img=FAKE_U, mask=FAKE_AUX, state=FAKE_WS, nx=64, ny=64, wmax=7)
        a.update(change)
        if "ny" in change:
            a.update(nx=1, mask=FAKE_U + (1 << 24), state=FAKE_U + (1 << 26))
        with pytest.raises(slr.SlrError) as e:
            slr.slr_detect_noise(a["img"], a["mask"], a["state"], a["nx"], a["ny"], a["wmax"])
        assert e.value.status == slr.SLR_ERR_INVALID_ARG, change
        assert words in slr.slr_last_error(None), (change, slr.slr_last_error(None))


def test_sobel_refuses_bad_arguments(slr):
    for img, out, nx, ny, words in [(0, FAKE_AUX, 64, 64, "device pointers"),
                                    (FAKE_U, 0, 64, 64, "device pointers"),
                                    (FAKE_U, FAKE_AUX, 0, 64, "[1, 2^31 - 4096)"),
                                    (FAKE_U, FAKE_AUX, 64, -1, "[1, 2^31 - 4096)"),
                                    (FAKE_U, FAKE_U + 63, 64, 64, "overlap")]:
        with pytest.raises(slr.SlrError) as e:
            slr.slr_sobel(img, out, nx, ny)
        assert e.value.status == slr.SLR_ERR_INVALID_ARG
        assert words in slr.slr_last_error(None)


def test_state_to_frame_refuses_bad_arguments(slr):
    for state, img, n in [(0, FAKE_AUX, 16), (FAKE_U, 0, 16), (FAKE_U + 2, FAKE_AUX, 16), (FAKE_U, FAKE_AUX, -1)]:
        with pytest.raises(slr.SlrError) as e:
            slr.slr_state_to_frame(state, img, n)
        assert e.value.status == slr.SLR_ERR_INVALID_ARG
    # an empty state is a no-op: nothing is enqueued
    assert slr.slr_state_to_frame(FAKE_U, FAKE_AUX, 0) == slr.SLR_OK


def test_static_solve_refuses_what_its_array_cannot_hold(slr):
    # 1024 x 1024 binary64 is 8 MiB of state; the static array holds 4 MiB
    d = slr.slr_desc_init(slr.SLR_J2D5, 1024, 1024, 1)
    st, *_ = slr.slr_run_static(d, FAKE_U, FAKE_AUX, 10, 0, check=False)
    assert st == slr.SLR_ERR_INVALID_ARG
    msg = slr.slr_static_last_error()
    assert "SLR_STATIC_STATE_BYTES" in msg and str(slr.SLR_STATIC_STATE_BYTES) in msg
    # 724 x 724 binary64 = 4,193,408 bytes fits; 725 x 724 does not
    assert 724 * 724 * 8 <= slr.SLR_STATIC_STATE_BYTES < 725 * 724 * 8
    d = slr.slr_desc_init(slr.SLR_J2D5, 724, 725, 1)
    st, *_ = slr.slr_run_static(d, FAKE_U, FAKE_AUX, 10, 0, check=False)
    assert st == slr.SLR_ERR_INVALID_ARG
    # other stencils, defect correction, a misaligned u, no f, a negative cap
    for stencil, change in [(slr.SLR_LIFE, {}), (slr.SLR_RESTORE8, {}),
                            (slr.SLR_J2D5, dict(defect_correction=1)), (slr.SLR_J2D5, dict(loop=slr.SLR_LOOP_HOST))]:
        d = slr.slr_desc_init(stencil, 64, 64, 1, **change)
        st, *_ = slr.slr_run_static(d, FAKE_U, FAKE_AUX, 10, 0, check=False)
        assert st == slr.SLR_ERR_UNSUPPORTED, (stencil, change)
    d = slr.slr_desc_init(slr.SLR_J2D5, 64, 64, 1)
    for u, f, cap in [(FAKE_U + 8, FAKE_AUX, 10), (FAKE_U, 0, 10), (FAKE_U, FAKE_AUX, -1)]:
        st, *_ = slr.slr_run_static(d, u, f, cap, 0, check=False)
        assert st == slr.SLR_ERR_INVALID_ARG, (u, f, cap)


def test_batch_sizes_and_create_checks(slr):
    assert slr.slr_batch_workspace_size(0) == 0
    assert slr.slr_batch_workspace_size(1025) == 0
    assert slr.slr_batch_workspace_size(1) > 0
    assert slr.slr_batch_workspace_size(1024) >= slr.slr_batch_workspace_size(512) >= slr.slr_batch_workspace_size(1)
    assert slr.slr_batch_workspace_size(7) % 256 == 0
    # the scratch of an instance is its second state buffer, rounded to 256 bytes
    d = slr.slr_desc_init(slr.SLR_J2D5, 100, 30, 1)
    assert slr.slr_batch_scratch_size(d) == -(-100 * 30 * 8 // 256) * 256
    assert slr.slr_batch_scratch_size(slr.slr_desc_init(slr.SLR_LIFE, 64, 64, 1)) == 0
    assert slr.slr_batch_scratch_size(slr.slr_desc_init(slr.SLR_J2D5, 0, 64, 1)) == 0
    need = slr.slr_batch_workspace_size(8)
    for n, ws, nbytes, status in [(0, FAKE_WS, need, slr.SLR_ERR_INVALID_ARG),
                                  (1025, FAKE_WS, 1 << 30, slr.SLR_ERR_INVALID_ARG),
                                  (8, FAKE_WS + 16, need, slr.SLR_ERR_INVALID_ARG),
                                  (8, 0, need, slr.SLR_ERR_INVALID_ARG),
                                  (8, FAKE_WS, need - 1, slr.SLR_ERR_WORKSPACE)]:
        with pytest.raises(slr.SlrError) as e:
            slr.slr_batch_create(n, ws, nbytes, 0)
        assert e.value.status == status, (n, ws, nbytes)


def _user_desc(slr, **change):
    d = slr.slr_user_desc()
    d.dtype, d.boundary, d.nx, d.ny, d.tol = slr.SLR_F32, slr.SLR_DIRICHLET, 64, 32, 1e-6
    d.reduce, d.loop = slr.SLR_USER_MAX, slr.SLR_LOOP_AUTO
    for k, v in change.items():
        setattr(d, k, v)
    return d


def test_user_descriptor_checks(slr):
    lib = slr.load()
    size = lambda d: int(lib.slr_user_workspace_size(ctypes.byref(d)))
    base = size(_user_desc(slr))
    assert base > 0 and base % 256 == 0
    assert size(_user_desc(slr, dtype=slr.SLR_F64)) > base        # twice the state bytes
    for change in [dict(dtype=slr.SLR_BF16), dict(dtype=slr.SLR_U8), dict(nx=0), dict(ny=-3),
                   dict(nx=1 << 21, ny=1 << 20), dict(boundary=2), dict(reduce=2), dict(loop=3)]:
        assert size(_user_desc(slr, **change)) == 0, change
    src = b"__device__ slr_t slr_update(const slr_nbr &u, slr_t f, long long i, long long j, const double *p)" \
          b"{ return u(0, 0); }\n__device__ double slr_delta(slr_t a, slr_t b) { return 0.0; }\n"
    h = ctypes.c_void_p()
    d = _user_desc(slr)
    cases = [(src, FAKE_U, FAKE_WS, base, slr.SLR_ERR_INVALID_ARG, "source"),           # NULL source below
             (src, FAKE_U + 2, FAKE_WS, base, slr.SLR_ERR_INVALID_ARG, "aligned"),
             (src, FAKE_U, FAKE_WS + 64, base, slr.SLR_ERR_INVALID_ARG, "256-byte"),
             (src, FAKE_U, FAKE_WS, base - 1, slr.SLR_ERR_WORKSPACE, "workspace")]
    for i, (s, u, ws, nbytes, status, words) in enumerate(cases):
        st = lib.slr_user_create(ctypes.byref(d), None if i == 0 else s, u, None, ws, nbytes, None,
                                 ctypes.byref(h))
        assert st == status, words
        assert words in lib.slr_user_last_error(None).decode(), words
        assert not h.value
    bad = _user_desc(slr, dtype=slr.SLR_U8)
    assert lib.slr_user_create(ctypes.byref(bad), src, FAKE_U, None, FAKE_WS, 1 << 20, None,
                               ctypes.byref(h)) == slr.SLR_ERR_INVALID_ARG
    assert "dtype" in lib.slr_user_last_error(None).decode()


NAN = float("nan")


@pytest.mark.parametrize("stencil,ext,fields,unsupported,words", [
    (9, (8, 8, 1), {}, False, "unknown stencil"),
    ("J2D5", (0, 8, 1), {}, False, "extents must be >= 1"),
    ("J2D5", (8, -1, 1), {}, False, "extents must be >= 1"),
    ("J3D7", (8, 8, (1 << 31) - 4095), {}, False, "extent too large"),
    ("J2D5", (8, 8, 2), {}, False, "nz == 1"),
    ("LIFE", (8, 8, 3), {}, False, "nz == 1"),
    ("J2D5", (8, 8, 1), dict(boundary=2), False, "unknown boundary"),
    ("J2D5", (8, 8, 1), dict(reduce=2), False, "reduce operator"),
    ("RESTORE8", (8, 8, 1), dict(reduce=0), False, "reduce operator"),
    ("J2D5", (8, 8, 1), dict(loop=3), False, "loop mode"),
    ("J2D5", (8, 8, 1), dict(math=2), False, "math mode"),
    ("LIFE", (8, 8, 1), dict(temporal_k=33), False, "temporal_k"),
    ("LIFE", (8, 8, 1), dict(temporal_k=-1), False, "temporal_k"),
    ("J2D5", (8, 8, 1), dict(grid_ctas=-2), False, "grid_ctas"),
    ("J2D5", (8, 8, 1), dict(tiling=-1), False, "tiling"),
    ("J2D5", (8, 8, 1), dict(storage=0), False, "Jacobi storage"),
    ("J3D7", (8, 8, 8), dict(sigma=NAN), False, "NaN"),
    ("J2D5", (8, 8, 1), dict(h=NAN), False, "NaN"),
    ("LIFE", (8, 8, 1), dict(storage=3), False, "Life storage"),
    ("RESTORE8", (8, 8, 1), dict(storage=4), False, "restoration storage"),
    ("RESTORE8", (8, 8, 1), dict(boundary=1), True, "DIRICHLET"),
    ("RESTORE8", (8, 8, 1), dict(alpha=0.0), False, "alpha"),
    ("RESTORE8", (8, 8, 1), dict(alpha=NAN), False, "alpha"),
    ("J2D5", (8, 8, 1), dict(defect_correction=1, storage=3), True, "defect correction"),
    ("J2D5", (8, 8, 1), dict(defect_correction=1, ghost=1.0), True, "defect correction"),
    ("J2D5", (8, 8, 1), dict(defect_correction=1, boundary=1), True, "defect correction"),
    ("J2D5", (8, 8, 1), dict(defect_correction=1, loop=1), True, "defect correction"),
    ("J3D7", (8, 8, 8), dict(defect_correction=1, storage=3), True, "defect correction"),
    ("LIFE", (64, 8, 1), dict(defect_correction=1), True, "defect correction"),
    ("J2D5", (8, 8, 1), dict(defect_correction=1, inner_sweeps=-1), False, "inner_sweeps"),
    ("J3D7", (8192, 8192, 1024), {}, False, "larger than device memory"),
])
def test_descriptor_rules(slr, stencil, ext, fields, unsupported, words):
    # each rule of the descriptor check: slr_workspace_size returns 0 and
    # slr_create refuses before it touches the device, with the status the
    # header documents and a message that names the rule
    s = getattr(slr, "SLR_" + stencil) if isinstance(stencil, str) else stencil
    d = slr.slr_desc_init(s if isinstance(stencil, str) else slr.SLR_J2D5, *ext, **fields)
    d.stencil = s
    assert slr.slr_workspace_size(d) == 0
    with pytest.raises(slr.SlrError) as e:
        slr.slr_create(d, FAKE_U, FAKE_AUX, FAKE_WS, 1 << 40, 0)
    assert e.value.status == (slr.SLR_ERR_UNSUPPORTED if unsupported else slr.SLR_ERR_INVALID_ARG)
    assert words in slr.slr_last_error(None), slr.slr_last_error(None)


def test_defaults_of_every_stencil_pass_the_rules(slr):
    for s, ext in ((slr.SLR_J2D5, (8, 8, 1)), (slr.SLR_J3D7, (8, 8, 8)), (slr.SLR_LIFE, (8, 8, 1)),
                   (slr.SLR_RESTORE8, (8, 8, 1))):
        assert slr.slr_workspace_size(slr.slr_desc_init(s, *ext)) > 0
    # and the defect correction's own defaults
    assert slr.slr_workspace_size(slr.slr_desc_init(slr.SLR_J2D5, 8, 8, 1, defect_correction=1)) > 0
    # 3D: the binary64 state buffer plus three binary32 buffers (r32, two e) of 6 x 7 x 8 cells
    plain3 = slr.slr_workspace_size(slr.slr_desc_init(slr.SLR_J3D7, 8, 7, 6))
    assert slr.slr_workspace_size(slr.slr_desc_init(slr.SLR_J3D7, 8, 7, 6, defect_correction=1)) == \
        plain3 + 3 * (-(-6 * 7 * 8 * 4 // 256) * 256)


def test_block_sweep_refuses_bad_ranges_before_any_device_work(slr):
    d = slr.slr_desc_init(slr.SLR_J2D5, 16, 32, 1)
    P = FAKE_WS + 4096
    cases = [
        (slr.slr_block(10, 5, 0, 10, 0, 10), "outside the block"),      # global row 4 is above row 0
        (slr.slr_block(10, 0, 0, 10, 0, 10), "outside the block"),      # global row 10 is below row 9
        (slr.slr_block(10, 0, 3, 2, 3, 2), "lo <= own_lo"),
        (slr.slr_block(10, 0, 0, 11, 0, 10), "lo <= own_lo"),
        (slr.slr_block(10, 0, 1, 9, 0, 9), "lo <= own_lo"),
        (slr.slr_block(0, 0, 0, 0, 0, 0), "rows >= 1"),
    ]
    for blk, words in cases:
        assert slr.slr_block_sweep(d, blk, FAKE_U, FAKE_U + 8192, FAKE_AUX, P, 0, check=False) == \
            slr.SLR_ERR_INVALID_ARG, words
        assert words in slr.slr_last_error(None), (words, slr.slr_last_error(None))
    good = slr.slr_block(10, 3, 1, 9, 1, 9)
    assert slr.slr_block_sweep(d, good, FAKE_U, FAKE_U, FAKE_AUX, P, 0, check=False) == slr.SLR_ERR_INVALID_ARG
    assert slr.slr_block_sweep(d, good, FAKE_U, FAKE_U + 8192, 0, P, 0, check=False) == slr.SLR_ERR_INVALID_ARG
    dc = slr.slr_desc_init(slr.SLR_J2D5, 16, 32, 1, defect_correction=1)
    assert slr.slr_block_sweep(dc, good, FAKE_U, FAKE_U + 8192, FAKE_AUX, P, 0, check=False) == \
        slr.SLR_ERR_UNSUPPORTED
