"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/slr.h declares; the binding mirrors the descriptor layout.  No GPU
needed: nothing here launches a kernel."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(slr_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1609_04567_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "slr_create" in names and "slr_run_until" in names
    assert "slr_reduce_value" in names and "slr_destroy" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_declared_functions():
    from paper_1609_04567_gb300 import slr
    assert sorted(slr.EXPORTS) == sorted(n for n in declared_functions() if n in slr.EXPORTS)
    for n in declared_functions():
        assert n in slr.EXPORTS, f"binding lacks {n}"


def test_desc_layout_and_defaults(lib):
    from paper_1609_04567_gb300 import slr
    slr.load()
    d = slr.slr_desc_init(slr.SLR_J2D5, 256, 256, 1)
    assert d.reduce == slr.SLR_RED_MAX_ABS_DELTA and d.storage == slr.SLR_F64
    assert d.tol == 1e-6 and d.sigma == 1.0 and d.boundary == slr.SLR_DIRICHLET
    d = slr.slr_desc_init(slr.SLR_LIFE, 64, 32, 1)
    assert d.boundary == slr.SLR_WRAP and d.storage == slr.SLR_U8
    d = slr.slr_desc_init(slr.SLR_RESTORE8, 64, 32, 1)
    assert d.storage == slr.SLR_F32 and d.alpha == pytest.approx(100.0) and d.tol == 1e-3
    assert d.reduce == slr.SLR_RED_MEAN_ABS_DELTA_MASKED


def test_workspace_size_and_validation(lib):
    from paper_1609_04567_gb300 import slr
    d = slr.slr_desc_init(slr.SLR_LIFE, 8192, 8192, 1)
    ws = slr.slr_workspace_size(d)
    assert ws >= 8192 * 8192 and ws % 256 == 0
    bad = slr.slr_desc_init(slr.SLR_LIFE, 0, 8, 1)
    assert slr.slr_workspace_size(bad) == 0
    bad = slr.slr_desc_init(slr.SLR_J2D5, 8, 8, 2)          # 2D stencil with nz > 1
    assert slr.slr_workspace_size(bad) == 0
    bad = slr.slr_desc_init(slr.SLR_J2D5, 8, 8, 1, reduce=slr.SLR_RED_LIVE_COUNT)
    assert slr.slr_workspace_size(bad) == 0


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    from paper_1609_04567_gb300 import slr
    d = slr.slr_desc_init(slr.SLR_J2D5, 8, 8, 1)
    with pytest.raises(slr.SlrError) as e:
        slr.slr_create(d, 0x1000, 0x2000, 0x3000, 0, 0)      # workspace too small
    assert e.value.status == slr.SLR_ERR_WORKSPACE
    with pytest.raises(slr.SlrError) as e:
        slr.slr_create(d, 0x1001, 0x2000, 0x3000, 1 << 20, 0)  # misaligned u
    assert e.value.status == slr.SLR_ERR_INVALID_ARG
    with pytest.raises(slr.SlrError) as e:
        slr.slr_create(d, 0x1000, 0, 0x3000, 1 << 20, 0)      # Jacobi needs f
    assert e.value.status == slr.SLR_ERR_INVALID_ARG
    r = slr.slr_desc_init(slr.SLR_RESTORE8, 8, 8, 1, boundary=slr.SLR_WRAP)
    with pytest.raises(slr.SlrError) as e:
        slr.slr_create(r, 0x1000, 0x2000, 0x3000, 1 << 20, 0)
    assert e.value.status == slr.SLR_ERR_UNSUPPORTED
    assert "restoration" in slr.slr_last_error(None)


def test_version_names_the_architecture(lib):
    from paper_1609_04567_gb300 import slr
    assert "sm_103a" in slr.slr_version()


def _c_layout(struct, fields, tmp_path):
    """sizeof and field offsets of a C struct of slr.h, from gcc."""
    src = tmp_path / "layout.c"
    body = "".join(f'    printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "slr.h"\nint main(void) {\n'
                   f'    printf("%zu\\n", sizeof({struct}));\n{body}    return 0;\n}}\n')
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return [int(x) for x in out]


@pytest.mark.parametrize("struct", ["slr_desc", "slr_tune_result", "slr_user_desc", "slr_block", "slr_partial"])
def test_binding_struct_layout_matches_the_header(struct, tmp_path):
    from paper_1609_04567_gb300 import slr
    cls = getattr(slr, struct)
    fields = [name for name, _ in cls._fields_]
    got = _c_layout(struct, fields, tmp_path)
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, f).offset for f in fields]


def test_tuning_fields_are_validated(lib):
    from paper_1609_04567_gb300 import slr
    d = slr.slr_desc_init(slr.SLR_J2D5, 64, 64, 1)
    assert d.grid_ctas == 0 and d.tiling == slr.SLR_TILING_AUTO
    assert slr.slr_workspace_size(d) > 0
    assert slr.slr_workspace_size(slr.slr_desc_init(slr.SLR_J2D5, 64, 64, 1, grid_ctas=-1)) == 0
    assert slr.slr_workspace_size(slr.slr_desc_init(slr.SLR_RESTORE8, 64, 64, 1, tiling=3)) == 0
    assert slr.slr_workspace_size(slr.slr_desc_init(slr.SLR_J2D5, 64, 64, 1, grid_ctas=7)) > 0


def test_tune_scratch_size_and_argument_checks(lib):
    from paper_1609_04567_gb300 import slr
    d = slr.slr_desc_init(slr.SLR_LIFE, 8192, 8192, 1)
    assert slr.slr_tune_scratch_size(d) == 8192 * 8192 + slr.slr_workspace_size(d)
    assert slr.slr_tune_scratch_size(slr.slr_desc_init(slr.SLR_LIFE, 0, 8, 1)) == 0
    assert slr.slr_tune_lookup(d) is None          # nothing tuned in this process
    with pytest.raises(slr.SlrError) as e:
        slr.slr_tune(d, 0x1000, 0, 0x3000, 16, 0)   # scratch too small
    assert e.value.status == slr.SLR_ERR_WORKSPACE
    with pytest.raises(slr.SlrError) as e:
        slr.slr_tune(d, 0x1000, 0, 0x3001, 1 << 30, 0)  # misaligned scratch
    assert e.value.status == slr.SLR_ERR_INVALID_ARG
    j = slr.slr_desc_init(slr.SLR_J2D5, 8, 8, 1)
    with pytest.raises(slr.SlrError) as e:
        slr.slr_tune(j, 0x1000, 0, 0x3000, 1 << 20, 0)  # Jacobi needs f
    assert "aux" in slr.slr_tune_last_error()
    slr.slr_tune_clear()


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "slr.h"

int main(void)
{
    slr_desc d;
    slr_desc_init(&d, SLR_LIFE, 8192, 8192, 1);
    size_t ws = slr_workspace_size(&d);
    slr_desc j;
    slr_desc_init(&j, SLR_J3D7, 64, 64, 64);
    j.storage = SLR_BF16;
    size_t wj = slr_workspace_size(&j);
    slr_handle h = (slr_handle)0;
    slr_status st = slr_create(&j, (void *)0x1001, (const void *)0x2000, (void *)0x3000, wj, NULL, &h);
    printf("version %s\n", slr_version());
    printf("life_ws %zu %d %d\n", ws, d.boundary == SLR_WRAP, d.storage == SLR_U8);
    printf("j3d7_ws %zu\n", wj);
    printf("create %d %d %s\n", (int)st, h == (slr_handle)0, slr_last_error(NULL));
    printf("static_max %u\n", (unsigned)SLR_STATIC_STATE_BYTES);
    return 0;
}
"""


def test_plain_c_caller_links_and_uses_the_header(tmp_path):
    # A C99 program built against include/slr.h and libslr.so alone: the
    # boundary needs no Python, C++ or torch on the caller's side.  Only calls
    # that need no GPU run here.
    import subprocess
    from paper_1609_04567_gb300 import build
    lib = build.build()
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib),
                    "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    assert "sm_103a" in out[0]
    life = out[1].split()
    assert int(life[1]) >= 8192 * 8192 and life[2:] == ["1", "1"]
    wj = int(out[2].split()[1])
    assert wj >= 64 ** 3 * 2 and wj % 256 == 0
    create = out[3].split(maxsplit=3)
    assert int(create[1]) == -1 and create[2] == "1" and "16-byte aligned" in create[3]
    assert int(out[4].split()[1]) == 4 << 20


def test_restoration_workspace_holds_the_tile_records(lib):
    from paper_1609_04567_gb300 import slr
    up = lambda x: -(-x // 256) * 256
    # 4096 x 4096: control block, second state buffer, one 12,352-byte record per 64 x 64 tile
    d = slr.slr_desc_init(slr.SLR_RESTORE8, 4096, 4096, 1)
    assert slr.slr_workspace_size(d) == 4096 + up(4096 * 4096 * 4) + 64 * 64 * 12352
    # ragged tiles count whole
    assert slr.slr_workspace_size(slr.slr_desc_init(slr.SLR_RESTORE8, 80, 65, 1)) == \
        4096 + up(80 * 65 * 4) + up(2 * 2 * 12352)
    # rows that are not whole 16-byte mask groups: a copy of the mask with rows padded to 112 bytes
    assert slr.slr_workspace_size(slr.slr_desc_init(slr.SLR_RESTORE8, 100, 50, 1)) == \
        4096 + up(100 * 50 * 4) + up(2 * 12352) + up(112 * 50)
    # rows that are not whole 16-byte state groups: two copies of the state with rows of 92 floats too
    assert slr.slr_workspace_size(slr.slr_desc_init(slr.SLR_RESTORE8, 90, 30, 1)) == \
        4096 + up(90 * 30 * 4) + up(2 * 12352) + up(96 * 30) + 2 * up(92 * 30 * 4)
