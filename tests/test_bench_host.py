"""Host-side helpers of bench.py (CPU only): the recorded ncu traffic is keyed
by a hash of the dominant kernel's code without its comments."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_strip_comments_keeps_code_and_strings():
    src = 'a = "//x /* y */";  // line\n/* block\n   two */ int b; /* c */ char q = \'/\';\n\n'
    assert bench.strip_comments(src) == 'a = "//x /* y */";\n int b;  char q = \'/\';'


def test_a_comment_edit_keeps_the_hash_and_a_code_edit_changes_it():
    base = "int f(int x) {\n  return x + 1;  // one\n}\n"
    assert bench.strip_comments(base) == bench.strip_comments(base.replace("// one", "// another note"))
    assert bench.strip_comments(base) != bench.strip_comments(base.replace("x + 1", "x + 2"))


def test_recorded_traffic_matches_the_current_kernel():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)["life_8192_k25"]
    assert rec["kernel_hash"] == bench.kernel_hash()
    t = bench.recorded_traffic("life_8192x8192_u8_torus_b3s23_2000gens", 25)
    assert t == rec["fixed_bytes"] + 80 * rec["dram_bytes_per_pass"]


def test_jacobi_case_names():
    import torch
    from paper_1609_04567_gb300 import slr
    assert bench.jacobi_case_of("j3d7_512x512x512_bf16_k4_s48", slr, torch) == \
        ("j3d7_512x512x512_bf16_k4_s48", slr.SLR_J3D7, (512, 512, 512), torch.bfloat16, 48, 4)
    # the shape is listed x first: 300 columns, 200 rows
    assert bench.jacobi_case_of("j2d5_300x200_f16", slr, torch)[2:] == ((200, 300), torch.float16, 200, 1)
    import pytest
    with pytest.raises(ValueError):
        bench.jacobi_case_of("j3d7_64x64_f32", slr, torch)
    with pytest.raises(ValueError):
        bench.jacobi_case_of("j2d5_64x64_f32_q3", slr, torch)
