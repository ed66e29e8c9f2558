"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/slr_oracle.c (a dropped term,
a wrong sign, a shifted index, a changed rule, a wrong rounding or a moved
convergence test), rebuilds the copy with gcc and runs the oracle pin tests
against it in a subprocess; the pins must fail.  The unmutated copy must pass.
Only the copy under pytest's temporary directory is touched.  CPU only."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, exact text in slr_oracle.c, replacement)
MUTATIONS = [
    ("J2D5 drops the east neighbour",
     "            double uE = at2_f64(u, nx, ny, i, j + 1, wrap, ghost);\n            double s = ((uN + uS) + uW) + uE;",
     "            double uE = at2_f64(u, nx, ny, i, j + 1, wrap, ghost);\n            double s = ((uN + uS) + uW);"),
    ("J2D5 sigma term with the wrong sign",
     "    double hh = mesh_h(h, nx), h2 = hh * hh, d = 4.0 + sigma * h2;\n    size_t n = (size_t)(nx * ny);\n"
     "    double *v = (double *)malloc(n * sizeof(double));",
     "    double hh = mesh_h(h, nx), h2 = hh * hh, d = 4.0 - sigma * h2;\n    size_t n = (size_t)(nx * ny);\n"
     "    double *v = (double *)malloc(n * sizeof(double));"),
    ("J2D5 h instead of h squared",
     "            double t = h2 * f[i * nx + j];",
     "            double t = sqrt(h2) * f[i * nx + j];"),
    ("J2D5 south neighbour two rows down",
     "            double uS = at2_f64(u, nx, ny, i + 1, j, wrap, ghost);",
     "            double uS = at2_f64(u, nx, ny, i + 2, j, wrap, ghost);"),
    ("J3D7 drops the z+ neighbour",
     "                               at3_f64(u, nx, ny, nz, k + 1, i, j, wrap, ghost);\n"
     "                    size_t c = (size_t)((k * ny + i) * nx + j);\n                    double nv",
     "                               0.0;\n"
     "                    size_t c = (size_t)((k * ny + i) * nx + j);\n                    double nv"),
    ("J3D7 wraps z by the row count",
     "                      int64_t k, int64_t i, int64_t j, int wrap, double ghost)\n{\n"
     "    if (wrap) return a[(wrap_index(k, nz) * ny",
     "                      int64_t k, int64_t i, int64_t j, int wrap, double ghost)\n{\n"
     "    if (wrap) return a[(wrap_index(k, ny) * ny"),
    ("J3D7 ignores the Dirichlet ghost value",
     "    if (k < 0 || k >= nz || i < 0 || i >= ny || j < 0 || j >= nx) return ghost;\n"
     "    return a[(k * ny + i) * nx + j];\n}\n\nstatic float at3_f32",
     "    if (k < 0 || k >= nz || i < 0 || i >= ny || j < 0 || j >= nx) return 0.0;\n"
     "    return a[(k * ny + i) * nx + j];\n}\n\nstatic float at3_f32"),
    ("J3D7 binary32 path divides by the 2D constant",
     "    float h2 = (float)h2d, d = (float)(6.0 + sigma * h2d);   /* same constants as FP64, rounded */",
     "    float h2 = (float)h2d, d = (float)(4.0 + sigma * h2d);   /* same constants as FP64, rounded */"),
    ("J3D7 binary32 path skips the storage rounding",
     "                    float nv = to_storage((t + s) / d, storage);\n                    float dl = fabsf(nv - u[c]);\n"
     "                    if (dl > val) val = dl;\n                    v[c] = nv;\n                }\n"
     "        memcpy(u, v, n * sizeof(float));\n        it += 1;\n        conv = (double)val < tol;\n"
     "    } while (!conv && it < max_iters);\n    free(v);\n    res->iters = it; res->value = (double)val; res->converged = conv;\n"
     "    res->changed = val > 0.0f; res->count = 0;\n    return 0;\n}\n\n/* ----",
     "                    float nv = (t + s) / d;\n                    float dl = fabsf(nv - u[c]);\n"
     "                    if (dl > val) val = dl;\n                    v[c] = nv;\n                }\n"
     "        memcpy(u, v, n * sizeof(float));\n        it += 1;\n        conv = (double)val < tol;\n"
     "    } while (!conv && it < max_iters);\n    free(v);\n    res->iters = it; res->value = (double)val; res->converged = conv;\n"
     "    res->changed = val > 0.0f; res->count = 0;\n    return 0;\n}\n\n/* ----"),
    ("J2D5 wraps rows by the column count",
     "static double at2_f64(const double *a, int64_t nx, int64_t ny, int64_t i, int64_t j,\n"
     "                      int wrap, double ghost)\n{\n    if (wrap) return a[wrap_index(i, ny) * nx",
     "static double at2_f64(const double *a, int64_t nx, int64_t ny, int64_t i, int64_t j,\n"
     "                      int wrap, double ghost)\n{\n    if (wrap) return a[wrap_index(i, nx) * nx"),
    ("J2D5 binary32 path ignores the Dirichlet ghost value",
     "    if (i < 0 || i >= ny || j < 0 || j >= nx) return ghost;\n    return a[i * nx + j];\n}\n\n"
     "static double at3_f64",
     "    if (i < 0 || i >= ny || j < 0 || j >= nx) return 0.0f;\n    return a[i * nx + j];\n}\n\n"
     "static double at3_f64"),
    ("default mesh width 1/nx instead of 1/(nx + 1)",
     "static double mesh_h(double h, int64_t nx) { return h > 0.0 ? h : 1.0 / (double)(nx + 1); }",
     "static double mesh_h(double h, int64_t nx) { return h > 0.0 ? h : 1.0 / (double)nx; }"),
    ("J2D5 reduces the change against the new neighbour sum",
     "            double dl = fabs(nv - u[i * nx + j]);\n            if (dl > dmax) dmax = dl;\n            v[i * nx + j] = nv;",
     "            double dl = fabs(nv - s / 4.0);\n            if (dl > dmax) dmax = dl;\n            v[i * nx + j] = nv;"),
    ("J2D5 counts one sweep too few",
     "        memcpy(u, v, n * sizeof(double));   /* a = fst(b) */\n        it += 1;\n"
     "        conv = val < tol;\n    } while (!conv && it < max_iters);\n    free(v);\n"
     "    res->iters = it;",
     "        memcpy(u, v, n * sizeof(double));   /* a = fst(b) */\n        it += 1;\n"
     "        conv = val < tol;\n    } while (!conv && it < max_iters);\n    free(v);\n"
     "    res->iters = it - (it > 1);"),
    ("Life rule S23 becomes S3",
     "                int next = (alive_nbrs == 3) || (self && alive_nbrs == 2);",
     "                int next = (alive_nbrs == 3);"),
    ("Life wrap-around off by one to the west",
     "                        if (wrap) { y = wrap_index(y, ny); x = wrap_index(x, nx); }",
     "                        if (wrap) { y = wrap_index(y, ny); x = wrap_index(x + (x < 0), nx); }"),
    ("Life counts the cell itself as a neighbour",
     "                        if (di == 0 && dj == 0) continue;\n                        int64_t y = i + di, x = j + dj;\n"
     "                        if (wrap) {",
     "                        int64_t y = i + di, x = j + dj;\n"
     "                        if (wrap) {"),
    ("Life also births on six neighbours (HighLife)",
     "                int next = (alive_nbrs == 3) || (self && alive_nbrs == 2);",
     "                int next = (alive_nbrs == 3) || (!self && alive_nbrs == 6) || (self && alive_nbrs == 2);"),
    ("Life dead border wraps its columns",
     "                        else if (y < 0 || y >= ny || x < 0 || x >= nx) continue;\n"
     "                        alive_nbrs",
     "                        else if (y < 0 || y >= ny) continue;\n"
     "                        else if (x < 0 || x >= nx) x = wrap_index(x, nx);\n"
     "                        alive_nbrs"),
    ("restoration skips a neighbour",
     "                        if (di == 0 && dj == 0) continue;\n                        int64_t y = i + di, x = j + dj;\n"
     "                        if (y < 0 || y >= ny || x < 0 || x >= nx) continue;\n                        float uj",
     "                        if (di == 0 && dj >= 0) continue;\n                        int64_t y = i + di, x = j + dj;\n"
     "                        if (y < 0 || y >= ny || x < 0 || x >= nx) continue;\n                        float uj"),
    ("restoration weight without the square root",
     "                        float w = 1.0f / sqrtf(alpha + t * t);",
     "                        float w = 1.0f / (alpha + t * t);"),
    ("restoration weight with alpha 1",
     "                        float w = 1.0f / sqrtf(alpha + t * t);",
     "                        float w = 1.0f / sqrtf(1.0f + t * t);"),
    ("restoration mean over every pixel",
     "        mean = nmask ? ((double)sum * 0x1p-24) / (double)nmask : 0.0;",
     "        mean = nmask ? ((double)sum * 0x1p-24) / (double)n : 0.0;"),
    ("restoration reads this sweep's new values (Gauss-Seidel order)",
     "                        float uj = u[y * nx + x];",
     "                        float uj = (size_t)(y * nx + x) < c ? v[y * nx + x] : u[y * nx + x];"),
    ("restoration replicates the edge instead of leaving out-of-range neighbours",
     "                        if (y < 0 || y >= ny || x < 0 || x >= nx) continue;\n                        float uj",
     "                        if (y < 0) y = 0;\n                        if (y >= ny) y = ny - 1;\n"
     "                        if (x < 0) x = 0;\n                        if (x >= nx) x = nx - 1;\n                        float uj"),
    ("restoration rounds each change to 2^-24 instead of truncating",
     "static uint64_t fixed_2m24(float x) { return (uint64_t)((double)x * 16777216.0); }",
     "static uint64_t fixed_2m24(float x) { return (uint64_t)((double)x * 16777216.0 + 0.5); }"),
    ("defect correction with the defect's sign flipped",
     "            double rv = f[i * nx + j] - au;",
     "            double rv = au - f[i * nx + j];"),
    ("defect correction resumes the inner solve from the last correction",
     "        for (size_t c = 0; c < n; ++c) { r32[c] = (float)r[c]; e[c] = 0.0f; }\n"
     "        for (int64_t s = 0; s < k_in; ++s) {\n#pragma omp parallel for schedule(static)",
     "        for (size_t c = 0; c < n; ++c) { r32[c] = (float)r[c]; }\n"
     "        for (int64_t s = 0; s < k_in; ++s) {\n#pragma omp parallel for schedule(static)"),
    ("defect correction inner solve on the binary64 defect's first sweep only",
     "                    float t = h2f * r32[i * nx + j];\n                    e2[i * nx + j] = (t + sn) / df;",
     "                    float t = s == 0 ? h2f * r32[i * nx + j] : 0.0f;\n                    e2[i * nx + j] = (t + sn) / df;"),
    ("defect correction subtracts the correction",
     "        for (size_t c = 0; c < n; ++c) u[c] = u[c] + (double)e[c];\n        rho = defect_f64(",
     "        for (size_t c = 0; c < n; ++c) u[c] = u[c] - (double)e[c];\n        rho = defect_f64("),
    ("bfloat16 rounds half up instead of to even",
     "    if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u)))\n        keep += 1u;",
     "    if (rest >= 0x8000u)\n        keep += 1u;"),
    ("detector takes the upper median",
     "                int64_t m = (n - 1) / 2, seen = 0;",
     "                int64_t m = n / 2, seen = 0;"),
    ("detector keeps pixels equal to a window extreme",
     "                    out = (zmin < z && z < zmax) ? z : zmed;",
     "                    out = (zmin <= z && z <= zmax) ? z : zmed;"),
    ("detector decides on a window whose median is an extreme",
     "                if (zmin < zmed && zmed < zmax) {",
     "                if (zmin <= zmed && zmed < zmax) {"),
    ("detector keeps the pixel when no window decides",
     "            if (out < 0) out = zmed;",
     "            if (out < 0) out = z;"),
    ("detector replicates the image edge into clipped windows",
     "                        if (a >= 0 && a < ny && b >= 0 && b < nx) {\n                            cnt[img[a * nx + b]] += 1;",
     "                        {\n                            int64_t aa = a < 0 ? 0 : (a >= ny ? ny - 1 : a), bb = b < 0 ? 0 : (b >= nx ? nx - 1 : b);\n"
     "                            cnt[img[aa * nx + bb]] += 1;"),
    ("detector starts at the 5 x 5 window",
     "            for (int64_t r = 1; 2 * r + 1 <= wmax; ++r) {",
     "            for (int64_t r = 2; 2 * r + 1 <= wmax; ++r) {"),
    ("Sobel weights the wrong column of Gy",
     "            int64_t gy = ((int64_t)dn[j - 1] - up[j - 1]) + 2 * ((int64_t)dn[j] - up[j]) +\n"
     "                         ((int64_t)dn[j + 1] - up[j + 1]);",
     "            int64_t gy = ((int64_t)dn[j - 1] - up[j - 1]) + ((int64_t)dn[j] - up[j]) +\n"
     "                         2 * ((int64_t)dn[j + 1] - up[j + 1]);"),
    ("Sobel takes Gx one column to the left",
     "            int64_t gx = ((int64_t)up[j + 1] - up[j - 1]) + 2 * ((int64_t)mid[j + 1] - mid[j - 1]) +",
     "            int64_t gx = ((int64_t)up[j] - up[j - 1]) + 2 * ((int64_t)mid[j] - mid[j - 1]) +"),
    ("Sobel drops the centre row's weight 2",
     "            int64_t gx = ((int64_t)up[j + 1] - up[j - 1]) + 2 * ((int64_t)mid[j + 1] - mid[j - 1]) +",
     "            int64_t gx = ((int64_t)up[j + 1] - up[j - 1]) + ((int64_t)mid[j + 1] - mid[j - 1]) +"),
    ("Sobel magnitude rounded up",
     "    while ((r + 1) * (r + 1) <= n) ++r;",
     "    while (r * r < n) ++r;"),
    ("Sobel clamps at 254",
     "            out[i * nx + j] = (uint8_t)(m > 255 ? 255 : m);",
     "            out[i * nx + j] = (uint8_t)(m > 254 ? 254 : m);"),
    ("Sobel copies the border",
     "                out[i * nx + j] = 0;\n                continue;",
     "                out[i * nx + j] = img[i * nx + j];\n                continue;"),
    ("3D defect with the wrong sign of the neighbour sum",
     "                double au = (d * u[c] - s) / h2;",
     "                double au = (d * u[c] + s) / h2;"),
    ("3D defect correction with the 2D diagonal",
     "    double hh = mesh_h(h, nx), h2 = hh * hh, d = 6.0 + sigma * h2;\n    float h2f = (float)h2, df = (float)d;\n"
     "    size_t n = (size_t)(nx * ny * nz);",
     "    double hh = mesh_h(h, nx), h2 = hh * hh, d = 4.0 + sigma * h2;\n    float h2f = (float)h2, df = (float)d;\n"
     "    size_t n = (size_t)(nx * ny * nz);"),
    ("binary16 subnormal shift off by one",
     "    int32_t shift = -(e + 1);                        /* >= 14 */",
     "    int32_t shift = -(e + 2);                        /* >= 14 */"),
]


def run_pins(tmp_path, source: str) -> subprocess.CompletedProcess:
    """Run the oracle pin tests against `source` as oracle/slr_oracle.c."""
    work = tmp_path / "copy"
    shutil.copytree(os.path.join(ROOT, "oracle"), work / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    (work / "oracle" / "slr_oracle.c").write_text(source)
    (work / "tests").mkdir()
    for name in os.listdir(os.path.join(ROOT, "tests")):
        if name == "conftest.py" or (name.startswith("test_oracle_") and name.endswith(".py")
                                     and name != os.path.basename(__file__)):
            shutil.copy(os.path.join(ROOT, "tests", name), work / "tests" / name)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), work / "tests" / "golden")
    shutil.copy(os.path.join(ROOT, "pytest.ini"), work / "pytest.ini")
    env = dict(os.environ, PYTHONPATH=ROOT)     # the input generators come from the package
    # the exhaustive (slow) pins run once in the main suite, not for every mutant
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "not gpu and not slow", "tests"],
                          cwd=work, env=env, capture_output=True, text=True, timeout=300)


def oracle_source() -> str:
    with open(os.path.join(ROOT, "oracle", "slr_oracle.c")) as fh:
        return fh.read()


def test_unmutated_copy_passes(tmp_path):
    p = run_pins(tmp_path, oracle_source())
    assert p.returncode == 0, p.stdout[-2000:]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_mistake(tmp_path, name, old, new):
    src = oracle_source()
    assert src.count(old) == 1, f"mutation site of '{name}' not found once in slr_oracle.c"
    mutated = src.replace(old, new)
    # the mutant must build: a compile error would fail the pins for the wrong reason
    c = tmp_path / "mutant.c"
    c.write_text(mutated)
    subprocess.run(["gcc", "-std=c11", "-fsyntax-only", str(c)], check=True)
    p = run_pins(tmp_path, mutated)
    assert p.returncode != 0, f"'{name}' was not caught by any pin:\n{p.stdout[-1500:]}"
