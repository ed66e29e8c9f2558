/*
 * slr_oracle.c -- plain CPU oracle for the Loop-of-stencil-reduce hot path
 * (Aldinucci, Danelutto, Drocco, Kilpatrick, Misale, Peretti Pezzi, Torquati,
 * "A Parallel Pattern for Iterative Stencil + Reduce", arXiv 1609.04567).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct statement
 * of what the CUDA library computes.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no code, header or
 * constant with the CUDA library and the CUDA library never calls it.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * No fused multiply-add, IEEE round-to-nearest-even, no flush-to-zero.
 *
 * The same file also builds with -fopenmp, for timing the oracle on every host
 * core.  The only change that build makes is that the rows (3D: planes and
 * rows) of one sweep are shared among threads: every new item is still
 * computed from the old array alone by the same expression, and the per-sweep
 * reduces are a maximum, a 64-bit integer sum and an or, which give the same
 * result in any order.  So the threaded build returns bit-for-bit what the
 * single-threaded one does (a test checks this on every solver).
 *
 * Every solver is the loop-of-stencil-reduce-d-s procedure of Sec. 3.1 written
 * out step by step:
 *
 *     it = 0
 *     repeat
 *         b = stencil(sigma_1, f') : a      -- every new item from the old array only
 *         d = alpha(delta) : b              -- per-item change
 *         a = alpha(fst) : b                -- the new array becomes the state
 *         it = it + 1                       -- the global state of the -s variant
 *     until c(/(+):d, it)
 *
 * The test c is evaluated after the sweep (repeat-until), so at least one sweep
 * runs, and the returned state is the one that passed the test.
 *
 * Readings of the paper taken here (the paper leaves these open):
 *   - out-of-range neighbours (the "bottom" items of the stencil operator,
 *     Sec. 3.1) are the Dirichlet ghost value for the Jacobi stencils, the
 *     wrapped item for wrap_around, a dead cell for the dead-boundary Game of
 *     Life, and are left out of both sums for the restoration update;
 *   - the Helmholtz discretisation of Sec. 4.1 is the 5-point (3D: 7-point)
 *     Jacobi update u' = (h^2 f + sum of neighbours) / (2n + sigma h^2);
 *   - the restoration functional of Sec. 4.3 is phi(t) = sqrt(alpha + t^2),
 *     whose Jacobi fixed-point form is u' = sum w_j u_j / sum w_j with
 *     w_j = 1/sqrt(alpha + (u - u_j)^2), alpha = 100;
 *   - the mean |change| reduce of Sec. 4.3 truncates every |change| to a
 *     multiple of 2^-24 and adds integers, so the sum is exact and independent
 *     of summation order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Result of one solve: iterations run, reduced value of the last sweep,
 * whether the convergence test (rather than the cap) stopped the loop, and an
 * integer count (live cells for the Game of Life, masked items for the
 * restoration, 0 otherwise). */
typedef struct {
    int64_t iters;
    double value;
    int32_t converged;
    int32_t changed;
    uint64_t count;
} orc_result;

/* Threads a sweep may use: n >= 1 in the -fopenmp build; the single-threaded
 * build ignores n.  Returns the number that will be used. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Storage rounding (IEEE 754 round to nearest, ties to even).               */
/* ------------------------------------------------------------------------- */

static uint32_t f32_bits(float x) { uint32_t b; memcpy(&b, &x, 4); return b; }
static float bits_f32(uint32_t b) { float x; memcpy(&x, &b, 4); return x; }

/* binary32 -> bfloat16 (8-bit significand), round to nearest even.  NaN maps
 * to a quiet NaN of the same sign. */
uint16_t orc_f32_to_bf16(float x)
{
    uint32_t b = f32_bits(x);
    if ((b & 0x7F800000u) == 0x7F800000u && (b & 0x007FFFFFu) != 0)
        return (uint16_t)(((b >> 16) & 0x8000u) | 0x7FC0u);
    uint32_t keep = b >> 16;          /* truncated result */
    uint32_t rest = b & 0xFFFFu;      /* discarded low half */
    if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u)))
        keep += 1u;                    /* carries into the exponent correctly */
    return (uint16_t)keep;
}

float orc_bf16_to_f32(uint16_t h) { return bits_f32((uint32_t)h << 16); }

/* binary32 -> binary16 (11-bit significand, exponent bias 15), round to
 * nearest even, with gradual underflow and overflow to infinity. */
uint16_t orc_f32_to_f16(float x)
{
    uint32_t b = f32_bits(x);
    uint32_t sign = (b >> 16) & 0x8000u;
    int32_t ebits = (int32_t)((b >> 23) & 0xFFu);
    uint32_t man = b & 0x007FFFFFu;
    if (ebits == 0xFF)                               /* inf or NaN */
        return (uint16_t)(sign | (man ? 0x7E00u : 0x7C00u));
    if (ebits == 0)                                  /* |x| < 2^-126: rounds to 0 */
        return (uint16_t)sign;
    int32_t e = ebits - 127;                         /* x = m * 2^(e-23) */
    uint32_t m = man | 0x00800000u;                  /* 24-bit significand */
    if (e >= -14) {                                  /* binary16 normal range */
        uint32_t q = m >> 13, rest = m & 0x1FFFu;
        if (rest > 0x1000u || (rest == 0x1000u && (q & 1u))) q += 1u;
        int32_t he = e + 15;
        if (q == 0x800u) { q = 0x400u; he += 1; }    /* significand overflow */
        if (he >= 31) return (uint16_t)(sign | 0x7C00u);
        return (uint16_t)(sign | ((uint32_t)he << 10) | (q & 0x3FFu));
    }
    /* subnormal range: result in units of 2^-24 is m * 2^(e+1) */
    int32_t shift = -(e + 1);                        /* >= 14 */
    if (shift > 25) return (uint16_t)sign;           /* below half the least subnormal */
    uint32_t q = m >> shift;
    uint32_t rest = m & ((1u << shift) - 1u);
    uint32_t half = 1u << (shift - 1);
    if (rest > half || (rest == half && (q & 1u))) q += 1u;
    return (uint16_t)(sign | q);                     /* q == 0x400 is the least normal */
}

float orc_f16_to_f32(uint16_t h)
{
    uint32_t sign = ((uint32_t)h & 0x8000u) << 16;
    uint32_t e = ((uint32_t)h >> 10) & 0x1Fu, man = (uint32_t)h & 0x3FFu;
    float mag;
    if (e == 0x1F) return bits_f32(sign | 0x7F800000u | (man << 13));
    if (e == 0) mag = ldexpf((float)man, -24);                /* subnormal or zero */
    else mag = ldexpf((float)(man | 0x400u), (int)e - 25);    /* normal */
    return bits_f32(sign | f32_bits(mag));
}

/* Round a binary32 value to the storage precision and back.
 * storage: 0 = binary32 (identity), 1 = bfloat16, 2 = binary16. */
static float to_storage(float v, int storage)
{
    if (storage == 1) return orc_bf16_to_f32(orc_f32_to_bf16(v));
    if (storage == 2) return orc_f16_to_f32(orc_f32_to_f16(v));
    return v;
}

float orc_round_storage(float v, int storage) { return to_storage(v, storage); }

/* ------------------------------------------------------------------------- */
/* Neighbour access: the stencil operator sigma_1 of Sec. 3.1 with the       */
/* boundary reading of the boundary mode (0 = Dirichlet ghost, 1 = wrap).    */
/* ------------------------------------------------------------------------- */

static int64_t wrap_index(int64_t i, int64_t n) { return ((i % n) + n) % n; }

static double at2_f64(const double *a, int64_t nx, int64_t ny, int64_t i, int64_t j,
                      int wrap, double ghost)
{
    if (wrap) return a[wrap_index(i, ny) * nx + wrap_index(j, nx)];
    if (i < 0 || i >= ny || j < 0 || j >= nx) return ghost;
    return a[i * nx + j];
}

static float at2_f32(const float *a, int64_t nx, int64_t ny, int64_t i, int64_t j,
                     int wrap, float ghost)
{
    if (wrap) return a[wrap_index(i, ny) * nx + wrap_index(j, nx)];
    if (i < 0 || i >= ny || j < 0 || j >= nx) return ghost;
    return a[i * nx + j];
}

static double at3_f64(const double *a, int64_t nx, int64_t ny, int64_t nz,
                      int64_t k, int64_t i, int64_t j, int wrap, double ghost)
{
    if (wrap) return a[(wrap_index(k, nz) * ny + wrap_index(i, ny)) * nx + wrap_index(j, nx)];
    if (k < 0 || k >= nz || i < 0 || i >= ny || j < 0 || j >= nx) return ghost;
    return a[(k * ny + i) * nx + j];
}

static float at3_f32(const float *a, int64_t nx, int64_t ny, int64_t nz,
                     int64_t k, int64_t i, int64_t j, int wrap, float ghost)
{
    if (wrap) return a[(wrap_index(k, nz) * ny + wrap_index(i, ny)) * nx + wrap_index(j, nx)];
    if (k < 0 || k >= nz || i < 0 || i >= ny || j < 0 || j >= nx) return ghost;
    return a[(k * ny + i) * nx + j];
}

/* Mesh width: h <= 0 selects h = 1/(nx+1), the unit square (cube) with nx
 * interior points per side (Sec. 4.1 problem on a uniform mesh). */
static double mesh_h(double h, int64_t nx) { return h > 0.0 ? h : 1.0 / (double)(nx + 1); }

/* ------------------------------------------------------------------------- */
/* 2D 5-point Helmholtz Jacobi (Sec. 4.1), FP64.                             */
/*   u'_ij = (h^2 f_ij + ((u_N + u_S) + u_W) + u_E) / (4 + sigma h^2)        */
/* delta = |u' - u|, reduce = max (identity 0), c: max < tol or it == cap.   */
/* ------------------------------------------------------------------------- */

static double j2d5_sweep_f64(const double *u, double *v, const double *f,
                             int64_t nx, int64_t ny, double h2, double d,
                             int wrap, double ghost)
{
    double dmax = 0.0;
#pragma omp parallel for reduction(max : dmax) schedule(static)
    for (int64_t i = 0; i < ny; ++i)
        for (int64_t j = 0; j < nx; ++j) {
            double uN = at2_f64(u, nx, ny, i - 1, j, wrap, ghost);
            double uS = at2_f64(u, nx, ny, i + 1, j, wrap, ghost);
            double uW = at2_f64(u, nx, ny, i, j - 1, wrap, ghost);
            double uE = at2_f64(u, nx, ny, i, j + 1, wrap, ghost);
            double s = ((uN + uS) + uW) + uE;
            double t = h2 * f[i * nx + j];
            double nv = (t + s) / d;
            double dl = fabs(nv - u[i * nx + j]);
            if (dl > dmax) dmax = dl;
            v[i * nx + j] = nv;
        }
    return dmax;
}

int orc_j2d5_f64(double *u, const double *f, int64_t nx, int64_t ny, double sigma,
                 double h, int wrap, double ghost, double tol, int64_t max_iters,
                 orc_result *res)
{
    if (nx < 1 || ny < 1 || max_iters < 1) return -1;
    double hh = mesh_h(h, nx), h2 = hh * hh, d = 4.0 + sigma * h2;
    size_t n = (size_t)(nx * ny);
    double *v = (double *)malloc(n * sizeof(double));
    if (!v) return -2;
    int64_t it = 0;
    double val = 0.0;
    int conv = 0;
    do {
        val = j2d5_sweep_f64(u, v, f, nx, ny, h2, d, wrap, ghost);
        memcpy(u, v, n * sizeof(double));   /* a = fst(b) */
        it += 1;
        conv = val < tol;
    } while (!conv && it < max_iters);
    free(v);
    res->iters = it; res->value = val; res->converged = conv; res->changed = val > 0.0;
    res->count = 0;
    return 0;
}

/* Same update in FP32 arithmetic with the state kept in a storage precision
 * (0 binary32, 1 bfloat16, 2 binary16): every new value is rounded to the
 * storage precision before it is stored, and the change is taken between the
 * stored values.  u and f hold values already representable in storage. */
int orc_j2d5_f32(float *u, const float *f, int64_t nx, int64_t ny, double sigma,
                 double h, int wrap, float ghost, int storage, double tol,
                 int64_t max_iters, orc_result *res)
{
    if (nx < 1 || ny < 1 || max_iters < 1) return -1;
    double hh = mesh_h(h, nx), h2d = hh * hh;
    float h2 = (float)h2d, d = (float)(4.0 + sigma * h2d);   /* same constants as FP64, rounded */
    size_t n = (size_t)(nx * ny);
    float *v = (float *)malloc(n * sizeof(float));
    if (!v) return -2;
    int64_t it = 0;
    float val = 0.0f;
    int conv = 0;
    do {
        val = 0.0f;
#pragma omp parallel for reduction(max : val) schedule(static)
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                float s = ((at2_f32(u, nx, ny, i - 1, j, wrap, ghost) +
                            at2_f32(u, nx, ny, i + 1, j, wrap, ghost)) +
                           at2_f32(u, nx, ny, i, j - 1, wrap, ghost)) +
                          at2_f32(u, nx, ny, i, j + 1, wrap, ghost);
                float t = h2 * f[i * nx + j];
                float nv = to_storage((t + s) / d, storage);
                float dl = fabsf(nv - u[i * nx + j]);
                if (dl > val) val = dl;
                v[i * nx + j] = nv;
            }
        memcpy(u, v, n * sizeof(float));
        it += 1;
        conv = (double)val < tol;
    } while (!conv && it < max_iters);
    free(v);
    res->iters = it; res->value = (double)val; res->converged = conv;
    res->changed = val > 0.0f; res->count = 0;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 3D 7-point Helmholtz Jacobi (the n-dimensional stencil of Sec. 3.1 applied */
/* to the Sec. 4.1 problem in 3D):                                           */
/*   u' = (h^2 f + ((((u_x- + u_x+) + u_y-) + u_y+) + u_z-) + u_z+)          */
/*        / (6 + sigma h^2)                                                  */
/* x is the contiguous index j, y the row i, z the plane k.                  */
/* ------------------------------------------------------------------------- */

int orc_j3d7_f64(double *u, const double *f, int64_t nx, int64_t ny, int64_t nz,
                 double sigma, double h, int wrap, double ghost, double tol,
                 int64_t max_iters, orc_result *res)
{
    if (nx < 1 || ny < 1 || nz < 1 || max_iters < 1) return -1;
    double hh = mesh_h(h, nx), h2 = hh * hh, d = 6.0 + sigma * h2;
    size_t n = (size_t)(nx * ny * nz);
    double *v = (double *)malloc(n * sizeof(double));
    if (!v) return -2;
    int64_t it = 0;
    double val = 0.0;
    int conv = 0;
    do {
        val = 0.0;
#pragma omp parallel for collapse(2) reduction(max : val) schedule(static)
        for (int64_t k = 0; k < nz; ++k)
            for (int64_t i = 0; i < ny; ++i)
                for (int64_t j = 0; j < nx; ++j) {
                    double s = ((((at3_f64(u, nx, ny, nz, k, i, j - 1, wrap, ghost) +
                                   at3_f64(u, nx, ny, nz, k, i, j + 1, wrap, ghost)) +
                                  at3_f64(u, nx, ny, nz, k, i - 1, j, wrap, ghost)) +
                                 at3_f64(u, nx, ny, nz, k, i + 1, j, wrap, ghost)) +
                                at3_f64(u, nx, ny, nz, k - 1, i, j, wrap, ghost)) +
                               at3_f64(u, nx, ny, nz, k + 1, i, j, wrap, ghost);
                    size_t c = (size_t)((k * ny + i) * nx + j);
                    double nv = (h2 * f[c] + s) / d;
                    double dl = fabs(nv - u[c]);
                    if (dl > val) val = dl;
                    v[c] = nv;
                }
        memcpy(u, v, n * sizeof(double));
        it += 1;
        conv = val < tol;
    } while (!conv && it < max_iters);
    free(v);
    res->iters = it; res->value = val; res->converged = conv; res->changed = val > 0.0;
    res->count = 0;
    return 0;
}

int orc_j3d7_f32(float *u, const float *f, int64_t nx, int64_t ny, int64_t nz,
                 double sigma, double h, int wrap, float ghost, int storage,
                 double tol, int64_t max_iters, orc_result *res)
{
    if (nx < 1 || ny < 1 || nz < 1 || max_iters < 1) return -1;
    double hh = mesh_h(h, nx), h2d = hh * hh;
    float h2 = (float)h2d, d = (float)(6.0 + sigma * h2d);   /* same constants as FP64, rounded */
    size_t n = (size_t)(nx * ny * nz);
    float *v = (float *)malloc(n * sizeof(float));
    if (!v) return -2;
    int64_t it = 0;
    float val = 0.0f;
    int conv = 0;
    do {
        val = 0.0f;
#pragma omp parallel for collapse(2) reduction(max : val) schedule(static)
        for (int64_t k = 0; k < nz; ++k)
            for (int64_t i = 0; i < ny; ++i)
                for (int64_t j = 0; j < nx; ++j) {
                    float s = ((((at3_f32(u, nx, ny, nz, k, i, j - 1, wrap, ghost) +
                                  at3_f32(u, nx, ny, nz, k, i, j + 1, wrap, ghost)) +
                                 at3_f32(u, nx, ny, nz, k, i - 1, j, wrap, ghost)) +
                                at3_f32(u, nx, ny, nz, k, i + 1, j, wrap, ghost)) +
                               at3_f32(u, nx, ny, nz, k - 1, i, j, wrap, ghost)) +
                              at3_f32(u, nx, ny, nz, k + 1, i, j, wrap, ghost);
                    size_t c = (size_t)((k * ny + i) * nx + j);
                    float t = h2 * f[c];
                    float nv = to_storage((t + s) / d, storage);
                    float dl = fabsf(nv - u[c]);
                    if (dl > val) val = dl;
                    v[c] = nv;
                }
        memcpy(u, v, n * sizeof(float));
        it += 1;
        conv = (double)val < tol;
    } while (!conv && it < max_iters);
    free(v);
    res->iters = it; res->value = (double)val; res->converged = conv;
    res->changed = val > 0.0f; res->count = 0;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Game of Life, B3/S23 over the 8 Moore neighbours (Fig. 1 elemental         */
/* function).  Boundary: wrap = 1 is the torus (the wrap_around option of     */
/* Sec. 3), wrap = 0 the dead border of Fig. 1.  Two reduces per generation: */
/* the live count (+ on 64-bit integers, identity 0) and "any cell changed"  */
/* (delta = new != old, reduce = or).  c: nothing changed, or it == cap.     */
/* ------------------------------------------------------------------------- */

int orc_life(uint8_t *a, int64_t nx, int64_t ny, int wrap, int64_t max_gens,
             orc_result *res)
{
    if (nx < 1 || ny < 1 || max_gens < 1) return -1;
    size_t n = (size_t)(nx * ny);
    uint8_t *b = (uint8_t *)malloc(n);
    if (!b) return -2;
    int64_t it = 0;
    uint64_t live = 0;
    int changed = 0;
    do {
        live = 0;
        changed = 0;
#pragma omp parallel for reduction(+ : live) reduction(| : changed) schedule(static)
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                int alive_nbrs = 0;
                for (int64_t di = -1; di <= 1; ++di)
                    for (int64_t dj = -1; dj <= 1; ++dj) {
                        if (di == 0 && dj == 0) continue;
                        int64_t y = i + di, x = j + dj;
                        if (wrap) { y = wrap_index(y, ny); x = wrap_index(x, nx); }
                        else if (y < 0 || y >= ny || x < 0 || x >= nx) continue;
                        alive_nbrs += a[y * nx + x] != 0;
                    }
                int self = a[i * nx + j] != 0;
                int next = (alive_nbrs == 3) || (self && alive_nbrs == 2);
                b[i * nx + j] = (uint8_t)next;
                live += (uint64_t)next;
                changed |= next != self;
            }
        memcpy(a, b, n);
        it += 1;
    } while (changed && it < max_gens);
    free(b);
    res->iters = it; res->value = (double)live; res->converged = !changed;
    res->changed = changed; res->count = live;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Restoration phase of the two-phase denoiser (Sec. 4.3).                   */
/* For every noisy (masked) pixel, with the neighbours taken in row-major    */
/* order (dy = -1..1, dx = -1..1, centre skipped, out-of-range left out):    */
/*     t = u - u_j,  w_j = 1 / sqrt(alpha + t*t),                            */
/*     num += w_j * u_j,  den += w_j,   u' = num / den                       */
/* all in binary32.  Unmasked pixels are copied unchanged.                   */
/* delta = |u' - u| on masked pixels, truncated to a multiple of 2^-24 and   */
/* added as unsigned 64-bit integers; the reduced value is that sum * 2^-24  */
/* divided by the number of masked pixels (0 when there are none).           */
/* c: mean < tol, or it == cap.                                              */
/* ------------------------------------------------------------------------- */

static uint64_t fixed_2m24(float x) { return (uint64_t)((double)x * 16777216.0); }

int orc_restore8(float *u, const uint8_t *mask, int64_t nx, int64_t ny, float alpha,
                 double tol, int64_t max_iters, orc_result *res)
{
    if (nx < 1 || ny < 1 || max_iters < 1) return -1;
    size_t n = (size_t)(nx * ny);
    float *v = (float *)malloc(n * sizeof(float));
    if (!v) return -2;
    uint64_t nmask = 0;
    for (size_t c = 0; c < n; ++c) nmask += mask[c] != 0;
    int64_t it = 0;
    double mean = 0.0;
    int conv = 0;
    uint64_t sum = 0;
    do {
        sum = 0;
#pragma omp parallel for reduction(+ : sum) schedule(static)
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                size_t c = (size_t)(i * nx + j);
                float uc = u[c];
                if (!mask[c]) { v[c] = uc; continue; }
                float num = 0.0f, den = 0.0f;
                for (int64_t di = -1; di <= 1; ++di)
                    for (int64_t dj = -1; dj <= 1; ++dj) {
                        if (di == 0 && dj == 0) continue;
                        int64_t y = i + di, x = j + dj;
                        if (y < 0 || y >= ny || x < 0 || x >= nx) continue;
                        float uj = u[y * nx + x];
                        float t = uc - uj;
                        float w = 1.0f / sqrtf(alpha + t * t);
                        num = num + w * uj;
                        den = den + w;
                    }
                float nv = den > 0.0f ? num / den : uc;   /* a 1x1 image has no neighbours */
                v[c] = nv;
                sum += fixed_2m24(fabsf(nv - uc));
            }
        memcpy(u, v, n * sizeof(float));
        it += 1;
        mean = nmask ? ((double)sum * 0x1p-24) / (double)nmask : 0.0;
        conv = mean < tol;
    } while (!conv && it < max_iters);
    free(v);
    res->iters = it; res->value = mean; res->converged = conv; res->changed = sum != 0;
    res->count = nmask;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* FP64 defect correction around an FP32 Jacobi inner solve (2D 5-point).    */
/*   A u = ((4 + sigma h^2) u - sum of neighbours) / h^2,  ghost 0.          */
/* Starting from u (FP64), with r = f - A u:                                 */
/*   repeat                                                                  */
/*       r32 = (float) r                                                     */
/*       e = 0;  k_in FP32 Jacobi sweeps of A e = r32 (ghost 0):             */
/*             e' = (h2 * r32 + ((e_N + e_S) + e_W) + e_E) / d   (binary32)  */
/*       u = u + (double) e                                                  */
/*       r = f - A u (FP64);  rho = max |h^2 r / (4 + sigma h^2)|             */
/*       it = it + 1                                                         */
/*   until rho < tol or it == cap                                            */
/* rho equals the change the next FP64 Jacobi sweep would make, the same     */
/* measure as the plain FP64 solve.                                          */
/* ------------------------------------------------------------------------- */

static double defect_f64(const double *u, const double *f, double *r, int64_t nx,
                         int64_t ny, double h2, double d)
{
    double rho = 0.0;
#pragma omp parallel for reduction(max : rho) schedule(static)
    for (int64_t i = 0; i < ny; ++i)
        for (int64_t j = 0; j < nx; ++j) {
            double s = ((at2_f64(u, nx, ny, i - 1, j, 0, 0.0) +
                         at2_f64(u, nx, ny, i + 1, j, 0, 0.0)) +
                        at2_f64(u, nx, ny, i, j - 1, 0, 0.0)) +
                       at2_f64(u, nx, ny, i, j + 1, 0, 0.0);
            double au = (d * u[i * nx + j] - s) / h2;
            double rv = f[i * nx + j] - au;
            r[i * nx + j] = rv;
            double sc = fabs(h2 * rv / d);
            if (sc > rho) rho = sc;
        }
    return rho;
}

int orc_j2d5_dc(double *u, const double *f, int64_t nx, int64_t ny, double sigma,
                double h, double tol, int64_t k_in, int64_t max_outer,
                orc_result *res)
{
    if (nx < 1 || ny < 1 || max_outer < 1 || k_in < 1) return -1;
    double hh = mesh_h(h, nx), h2 = hh * hh, d = 4.0 + sigma * h2;
    float h2f = (float)h2, df = (float)d;
    size_t n = (size_t)(nx * ny);
    double *r = (double *)malloc(n * sizeof(double));
    float *r32 = (float *)malloc(n * sizeof(float));
    float *e = (float *)malloc(n * sizeof(float));
    float *e2 = (float *)malloc(n * sizeof(float));
    if (!r || !r32 || !e || !e2) { free(r); free(r32); free(e); free(e2); return -2; }
    defect_f64(u, f, r, nx, ny, h2, d);
    int64_t it = 0;
    double rho = 0.0;
    int conv = 0;
    do {
        for (size_t c = 0; c < n; ++c) { r32[c] = (float)r[c]; e[c] = 0.0f; }
        for (int64_t s = 0; s < k_in; ++s) {
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < ny; ++i)
                for (int64_t j = 0; j < nx; ++j) {
                    float sn = ((at2_f32(e, nx, ny, i - 1, j, 0, 0.0f) +
                                 at2_f32(e, nx, ny, i + 1, j, 0, 0.0f)) +
                                at2_f32(e, nx, ny, i, j - 1, 0, 0.0f)) +
                               at2_f32(e, nx, ny, i, j + 1, 0, 0.0f);
                    float t = h2f * r32[i * nx + j];
                    e2[i * nx + j] = (t + sn) / df;
                }
            memcpy(e, e2, n * sizeof(float));
        }
        for (size_t c = 0; c < n; ++c) u[c] = u[c] + (double)e[c];
        rho = defect_f64(u, f, r, nx, ny, h2, d);
        it += 1;
        conv = rho < tol;
    } while (!conv && it < max_outer);
    free(r); free(r32); free(e); free(e2);
    res->iters = it; res->value = rho; res->converged = conv; res->changed = 1;
    res->count = 0;
    return 0;
}

/* Scaled FP64 defect max |h^2 (f - A u) / (4 + sigma h^2)| of a 2D state with
 * ghost 0, used by the tests to check a returned solution. */
double orc_j2d5_scaled_defect(const double *u, const double *f, int64_t nx, int64_t ny,
                              double sigma, double h)
{
    double hh = mesh_h(h, nx), h2 = hh * hh, d = 4.0 + sigma * h2;
    double *r = (double *)malloc((size_t)(nx * ny) * sizeof(double));
    if (!r) return -1.0;
    double rho = defect_f64(u, f, r, nx, ny, h2, d);
    free(r);
    return rho;
}

/* The same defect correction for the 3D 7-point operator:
 *   A u = ((6 + sigma h^2) u - sum of the 6 neighbours) / h^2,  ghost 0,
 * neighbours summed x-, x+, y-, y+, z-, z+; inner binary32 Jacobi sweeps
 *   e' = (h2 * r32 + (((((e_x- + e_x+) + e_y-) + e_y+) + e_z-) + e_z+)) / d;
 * rho = max |h^2 r / (6 + sigma h^2)|, the change of the next FP64 sweep. */
static double defect3_f64(const double *u, const double *f, double *r, int64_t nx, int64_t ny, int64_t nz,
                          double h2, double d)
{
    double rho = 0.0;
#pragma omp parallel for collapse(2) reduction(max : rho) schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                double s = ((((at3_f64(u, nx, ny, nz, k, i, j - 1, 0, 0.0) +
                               at3_f64(u, nx, ny, nz, k, i, j + 1, 0, 0.0)) +
                              at3_f64(u, nx, ny, nz, k, i - 1, j, 0, 0.0)) +
                             at3_f64(u, nx, ny, nz, k, i + 1, j, 0, 0.0)) +
                            at3_f64(u, nx, ny, nz, k - 1, i, j, 0, 0.0)) +
                           at3_f64(u, nx, ny, nz, k + 1, i, j, 0, 0.0);
                size_t c = (size_t)((k * ny + i) * nx + j);
                double au = (d * u[c] - s) / h2;
                double rv = f[c] - au;
                r[c] = rv;
                double sc = fabs(h2 * rv / d);
                if (sc > rho) rho = sc;
            }
    return rho;
}

int orc_j3d7_dc(double *u, const double *f, int64_t nx, int64_t ny, int64_t nz, double sigma,
                double h, double tol, int64_t k_in, int64_t max_outer, orc_result *res)
{
    if (nx < 1 || ny < 1 || nz < 1 || max_outer < 1 || k_in < 1) return -1;
    double hh = mesh_h(h, nx), h2 = hh * hh, d = 6.0 + sigma * h2;
    float h2f = (float)h2, df = (float)d;
    size_t n = (size_t)(nx * ny * nz);
    double *r = (double *)malloc(n * sizeof(double));
    float *r32 = (float *)malloc(n * sizeof(float));
    float *e = (float *)malloc(n * sizeof(float));
    float *e2 = (float *)malloc(n * sizeof(float));
    if (!r || !r32 || !e || !e2) { free(r); free(r32); free(e); free(e2); return -2; }
    defect3_f64(u, f, r, nx, ny, nz, h2, d);
    int64_t it = 0;
    double rho = 0.0;
    int conv = 0;
    do {
        for (size_t c = 0; c < n; ++c) { r32[c] = (float)r[c]; e[c] = 0.0f; }
        for (int64_t s = 0; s < k_in; ++s) {
#pragma omp parallel for collapse(2) schedule(static)
            for (int64_t k = 0; k < nz; ++k)
                for (int64_t i = 0; i < ny; ++i)
                    for (int64_t j = 0; j < nx; ++j) {
                        float sn = ((((at3_f32(e, nx, ny, nz, k, i, j - 1, 0, 0.0f) +
                                       at3_f32(e, nx, ny, nz, k, i, j + 1, 0, 0.0f)) +
                                      at3_f32(e, nx, ny, nz, k, i - 1, j, 0, 0.0f)) +
                                     at3_f32(e, nx, ny, nz, k, i + 1, j, 0, 0.0f)) +
                                    at3_f32(e, nx, ny, nz, k - 1, i, j, 0, 0.0f)) +
                                   at3_f32(e, nx, ny, nz, k + 1, i, j, 0, 0.0f);
                        size_t c = (size_t)((k * ny + i) * nx + j);
                        float t = h2f * r32[c];
                        e2[c] = (t + sn) / df;
                    }
            memcpy(e, e2, n * sizeof(float));
        }
        for (size_t c = 0; c < n; ++c) u[c] = u[c] + (double)e[c];
        rho = defect3_f64(u, f, r, nx, ny, nz, h2, d);
        it += 1;
        conv = rho < tol;
    } while (!conv && it < max_outer);
    free(r); free(r32); free(e); free(e2);
    res->iters = it; res->value = rho; res->converged = conv; res->changed = 1;
    res->count = 0;
    return 0;
}

double orc_j3d7_scaled_defect(const double *u, const double *f, int64_t nx, int64_t ny, int64_t nz,
                              double sigma, double h)
{
    double hh = mesh_h(h, nx), h2 = hh * hh, d = 6.0 + sigma * h2;
    double *r = (double *)malloc((size_t)(nx * ny * nz) * sizeof(double));
    if (!r) return -1.0;
    double rho = defect3_f64(u, f, r, nx, ny, nz, h2, d);
    free(r);
    return rho;
}

/* Array forms of the storage conversions, for the tests. */
void orc_f32_to_bf16_array(const float *x, uint16_t *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_f32_to_bf16(x[i]);
}

void orc_f32_to_f16_array(const float *x, uint16_t *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_f32_to_f16(x[i]);
}

void orc_f16_to_f32_array(const uint16_t *x, float *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_f16_to_f32(x[i]);
}

void orc_round_storage_array(const float *x, float *out, int64_t n, int storage)
{
    for (int64_t i = 0; i < n; ++i) out[i] = to_storage(x[i], storage);
}

/* ------------------------------------------------------------------------- */
/* Adaptive median noise detector: the detection phase of the two-phase      */
/* restoration of Sec. 4.3 ("a traditional adaptive median filter"; the      */
/* paper does not define it, this is the textbook filter).  For the pixel z  */
/* at (i, j), square windows of side w = 3, 5, ..., wmax centred on it and   */
/* clipped to the image give zmin, zmax and zmed, the lower median (element  */
/* floor((n - 1) / 2) of the window's n values in ascending order).  The     */
/* first window with zmin < zmed < zmax decides: the filter outputs z when   */
/* zmin < z < zmax, else zmed.  When no window qualifies the output is zmed  */
/* of the largest window.  mask = 1 where the output differs from z (a noisy */
/* pixel), else 0.  The window values are counted in a 256-bin histogram.    */
/* ------------------------------------------------------------------------- */

int orc_amf_detect(const uint8_t *img, uint8_t *mask, int64_t nx, int64_t ny, int wmax)
{
    if (nx < 1 || ny < 1 || wmax < 3 || wmax % 2 == 0) return -1;
    int64_t cnt[256];
    for (int64_t i = 0; i < ny; ++i)
        for (int64_t j = 0; j < nx; ++j) {
            int z = img[i * nx + j];
            int out = -1, zmed = z;
            for (int64_t r = 1; 2 * r + 1 <= wmax; ++r) {
                memset(cnt, 0, sizeof cnt);
                int64_t n = 0;
                for (int64_t a = i - r; a <= i + r; ++a)
                    for (int64_t b = j - r; b <= j + r; ++b)
                        if (a >= 0 && a < ny && b >= 0 && b < nx) {
                            cnt[img[a * nx + b]] += 1;
                            n += 1;
                        }
                int zmin = 0, zmax = 255;
                while (cnt[zmin] == 0) ++zmin;
                while (cnt[zmax] == 0) --zmax;
                /* the value whose cumulative count first exceeds (n - 1) / 2 */
                int64_t m = (n - 1) / 2, seen = 0;
                int v = 0;
                while (seen + cnt[v] <= m) { seen += cnt[v]; ++v; }
                zmed = v;
                if (zmin < zmed && zmed < zmax) {
                    out = (zmin < z && z < zmax) ? z : zmed;
                    break;
                }
            }
            if (out < 0) out = zmed;
            mask[i * nx + j] = (uint8_t)(out != z);
        }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Sobel edge detector (Sec. 4.2): one 3x3 stencil sweep, no reduce.  The    */
/* paper applies the filter "from its definition" without fixing the         */
/* magnitude, the output type or the border; here: the two 3x3 gradients     */
/*   Gx = (z[i-1][j+1] - z[i-1][j-1]) + 2 (z[i][j+1] - z[i][j-1])            */
/*        + (z[i+1][j+1] - z[i+1][j-1])                                       */
/*   Gy = (z[i+1][j-1] - z[i-1][j-1]) + 2 (z[i+1][j] - z[i-1][j])            */
/*        + (z[i+1][j+1] - z[i-1][j+1])                                       */
/* in integers, out = min(255, floor(sqrt(Gx^2 + Gy^2))) for pixels with a   */
/* full 3x3 neighbourhood, 0 on the image's border.                          */
/* ------------------------------------------------------------------------- */

static int64_t isqrt_floor(int64_t n)
{
    int64_t r = (int64_t)sqrt((double)n);
    while (r * r > n) --r;
    while ((r + 1) * (r + 1) <= n) ++r;
    return r;
}

int orc_sobel(const uint8_t *img, uint8_t *out, int64_t nx, int64_t ny)
{
    if (nx < 1 || ny < 1) return -1;
    for (int64_t i = 0; i < ny; ++i)
        for (int64_t j = 0; j < nx; ++j) {
            if (i == 0 || j == 0 || i == ny - 1 || j == nx - 1) {
                out[i * nx + j] = 0;
                continue;
            }
            const uint8_t *up = img + (i - 1) * nx, *mid = img + i * nx, *dn = img + (i + 1) * nx;
            int64_t gx = ((int64_t)up[j + 1] - up[j - 1]) + 2 * ((int64_t)mid[j + 1] - mid[j - 1]) +
                         ((int64_t)dn[j + 1] - dn[j - 1]);
            int64_t gy = ((int64_t)dn[j - 1] - up[j - 1]) + 2 * ((int64_t)dn[j] - up[j]) +
                         ((int64_t)dn[j + 1] - up[j + 1]);
            int64_t m = isqrt_floor(gx * gx + gy * gy);
            out[i * nx + j] = (uint8_t)(m > 255 ? 255 : m);
        }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* One sweep of a block of rows: the 1:n deployment of Sec. 3.3 (Fig. 2), in  */
/* which one grid is cut into row blocks (3D: slabs of z-planes) over n       */
/* devices and, before each sweep, the rows next to a block are copied in     */
/* from the blocks that own them.  A block array holds `rows` consecutive     */
/* rows (planes) of the grid, the first of them global row row0 (negative or */
/* beyond the grid where the block sits at an edge); rows [lo, hi) are       */
/* updated from src into dst by exactly the expressions of the whole-grid     */
/* sweeps above, and the per-item change is reduced over rows [own_lo,        */
/* own_hi) only: the maximum as binary64 bits, the 2^-24 fixed-point sum, the */
/* count (live cells, masked pixels) and "any changed".  A row beyond the     */
/* grid's first or last row is the boundary (the Dirichlet ghost, a dead      */
/* cell, or left out for the restoration); with wrap the block's copied-in    */
/* rows already hold the wrapped rows.  Returns -1 when a row it must read    */
/* lies outside the block array.                                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t rows, row0, lo, hi, own_lo, own_hi;
} orc_block;

typedef struct {
    uint64_t maxbits, sum, count, changed;
} orc_partial;

/* Local index of the row d rows away from local row r, or -1 for the
 * boundary beyond the grid, or -2 when it lies outside the block array. */
static int64_t blk_row(const orc_block *b, int64_t r, int64_t d, int64_t ny, int wrap)
{
    int64_t g = b->row0 + r + d;
    if (!wrap && (g < 0 || g >= ny)) return -1;
    if (r + d < 0 || r + d >= b->rows) return -2;
    return r + d;
}

/* whether local row r is a row of the grid that this sweep updates */
static int blk_updates(const orc_block *b, int64_t r, int64_t ny, int wrap)
{
    int64_t g = b->row0 + r;
    return wrap || (g >= 0 && g < ny);
}

static uint64_t f64_bits(double x) { uint64_t v; memcpy(&v, &x, 8); return v; }

int orc_j2d5_block_f64(const double *u, double *v, const double *f, int64_t nx, int64_t ny,
                       const orc_block *b, double sigma, double h, int wrap, double ghost,
                       orc_partial *out)
{
    double hh = mesh_h(h, nx), h2 = hh * hh, d = 4.0 + sigma * h2;
    double dmax = 0.0;
    for (int64_t r = b->lo; r < b->hi; ++r) {
        if (!blk_updates(b, r, ny, wrap)) continue;
        int64_t rn = blk_row(b, r, -1, ny, wrap), rs = blk_row(b, r, 1, ny, wrap);
        if (rn == -2 || rs == -2) return -1;
        for (int64_t j = 0; j < nx; ++j) {
            double uN = rn < 0 ? ghost : u[rn * nx + j];
            double uS = rs < 0 ? ghost : u[rs * nx + j];
            double uW = at2_f64(u + r * nx, nx, 1, 0, j - 1, wrap, ghost);
            double uE = at2_f64(u + r * nx, nx, 1, 0, j + 1, wrap, ghost);
            double s = ((uN + uS) + uW) + uE;
            double t = h2 * f[r * nx + j];
            double nv = (t + s) / d;
            double dl = fabs(nv - u[r * nx + j]);
            if (r >= b->own_lo && r < b->own_hi && dl > dmax) dmax = dl;
            v[r * nx + j] = nv;
        }
    }
    out->maxbits = f64_bits(dmax); out->sum = 0; out->count = 0; out->changed = dmax > 0.0;
    return 0;
}

int orc_j2d5_block_f32(const float *u, float *v, const float *f, int64_t nx, int64_t ny,
                       const orc_block *b, double sigma, double h, int wrap, float ghost,
                       int storage, orc_partial *out)
{
    double hh = mesh_h(h, nx), h2d = hh * hh;
    float h2 = (float)h2d, d = (float)(4.0 + sigma * h2d);
    float val = 0.0f;
    for (int64_t r = b->lo; r < b->hi; ++r) {
        if (!blk_updates(b, r, ny, wrap)) continue;
        int64_t rn = blk_row(b, r, -1, ny, wrap), rs = blk_row(b, r, 1, ny, wrap);
        if (rn == -2 || rs == -2) return -1;
        for (int64_t j = 0; j < nx; ++j) {
            float s = (((rn < 0 ? ghost : u[rn * nx + j]) + (rs < 0 ? ghost : u[rs * nx + j])) +
                       at2_f32(u + r * nx, nx, 1, 0, j - 1, wrap, ghost)) +
                      at2_f32(u + r * nx, nx, 1, 0, j + 1, wrap, ghost);
            float t = h2 * f[r * nx + j];
            float nv = to_storage((t + s) / d, storage);
            float dl = fabsf(nv - u[r * nx + j]);
            if (r >= b->own_lo && r < b->own_hi && dl > val) val = dl;
            v[r * nx + j] = nv;
        }
    }
    out->maxbits = f64_bits((double)val); out->sum = 0; out->count = 0; out->changed = val > 0.0f;
    return 0;
}

/* 3D: the block's rows are z-planes of ny x nx items; nz is the grid's plane count. */
int orc_j3d7_block_f64(const double *u, double *v, const double *f, int64_t nx, int64_t ny, int64_t nz,
                       const orc_block *b, double sigma, double h, int wrap, double ghost,
                       orc_partial *out)
{
    double hh = mesh_h(h, nx), h2 = hh * hh, d = 6.0 + sigma * h2;
    double dmax = 0.0;
    int64_t pl = nx * ny;
    for (int64_t k = b->lo; k < b->hi; ++k) {
        if (!blk_updates(b, k, nz, wrap)) continue;
        int64_t kd = blk_row(b, k, -1, nz, wrap), ku = blk_row(b, k, 1, nz, wrap);
        if (kd == -2 || ku == -2) return -1;
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                const double *P = u + k * pl;
                double s = ((((at2_f64(P, nx, ny, i, j - 1, wrap, ghost) +
                               at2_f64(P, nx, ny, i, j + 1, wrap, ghost)) +
                              at2_f64(P, nx, ny, i - 1, j, wrap, ghost)) +
                             at2_f64(P, nx, ny, i + 1, j, wrap, ghost)) +
                            (kd < 0 ? ghost : u[kd * pl + i * nx + j])) +
                           (ku < 0 ? ghost : u[ku * pl + i * nx + j]);
                size_t c = (size_t)(k * pl + i * nx + j);
                double nv = (h2 * f[c] + s) / d;
                double dl = fabs(nv - u[c]);
                if (k >= b->own_lo && k < b->own_hi && dl > dmax) dmax = dl;
                v[c] = nv;
            }
    }
    out->maxbits = f64_bits(dmax); out->sum = 0; out->count = 0; out->changed = dmax > 0.0;
    return 0;
}

int orc_j3d7_block_f32(const float *u, float *v, const float *f, int64_t nx, int64_t ny, int64_t nz,
                       const orc_block *b, double sigma, double h, int wrap, float ghost, int storage,
                       orc_partial *out)
{
    double hh = mesh_h(h, nx), h2d = hh * hh;
    float h2 = (float)h2d, d = (float)(6.0 + sigma * h2d);
    float val = 0.0f;
    int64_t pl = nx * ny;
    for (int64_t k = b->lo; k < b->hi; ++k) {
        if (!blk_updates(b, k, nz, wrap)) continue;
        int64_t kd = blk_row(b, k, -1, nz, wrap), ku = blk_row(b, k, 1, nz, wrap);
        if (kd == -2 || ku == -2) return -1;
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                const float *P = u + k * pl;
                float s = ((((at2_f32(P, nx, ny, i, j - 1, wrap, ghost) +
                              at2_f32(P, nx, ny, i, j + 1, wrap, ghost)) +
                             at2_f32(P, nx, ny, i - 1, j, wrap, ghost)) +
                            at2_f32(P, nx, ny, i + 1, j, wrap, ghost)) +
                           (kd < 0 ? ghost : u[kd * pl + i * nx + j])) +
                          (ku < 0 ? ghost : u[ku * pl + i * nx + j]);
                size_t c = (size_t)(k * pl + i * nx + j);
                float t = h2 * f[c];
                float nv = to_storage((t + s) / d, storage);
                float dl = fabsf(nv - u[c]);
                if (k >= b->own_lo && k < b->own_hi && dl > val) val = dl;
                v[c] = nv;
            }
    }
    out->maxbits = f64_bits((double)val); out->sum = 0; out->count = 0; out->changed = val > 0.0f;
    return 0;
}

int orc_life_block(const uint8_t *a, uint8_t *c, int64_t nx, int64_t ny, const orc_block *b, int wrap,
                   orc_partial *out)
{
    uint64_t live = 0;
    int changed = 0;
    for (int64_t r = b->lo; r < b->hi; ++r) {
        if (!blk_updates(b, r, ny, wrap)) continue;
        int64_t rows[3] = {blk_row(b, r, -1, ny, wrap), r, blk_row(b, r, 1, ny, wrap)};
        if (rows[0] == -2 || rows[2] == -2) return -1;
        for (int64_t j = 0; j < nx; ++j) {
            int alive_nbrs = 0;
            for (int di = 0; di < 3; ++di)
                for (int64_t dj = -1; dj <= 1; ++dj) {
                    if (di == 1 && dj == 0) continue;
                    int64_t y = rows[di], x = j + dj;
                    if (y < 0) continue;                          /* dead border */
                    if (wrap) x = wrap_index(x, nx);
                    else if (x < 0 || x >= nx) continue;
                    alive_nbrs += a[y * nx + x] != 0;
                }
            int self = a[r * nx + j] != 0;
            int next = (alive_nbrs == 3) || (self && alive_nbrs == 2);
            c[r * nx + j] = (uint8_t)next;
            if (r >= b->own_lo && r < b->own_hi) {
                live += (uint64_t)next;
                changed |= next != self;
            }
        }
    }
    out->maxbits = 0; out->sum = 0; out->count = live; out->changed = (uint64_t)changed;
    return 0;
}

int orc_restore8_block(const float *u, float *v, const uint8_t *mask, int64_t nx, int64_t ny,
                       const orc_block *b, float alpha, orc_partial *out)
{
    uint64_t sum = 0, nmask = 0;
    for (int64_t r = b->lo; r < b->hi; ++r) {
        if (!blk_updates(b, r, ny, 0)) continue;
        int64_t rows[3] = {blk_row(b, r, -1, ny, 0), r, blk_row(b, r, 1, ny, 0)};
        if (rows[0] == -2 || rows[2] == -2) return -1;
        for (int64_t j = 0; j < nx; ++j) {
            size_t c = (size_t)(r * nx + j);
            float uc = u[c];
            if (!mask[c]) { v[c] = uc; continue; }
            float num = 0.0f, den = 0.0f;
            for (int di = 0; di < 3; ++di)
                for (int64_t dj = -1; dj <= 1; ++dj) {
                    if (di == 1 && dj == 0) continue;
                    int64_t y = rows[di], x = j + dj;
                    if (y < 0 || x < 0 || x >= nx) continue;      /* out of range: left out */
                    float uj = u[y * nx + x];
                    float t = uc - uj;
                    float w = 1.0f / sqrtf(alpha + t * t);
                    num = num + w * uj;
                    den = den + w;
                }
            float nv = den > 0.0f ? num / den : uc;
            v[c] = nv;
            if (r >= b->own_lo && r < b->own_hi) {
                sum += fixed_2m24(fabsf(nv - uc));
                nmask += 1;
            }
        }
    }
    out->maxbits = 0; out->sum = sum; out->count = nmask; out->changed = sum != 0;
    return 0;
}
