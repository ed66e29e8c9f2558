// split.cu -- one sweep of a row block of a larger grid: the device step of
// the 1:n deployment of Sec. 3.3 (Fig. 2), in which one grid is cut into row
// blocks (3D: slabs of z-planes) over n devices and, before each sweep (or
// each pass of k sweeps), the rows next to a block are copied in from the
// blocks that own them; the per-device partial reduces are then combined
// into the value the convergence test reads.
//
// A block array holds `rows` consecutive rows of the grid, the first of them
// global row row0; rows [lo, hi) are updated from src into dst by the same
// operations, in the same order, as the whole-grid sweeps (every item from old
// values only), and the change is reduced over rows [own_lo, own_hi) into one
// partial (max |delta| as binary64 bits, the 2^-24 fixed-point sum of the
// restoration, the live or masked count, "any changed").  Rows beyond the
// grid's first and last row are the boundary: the Dirichlet ghost, a dead
// cell, or left out of the restoration's sums; with wrap_around the block's
// copied-in rows already hold the wrapped rows.  Columns (and 3D rows) follow
// the descriptor's boundary as in the whole-grid sweeps.
//
// The kernel is a plain grid-stride sweep, one item per thread per step: the
// partitioned loop exchanges halos and reduces on the host between sweeps,
// and its device step needs exactness, not the tiled kernels' staging.
#include <string>

#include "restore_math.cuh"
#include "slr_internal.cuh"

namespace slr {
void set_handleless_error(const std::string &msg);   // slr_api.cu: slr_last_error(NULL)

namespace {

static_assert(sizeof(slr_partial) == sizeof(Slot), "a partial is one reduce slot");

struct Geo {
    long long nx, ny;          // columns; rows of a plane (3D) or 1
    long long rows, row0, lo, hi, own_lo, own_hi;
    long long grid_rows;       // the grid's rows (2D) or planes (3D)
    int wrap;
};

// local index of the row d away from local row r, or -1 for the boundary
__device__ __forceinline__ long long brow(const Geo &g, long long r, int d)
{
    const long long gr = g.row0 + r + d;
    if (!g.wrap && (gr < 0 || gr >= g.grid_rows)) return -1;
    return r + d;
}

__device__ __forceinline__ bool updated(const Geo &g, long long r)
{
    const long long gr = g.row0 + r;
    return g.wrap || (gr >= 0 && gr < g.grid_rows);
}

__device__ __forceinline__ bool owned(const Geo &g, long long r) { return r >= g.own_lo && r < g.own_hi; }

__device__ __forceinline__ long long wrapc(long long j, long long n) { return j < 0 ? j + n : (j >= n ? j - n : j); }

// storage <-> binary32
__device__ __forceinline__ float ld32(const float *p) { return *p; }
__device__ __forceinline__ float ld32(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld32(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void st32(float *p, float v) { *p = v; }
__device__ __forceinline__ void st32(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st32(__half *p, float v) { *p = __float2half_rn(v); }

// ---- Jacobi, binary64 -------------------------------------------------------
// 2D: ny == 1 and a row is nx items.  3D: a row is a plane of ny x nx items.
template <int DIM>
__global__ void jacobi_block_f64(const double *u, double *v, const double *f, Geo g, double h2, double d, double ghost,
                                 Slot *slot)
{
    const long long pl = g.nx * g.ny;
    const long long n = (g.hi - g.lo) * pl;
    unsigned long long mx = 0ull;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = g.lo + i / pl, q = i % pl, y = q / g.nx, x = q % g.nx;
        if (!updated(g, r)) continue;
        const long long c = r * pl + q;
        const long long rm = brow(g, r, -1), rp = brow(g, r, 1);
        const double *P = u + r * pl;
        const double uW = g.wrap ? P[y * g.nx + wrapc(x - 1, g.nx)] : (x > 0 ? P[y * g.nx + x - 1] : ghost);
        const double uE = g.wrap ? P[y * g.nx + wrapc(x + 1, g.nx)] : (x + 1 < g.nx ? P[y * g.nx + x + 1] : ghost);
        const double zm = rm < 0 ? ghost : u[rm * pl + q], zp = rp < 0 ? ghost : u[rp * pl + q];
        double s;
        if (DIM == 2) {
            s = __dadd_rn(__dadd_rn(__dadd_rn(zm, zp), uW), uE);
        } else {
            const double uS = g.wrap ? P[wrapc(y - 1, g.ny) * g.nx + x] : (y > 0 ? P[(y - 1) * g.nx + x] : ghost);
            const double uN = g.wrap ? P[wrapc(y + 1, g.ny) * g.nx + x] : (y + 1 < g.ny ? P[(y + 1) * g.nx + x] : ghost);
            s = __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(uW, uE), uS), uN), zm), zp);
        }
        const double nv = __ddiv_rn(__dadd_rn(__dmul_rn(h2, f[c]), s), d);
        v[c] = nv;
        if (owned(g, r)) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(__dsub_rn(nv, u[c])));
            mx = b > mx ? b : mx;
        }
    }
    block_to_slot(slot, mx, 0ull, 0ull, mx != 0ull);
}

// ---- Jacobi, binary32 arithmetic, storage T ----------------------------------
template <int DIM, class T>
__global__ void jacobi_block_f32(const T *u, T *v, const T *f, Geo g, float h2, float d, float ghost, Slot *slot)
{
    const long long pl = g.nx * g.ny;
    const long long n = (g.hi - g.lo) * pl;
    float mx = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = g.lo + i / pl, q = i % pl, y = q / g.nx, x = q % g.nx;
        if (!updated(g, r)) continue;
        const long long c = r * pl + q;
        const long long rm = brow(g, r, -1), rp = brow(g, r, 1);
        const T *P = u + r * pl;
        const float uW = g.wrap ? ld32(P + y * g.nx + wrapc(x - 1, g.nx)) : (x > 0 ? ld32(P + y * g.nx + x - 1) : ghost);
        const float uE = g.wrap ? ld32(P + y * g.nx + wrapc(x + 1, g.nx))
                                : (x + 1 < g.nx ? ld32(P + y * g.nx + x + 1) : ghost);
        const float zm = rm < 0 ? ghost : ld32(u + rm * pl + q), zp = rp < 0 ? ghost : ld32(u + rp * pl + q);
        float s;
        if (DIM == 2) {
            s = __fadd_rn(__fadd_rn(__fadd_rn(zm, zp), uW), uE);
        } else {
            const float uS = g.wrap ? ld32(P + wrapc(y - 1, g.ny) * g.nx + x) : (y > 0 ? ld32(P + (y - 1) * g.nx + x) : ghost);
            const float uN = g.wrap ? ld32(P + wrapc(y + 1, g.ny) * g.nx + x)
                                    : (y + 1 < g.ny ? ld32(P + (y + 1) * g.nx + x) : ghost);
            s = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(uW, uE), uS), uN), zm), zp);
        }
        st32(v + c, __fdiv_rn(__fadd_rn(__fmul_rn(h2, ld32(f + c)), s), d));
        if (owned(g, r)) mx = fmaxf(mx, fabsf(__fsub_rn(ld32(v + c), ld32(u + c))));
    }
    block_to_slot(slot, (unsigned long long)__double_as_longlong((double)mx), 0ull, 0ull, mx != 0.0f);
}

// ---- Game of Life -----------------------------------------------------------
__global__ void life_block(const unsigned char *a, unsigned char *b, Geo g, Slot *slot)
{
    const long long n = (g.hi - g.lo) * g.nx;
    unsigned long long live = 0ull;
    unsigned int changed = 0u;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = g.lo + i / g.nx, x = i % g.nx;
        if (!updated(g, r)) continue;
        const long long rr[3] = {brow(g, r, -1), r, brow(g, r, 1)};
        int nb = 0;
#pragma unroll
        for (int di = 0; di < 3; ++di) {
            if (rr[di] < 0) continue;                       // dead border
#pragma unroll
            for (int dj = -1; dj <= 1; ++dj) {
                if (di == 1 && dj == 0) continue;
                long long xx = x + dj;
                if (g.wrap) xx = wrapc(xx, g.nx);
                else if (xx < 0 || xx >= g.nx) continue;
                nb += a[rr[di] * g.nx + xx] != 0;
            }
        }
        const int self = a[r * g.nx + x] != 0;
        const int next = nb == 3 || (self && nb == 2);
        b[r * g.nx + x] = (unsigned char)next;
        if (owned(g, r)) {
            live += (unsigned long long)next;
            changed |= (unsigned)(next != self);
        }
    }
    block_to_slot(slot, 0ull, 0ull, live, changed);
}

// ---- restoration --------------------------------------------------------------
__global__ void restore_block(const float *u, float *v, const unsigned char *mask, Geo g, float alpha, Slot *slot)
{
    const long long n = (g.hi - g.lo) * g.nx;
    unsigned long long sum = 0ull, cnt = 0ull;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = g.lo + i / g.nx, x = i % g.nx;
        if (!updated(g, r)) continue;
        const long long c = r * g.nx + x;
        const float uc = u[c];
        if (!mask[c]) {
            v[c] = uc;
            continue;
        }
        const long long rr[3] = {brow(g, r, -1), r, brow(g, r, 1)};
        float num = 0.0f, den = 0.0f;
#pragma unroll
        for (int di = 0; di < 3; ++di) {
            if (rr[di] < 0) continue;                       // beyond the grid: left out
#pragma unroll
            for (int dj = -1; dj <= 1; ++dj) {
                if ((di == 1 && dj == 0) || x + dj < 0 || x + dj >= g.nx) continue;
                restore_accumulate<false>(uc, u[rr[di] * g.nx + x + dj], alpha, num, den);
            }
        }
        const float nv = restore_quotient<false>(num, den, uc);
        v[c] = nv;
        if (owned(g, r)) {
            sum += fixed_2m24(__fsub_rn(nv, uc));
            cnt += 1ull;
        }
    }
    block_to_slot(slot, 0ull, sum, cnt, sum != 0ull);
}

int grid_for(long long items)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (items + 255) / 256;
    const long long cap = (long long)(sms > 0 ? sms : 1) * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

slr_status fail(slr_status s, const std::string &msg)
{
    set_handleless_error("slr_block_sweep: " + msg);
    return s;
}

}  // namespace
}  // namespace slr

extern "C" slr_status slr_block_sweep(const slr_desc *d, const slr_block *b, const void *src, void *dst,
                                      const void *aux, slr_partial *partial, void *stream)
{
    using namespace slr;
    bool unsup = false;
    const std::string why = describe_invalid(d, &unsup);
    if (!why.empty()) return fail(unsup ? SLR_ERR_UNSUPPORTED : SLR_ERR_INVALID_ARG, why);
    if (d->defect_correction) return fail(SLR_ERR_UNSUPPORTED, "defect correction is not split");
    if (!b) return fail(SLR_ERR_INVALID_ARG, "block is NULL");
    if (!src || !dst || !partial || src == dst) return fail(SLR_ERR_INVALID_ARG, "src, dst and partial must be distinct device pointers");
    if (d->stencil != SLR_LIFE && !aux) return fail(SLR_ERR_INVALID_ARG, "aux (f or mask) is required");
    const bool three = d->stencil == SLR_J3D7;
    Geo g;
    g.nx = d->nx;
    g.ny = three ? d->ny : 1;
    g.grid_rows = three ? d->nz : d->ny;
    g.rows = b->rows;
    g.row0 = b->row0;
    g.lo = b->lo;
    g.hi = b->hi;
    g.own_lo = b->own_lo;
    g.own_hi = b->own_hi;
    g.wrap = d->boundary == SLR_WRAP;
    if (g.rows < 1 || g.lo < 0 || g.hi > g.rows || g.lo > g.hi || g.own_lo < g.lo || g.own_hi > g.hi ||
        g.own_lo > g.own_hi)
        return fail(SLR_ERR_INVALID_ARG, "need 0 <= lo <= own_lo <= own_hi <= hi <= rows, rows >= 1");
    // the rows next to the first and last updated rows must be in the block
    // array unless they lie beyond the grid (the boundary)
    long long first = g.lo, last = g.hi - 1;
    if (!g.wrap) {
        first = first > -g.row0 ? first : -g.row0;
        last = last < g.grid_rows - 1 - g.row0 ? last : g.grid_rows - 1 - g.row0;
    }
    if (first <= last) {
        const bool below_in_grid = g.wrap || g.row0 + first - 1 >= 0;
        const bool above_in_grid = g.wrap || g.row0 + last + 1 < g.grid_rows;
        if ((first == 0 && below_in_grid) || (last == g.rows - 1 && above_in_grid))
            return fail(SLR_ERR_INVALID_ARG, "an updated row's neighbour row lies outside the block array");
    }
    cudaStream_t st = (cudaStream_t)stream;
    Slot *slot = (Slot *)partial;
    cudaError_t e = cudaMemsetAsync(slot, 0, sizeof(Slot), st);
    if (e != cudaSuccess) return fail(SLR_ERR_CUDA, std::string("clear partial: ") + cudaGetErrorString(e));
    const Problem p = problem_of(d);
    const long long items = (g.hi - g.lo) * g.nx * g.ny;
    const int grid = grid_for(items);
    if (items > 0) {
        switch (d->stencil) {
        case SLR_LIFE:
            life_block<<<grid, 256, 0, st>>>((const unsigned char *)src, (unsigned char *)dst, g, slot);
            break;
        case SLR_RESTORE8:
            restore_block<<<grid, 256, 0, st>>>((const float *)src, (float *)dst, (const unsigned char *)aux, g,
                                                p.alpha, slot);
            break;
        default:
            switch (p.storage) {
            case SLR_F64:
                if (three)
                    jacobi_block_f64<3><<<grid, 256, 0, st>>>((const double *)src, (double *)dst, (const double *)aux,
                                                               g, p.h2, p.d, p.ghost, slot);
                else
                    jacobi_block_f64<2><<<grid, 256, 0, st>>>((const double *)src, (double *)dst, (const double *)aux,
                                                               g, p.h2, p.d, p.ghost, slot);
                break;
            case SLR_F32:
                if (three)
                    jacobi_block_f32<3, float><<<grid, 256, 0, st>>>((const float *)src, (float *)dst,
                                                                      (const float *)aux, g, p.h2f, p.df, p.ghostf, slot);
                else
                    jacobi_block_f32<2, float><<<grid, 256, 0, st>>>((const float *)src, (float *)dst,
                                                                      (const float *)aux, g, p.h2f, p.df, p.ghostf, slot);
                break;
            case SLR_BF16:
                if (three)
                    jacobi_block_f32<3, __nv_bfloat16><<<grid, 256, 0, st>>>(
                        (const __nv_bfloat16 *)src, (__nv_bfloat16 *)dst, (const __nv_bfloat16 *)aux, g, p.h2f, p.df,
                        p.ghostf, slot);
                else
                    jacobi_block_f32<2, __nv_bfloat16><<<grid, 256, 0, st>>>(
                        (const __nv_bfloat16 *)src, (__nv_bfloat16 *)dst, (const __nv_bfloat16 *)aux, g, p.h2f, p.df,
                        p.ghostf, slot);
                break;
            case SLR_F16:
                if (three)
                    jacobi_block_f32<3, __half><<<grid, 256, 0, st>>>((const __half *)src, (__half *)dst,
                                                                       (const __half *)aux, g, p.h2f, p.df, p.ghostf, slot);
                else
                    jacobi_block_f32<2, __half><<<grid, 256, 0, st>>>((const __half *)src, (__half *)dst,
                                                                       (const __half *)aux, g, p.h2f, p.df, p.ghostf, slot);
                break;
            default: return fail(SLR_ERR_UNSUPPORTED, "storage");
            }
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(SLR_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    return SLR_OK;
}
