// batch.cu -- many loop-of-stencil-reduce instances in one persistent launch.
//
// Each instance is its own loop of Sec. 3.1 (its own grid, stencil, storage,
// reduce, tolerance and iteration cap); one cooperative launch runs a budget
// of sweeps over all instances still running, with one bounded grid barrier
// per sweep for the whole batch.  Work is cut into warp units (a 64 x 16 tile
// of one plane of one instance); the units of all running instances form one
// index space that every warp walks with a grid stride, so small grids no
// longer pay a launch or a barrier each, and large and small grids share the
// machine.  After each sweep every CTA reads the per-instance reduce slots and
// takes the same per-instance decision (test passed, or the instance's cap
// reached); stopped instances drop out of the index space.  At the end of a
// run the state of every stopped instance is in its caller buffer u.
//
// The elemental functions and the evaluation order are those of jacobi.cu,
// restore.cu and dc.cu (EXACT math), so every instance gets the same result
// alone, in a batch, or through slr_create.
//
// A defect-correction instance (FP64 outer loop around FP32 Jacobi inner
// sweeps, dc.cu) advances one phase per batch step: the initial defect, then
// per correction its inner sweeps and the correction with the new defect; its
// test runs after each correction only, and its iteration count is the number
// of corrections.
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "crmath.cuh"
#include "slr_internal.cuh"

namespace slr {
namespace {

constexpr int kBThreads = 256;
constexpr int kTileW = 64, kTileH = 16;
constexpr int kMaxBatch = 1024;
// Jacobi instances whose grid (two states and f in the compute type) fits the
// CTA's staging area are run by one CTA, in shared memory, for all the sweeps
// of a launch, with CTA barriers instead of the grid barrier.

// One instance as the kernel sees it.  Host-written fields first; the kernel
// writes the results at the end of a run (and value/count/converged when the
// instance stops).
struct BInst {
    int stencil, storage, wrap, reduce;
    long long nx, ny, nz;
    double ghost, h2, d, tol;
    float ghostf, h2f, df, alpha;
    void *a, *b;
    const void *aux;
    long long max_iters;
    long long tiles_x, tiles_y, units;
    // results
    long long iters;
    int parity;       // 0: current state in a, 1: in b
    int done;         // stopped (converged or capped)
    int converged;
    int cs;           // > 0: run by a thread-block cluster of cs CTAs (cluster_run), not in batch_kernel
    int pad;
    double value;
    unsigned long long count;
    // defect correction
    int dc;           // 1: FP64 defect correction around binary32 inner sweeps
    int inner;        // inner sweeps per correction
    float *r32, *e0, *e1;   // binary32 defect and correction buffers (in the instance's scratch)
    long long phase;  // phases run so far: 0 the initial defect, then inner + 1 per correction
};

struct BatchArgs {
    BInst *inst;
    Slot *slots;               // [kMaxBatch][kSlots]
    const int *act;            // indices of the running instances
    const long long *prefix;   // unit offsets of act[] (nact + 1 entries)
    int nact;
    long long sweeps;
    Ctl *ctl;                  // barrier counter and error word (reduce slots unused)
    long long limit_ns;
    int nblocks;
};

// Instances run by a thread-block cluster of their own (cluster_run).
struct ClusterArgs {
    BInst *inst;
    const int *list;           // table indices of this launch's instances, one per cluster
    int cs;                    // CTAs per cluster
    long long sweeps;
};

// Jacobi instances (with or without defect correction) of at most
// kMaxCluster * kClusterCells cells run on a cluster of cs CTAs, cs the power
// of two that gives each CTA at most kClusterCells cells (see cluster_run and
// cluster_dc_run).  A defect-correction cell costs several binary64
// operations a phase, so those grids are spread over twice the CTAs.
constexpr int kClusterCells = 4096;
constexpr int kClusterCellsDc = 2048;
constexpr int kMaxCluster = 16;                 // beyond the portable 8: the kernel allows it
constexpr int kClusterGroups = 5;               // cluster sizes 1, 2, 4, 8, 16
constexpr size_t kClusterSmem = 200 * 1024;     // most shared memory a cluster CTA may take

// The cluster size of an instance (0: not run by a cluster) and its CTAs' shared memory.
size_t cluster_smem(const BInst &I, int cs)
{
    const long long planes = I.stencil == SLR_J3D7 ? I.nz : I.ny;
    const long long pc = I.stencil == SLR_J3D7 ? I.nx * I.ny : I.nx;
    // Jacobi: both states and f in the compute type; defect correction: r32, e0, e1
    return 16 + 3 * (size_t)((planes + cs - 1) / cs) * (size_t)pc * (I.storage == SLR_F64 && !I.dc ? 8 : 4);
}
int cluster_size(const BInst &I)
{
    if (I.stencil == SLR_RESTORE8) return 0;
    const long long cells = I.nx * I.ny * I.nz;
    const long long lim = I.dc ? kClusterCellsDc : kClusterCells;
    int cs = 1;
    while (cs < kMaxCluster && cells > cs * lim) cs <<= 1;
    if (cells > cs * lim || cluster_smem(I, cs) > kClusterSmem) return 0;
    return cs;
}

// ---- per-cell elemental functions (same order as jacobi.cu / restore.cu) -----
template <class T> struct St;
template <> struct St<double> {
    using C = double;
    __device__ static C ld(const void *p, long long i) { return __ldcg((const double *)p + i); }
    __device__ static C ldf(const void *p, long long i) { return __ldg((const double *)p + i); }
    __device__ static C put(void *p, long long i, C v) { ((double *)p)[i] = v; return v; }
    __device__ static C rnd(C v) { return v; }
};
template <> struct St<float> {
    using C = float;
    __device__ static C ld(const void *p, long long i) { return __ldcg((const float *)p + i); }
    __device__ static C ldf(const void *p, long long i) { return __ldg((const float *)p + i); }
    __device__ static C put(void *p, long long i, C v) { ((float *)p)[i] = v; return v; }
    __device__ static C rnd(C v) { return v; }
};
template <> struct St<__nv_bfloat16> {
    using C = float;
    __device__ static C ld(const void *p, long long i)
    {
        return __uint_as_float((uint32_t)__ldcg((const unsigned short *)p + i) << 16);
    }
    __device__ static C ldf(const void *p, long long i)
    {
        return __uint_as_float((uint32_t)__ldg((const unsigned short *)p + i) << 16);
    }
    __device__ static C put(void *p, long long i, C v)
    {
        const __nv_bfloat16 s = __float2bfloat16_rn(v);
        ((__nv_bfloat16 *)p)[i] = s;
        return __bfloat162float(s);
    }
    __device__ static C rnd(C v) { return __bfloat162float(__float2bfloat16_rn(v)); }   // to storage and back
};
template <> struct St<__half> {
    using C = float;
    __device__ static C ld(const void *p, long long i)
    {
        return __half2float(__ushort_as_half(__ldcg((const unsigned short *)p + i)));
    }
    __device__ static C ldf(const void *p, long long i)
    {
        return __half2float(__ushort_as_half(__ldg((const unsigned short *)p + i)));
    }
    __device__ static C put(void *p, long long i, C v)
    {
        const __half s = __float2half_rn(v);
        ((__half *)p)[i] = s;
        return __half2float(s);
    }
    __device__ static C rnd(C v) { return __half2float(__float2half_rn(v)); }            // to storage and back
};

__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
// Running max of |delta| as bit patterns (unsigned order = numeric order for
// non-negative values); binary32 deltas stay 32-bit and widen once per unit.
__device__ __forceinline__ void max_bits(unsigned long long &m, double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
    m = b > m ? b : m;
}
__device__ __forceinline__ void max_bits(unsigned int &m, float v)
{
    const unsigned int b = __float_as_uint(fabsf(v));
    m = b > m ? b : m;
}
__device__ __forceinline__ unsigned long long widen_bits(unsigned long long m) { return m; }
__device__ __forceinline__ unsigned long long widen_bits(unsigned int m)
{
    return (unsigned long long)__double_as_longlong((double)__uint_as_float(m));
}
template <class C> struct MaxBits { using type = unsigned long long; };
template <> struct MaxBits<float> { using type = unsigned int; };

template <class T>
__device__ __forceinline__ typename St<T>::C at(const BInst &I, const void *u, long long k, long long i, long long j,
                                                typename St<T>::C ghost)
{
    if (i < 0 || i >= I.ny || j < 0 || j >= I.nx || k < 0 || k >= I.nz) {
        if (!I.wrap) return ghost;
        i = i < 0 ? i + I.ny : (i >= I.ny ? i - I.ny : i);
        j = j < 0 ? j + I.nx : (j >= I.nx ? j - I.nx : j);
        k = k < 0 ? k + I.nz : (k >= I.nz ? k - I.nz : k);
    }
    return St<T>::ld(u, (k * I.ny + i) * I.nx + j);
}

// Per-warp staging of a unit's plane tile with a one-cell halo: (kTileH + 2)
// rows x (kTileW + 2) columns in the compute type, boundary values applied
// while loading (ghost or wrapped neighbour).  Every lane issues its loads
// before any is used, so one warp keeps ~36 loads in flight.
constexpr int kSW = kTileW + 2, kSH = kTileH + 2;

template <class T>
__device__ __forceinline__ void stage_tile(const BInst &I, const void *u, long long k, long long y0, long long x0,
                                           typename St<T>::C *tile, typename St<T>::C ghost)
{
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < kSH; ++r) {
        const long long i = y0 - 1 + r;
        for (int c = lane; c < kSW; c += 32) tile[r * kSW + c] = at<T>(I, u, k, i, x0 - 1 + c, ghost);
    }
    __syncwarp();
}

// One warp unit of a Jacobi instance; returns the unit's max |delta| bits.
template <class T, int DIM>
__device__ unsigned long long jacobi_unit(const BInst &I, long long unit, const void *u, void *v, void *stage)
{
    using C = typename St<T>::C;
    const int lane = threadIdx.x & 31;
    const long long per_plane = I.tiles_x * I.tiles_y;
    const long long k = unit / per_plane, rem = unit - k * per_plane;
    const long long ty = rem / I.tiles_x, tx = rem - ty * I.tiles_x;
    const C ghost = sizeof(C) == 8 ? (C)I.ghost : (C)I.ghostf;
    const C h2 = sizeof(C) == 8 ? (C)I.h2 : (C)I.h2f;
    const C d = sizeof(C) == 8 ? (C)I.d : (C)I.df;
    C *tile = (C *)stage;
    stage_tile<T>(I, u, k, ty * kTileH, tx * kTileW, tile, ghost);
    typename MaxBits<C>::type mx = 0;
    for (int r = 0; r < kTileH; ++r) {
        const long long i = ty * kTileH + r;
        if (i >= I.ny) break;
        for (int c = lane; c < kTileW; c += 32) {
            const long long j = tx * kTileW + c;
            if (j >= I.nx) continue;
            const long long idx = (k * I.ny + i) * I.nx + j;
            const C *t = tile + (r + 1) * kSW + (c + 1);
            const C uc = t[0];
            C s;
            if (DIM == 2) {
                s = add_rn(add_rn(add_rn(t[-kSW], t[kSW]), t[-1]), t[1]);
            } else {
                s = add_rn(add_rn(add_rn(add_rn(add_rn(t[-1], t[1]), t[-kSW]), t[kSW]), at<T>(I, u, k - 1, i, j, ghost)),
                           at<T>(I, u, k + 1, i, j, ghost));
            }
            const C tt = mul_rn(h2, St<T>::ldf(I.aux, idx));
            const C stored = St<T>::put(v, idx, div_rn(add_rn(tt, s), d));
            max_bits(mx, sub_rn(stored, uc));
        }
    }
    __syncwarp();                                   // the stage is reused by the warp's next unit
    return widen_bits(mx);
}

// One warp unit of a restoration instance; returns (fixed-point sum, masked
// count).  Clean pixels are copied; the noisy pixels of each 4-row band are
// gathered with ballots and processed 32 at a time, so the weight arithmetic
// runs on full warps.
__device__ void restore_unit(const BInst &I, long long unit, const void *uv, void *vv, void *stage,
                             unsigned long long &sum, unsigned long long &cnt)
{
    float *v = (float *)vv;
    const unsigned char *mask = (const unsigned char *)I.aux;
    const int lane = threadIdx.x & 31;
    const long long ty = unit / I.tiles_x, tx = unit - ty * I.tiles_x;
    const long long y0 = ty * kTileH, x0 = tx * kTileW;
    float *tile = (float *)stage;
    stage_tile<float>(I, uv, 0, y0, x0, tile, 0.0f);
    for (int band = 0; band < kTileH / 4; ++band) {
        unsigned masks[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int rr = band * 4 + (h >> 1), cc = (h & 1) * 32 + lane;
            const long long y = y0 + rr, x = x0 + cc;
            const bool valid = y < I.ny && x < I.nx;
            const bool noisy = valid && __ldg(mask + y * I.nx + x) != 0;
            if (valid && !noisy) v[y * I.nx + x] = tile[(rr + 1) * kSW + cc + 1];
            masks[h] = __ballot_sync(0xffffffffu, noisy);
        }
        int total = 0;
#pragma unroll
        for (int h = 0; h < 8; ++h) total += __popc(masks[h]);
        for (int first = 0; first < total; first += 32) {
            const int t = first + lane;
            if (t >= total) continue;
            int h = 0, before = 0;
#pragma unroll
            for (int g = 0; g < 7; ++g) {
                const int c = __popc(masks[g]);
                if (h == g && t >= before + c) { before += c; h = g + 1; }
            }
            unsigned mh = 0u;
#pragma unroll
            for (int g = 0; g < 8; ++g)
                if (g == h) mh = masks[g];
            const unsigned fb = __fns(mh, 0u, t - before + 1);   // bit of the (t - before)-th noisy pixel
            if (fb > 31u) continue;                                // cannot happen: t < total
            const int bit = (int)fb;
            const int rr = band * 4 + (h >> 1), cc = (h & 1) * 32 + bit;
            const long long y = y0 + rr, x = x0 + cc;
            const float uc = tile[(rr + 1) * kSW + cc + 1];
            float num = 0.0f, den = 0.0f;
            const bool inner = y > 0 && y + 1 < I.ny && x > 0 && x + 1 < I.nx;
#pragma unroll
            for (int di = -1; di <= 1; ++di)
#pragma unroll
                for (int dj = -1; dj <= 1; ++dj) {
                    if (di == 0 && dj == 0) continue;
                    if (!inner && (y + di < 0 || y + di >= I.ny || x + dj < 0 || x + dj >= I.nx)) continue;
                    const float uj = tile[(rr + 1 + di) * kSW + cc + 1 + dj];
                    const float tt = __fsub_rn(uc, uj);
                    const float w = inv_sqrt_rn2(__fadd_rn(I.alpha, __fmul_rn(tt, tt)));
                    num = __fadd_rn(num, __fmul_rn(w, uj));
                    den = __fadd_rn(den, w);
                }
            const float nv = den > 0.0f ? __fdiv_rn(num, den) : uc;
            v[y * I.nx + x] = nv;
            sum += fixed_2m24(__fsub_rn(nv, uc));
            cnt += 1ull;
        }
    }
    __syncwarp();
}

// ---- defect correction (the operations and order of dc.cu) ----------------------
__device__ __forceinline__ bool dc_outside(const BInst &I, long long k, long long i, long long j)
{
    return k < 0 || k >= I.nz || i < 0 || i >= I.ny || j < 0 || j >= I.nx;
}

template <int DIM, class T, class V>
__device__ __forceinline__ T dc_sum(long long k, long long i, long long j, V val)
{
    if (DIM == 2)
        return add_rn(add_rn(add_rn(val(k, i - 1, j), val(k, i + 1, j)), val(k, i, j - 1)), val(k, i, j + 1));
    return add_rn(add_rn(add_rn(add_rn(add_rn(val(k, i, j - 1), val(k, i, j + 1)), val(k, i - 1, j)), val(k, i + 1, j)),
                         val(k - 1, i, j)),
                  val(k + 1, i, j));
}

// r = f - A v at (k, i, j), v read through `val` (ghost 0)
template <int DIM, class V>
__device__ __forceinline__ double dc_defect(const BInst &I, long long k, long long i, long long j, V val)
{
    const double sm = dc_sum<DIM, double>(k, i, j, val);
    const double au = __ddiv_rn(__dsub_rn(__dmul_rn(I.d, val(k, i, j)), sm), I.h2);
    return __dsub_rn(__ldg((const double *)I.aux + (k * I.ny + i) * I.nx + j), au);
}

// One warp unit of phase q of a defect-correction instance: q = 0 the
// initial defect r32 = f - A u; then, per correction n, phases 0 .. inner-1
// the binary32 sweeps of A e = r32 from e = 0 and phase inner the correction
// u' = u + e with its new defect; returns the correction's max |h2 r / d| as
// bits (0 in the other phases).
template <int DIM>
__device__ unsigned long long dc_unit(const BInst &I, long long unit, long long q)
{
    const int lane = threadIdx.x & 31;
    const long long per_plane = I.tiles_x * I.tiles_y;
    const long long k = unit / per_plane, rem = unit - k * per_plane;
    const long long ty = rem / I.tiles_x, tx = rem - ty * I.tiles_x;
    const long long P = I.inner + 1;
    const long long n = q >= 1 ? (q - 1) / P : 0;
    const int ph = q >= 1 ? (int)((q - 1) % P) : -1;
    const double *uo = (const double *)((n & 1) ? I.b : I.a);
    double *un = (double *)((n & 1) ? I.a : I.b);
    const float *es = (ph & 1) ? I.e1 : I.e0;
    float *ed = (ph & 1) ? I.e0 : I.e1;
    const float *ec = (I.inner & 1) ? I.e1 : I.e0;          // e after the inner sweeps
    unsigned long long mx = 0ull;
    for (int r = 0; r < kTileH; ++r) {
        const long long i = ty * kTileH + r;
        if (i >= I.ny) break;
        for (int c = lane; c < kTileW; c += 32) {
            const long long j = tx * kTileW + c;
            if (j >= I.nx) continue;
            const long long idx = (k * I.ny + i) * I.nx + j;
            if (ph < 0) {
                const double rv = dc_defect<DIM>(I, k, i, j, [&](long long z, long long y, long long x) {
                    return dc_outside(I, z, y, x) ? 0.0 : __ldcg(uo + (z * I.ny + y) * I.nx + x);
                });
                I.r32[idx] = (float)rv;
            } else if (ph < I.inner) {
                float sn = 0.0f;
                if (ph > 0)
                    sn = dc_sum<DIM, float>(k, i, j, [&](long long z, long long y, long long x) {
                        return dc_outside(I, z, y, x) ? 0.0f : __ldcg(es + (z * I.ny + y) * I.nx + x);
                    });
                const float t = __fmul_rn(I.h2f, __ldcg(I.r32 + idx));
                ed[idx] = __fdiv_rn(__fadd_rn(t, sn), I.df);
            } else {
                un[idx] = __dadd_rn(__ldcg(uo + idx), (double)__ldcg(ec + idx));
                const double rv = dc_defect<DIM>(I, k, i, j, [&](long long z, long long y, long long x) {
                    if (dc_outside(I, z, y, x)) return 0.0;
                    const long long qx = (z * I.ny + y) * I.nx + x;
                    return __dadd_rn(__ldcg(uo + qx), (double)__ldcg(ec + qx));
                });
                I.r32[idx] = (float)rv;
                const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(__ddiv_rn(__dmul_rn(I.h2, rv), I.d)));
                mx = b > mx ? b : mx;
            }
        }
    }
    return mx;
}

// corrections completed after `phases` phases of a defect-correction instance
__device__ __forceinline__ long long dc_corrections(const BInst &I, long long phases)
{
    return phases >= 1 ? (phases - 1) / (I.inner + 1) : 0;
}

__device__ void unit_copy(const BInst &I, long long unit, const void *src, void *dst)
{
    const int lane = threadIdx.x & 31;
    const size_t es = I.storage == SLR_F64 ? 8 : (I.storage == SLR_F32 ? 4 : 2);
    const long long per_plane = I.tiles_x * I.tiles_y;
    const long long k = unit / per_plane, rem = unit - k * per_plane;
    const long long ty = rem / I.tiles_x, tx = rem - ty * I.tiles_x;
    for (int r = 0; r < kTileH; ++r) {
        const long long i = ty * kTileH + r;
        if (i >= I.ny) break;
        for (int c = lane; c < kTileW; c += 32) {
            const long long j = tx * kTileW + c;
            if (j >= I.nx) continue;
            const long long idx = (k * I.ny + i) * I.nx + j;
            if (es == 8) ((double *)dst)[idx] = __ldcg((const double *)src + idx);
            else if (es == 4) ((float *)dst)[idx] = __ldcg((const float *)src + idx);
            else ((unsigned short *)dst)[idx] = __ldcg((const unsigned short *)src + idx);
        }
    }
}

__device__ __forceinline__ int find_instance(const long long *prefix, int n, long long u)
{
    int lo = 0, hi = n;     // prefix[lo] <= u < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= u) lo = mid; else hi = mid;
    }
    return lo;
}

constexpr size_t kStageBytesPerWarp = (size_t)kSW * kSH * 8;      // binary64 worst case

// Rebuild this CTA's list of running instances (s_aidx) and the exclusive
// prefix of their unit counts (s_upref, n_run + 1 entries) from s_stop; every
// CTA holds the same decisions, so every CTA builds the same list.  Returns
// the number of running instances.
__device__ int compact_running(int n, const int *s_stop, const int *s_units, int *s_aidx, int *s_upref)
{
    __shared__ int s_wsum_n[kBThreads / 32], s_wsum_u[kBThreads / 32];
    __shared__ int s_total_n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + kBThreads - 1) / kBThreads;
    const int lo = tid * per, hi = lo + per < n ? lo + per : n;
    int cn = 0, cu = 0;
    for (int i = lo; i < hi; ++i)
        if (s_stop[i] == -1) { ++cn; cu += s_units[i]; }
    // block exclusive scan of (cn, cu)
    int sn = cn, su = cu;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int tn = __shfl_up_sync(0xffffffffu, sn, o), tu = __shfl_up_sync(0xffffffffu, su, o);
        if (lane >= o) { sn += tn; su += tu; }
    }
    if (lane == 31) { s_wsum_n[warp] = sn; s_wsum_u[warp] = su; }
    __syncthreads();
    if (warp == 0) {
        int wn = lane < kBThreads / 32 ? s_wsum_n[lane] : 0, wu = lane < kBThreads / 32 ? s_wsum_u[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int tn = __shfl_up_sync(0xffffffffu, wn, o), tu = __shfl_up_sync(0xffffffffu, wu, o);
            if (lane >= o) { wn += tn; wu += tu; }
        }
        if (lane < kBThreads / 32) { s_wsum_n[lane] = wn; s_wsum_u[lane] = wu; }
        if (lane == kBThreads / 32 - 1) s_total_n = wn;
    }
    __syncthreads();
    int pn = sn - cn + (warp > 0 ? s_wsum_n[warp - 1] : 0);
    int pu = su - cu + (warp > 0 ? s_wsum_u[warp - 1] : 0);
    for (int i = lo; i < hi; ++i)
        if (s_stop[i] == -1) {
            s_aidx[pn] = i;
            s_upref[pn] = pu;
            ++pn;
            pu += s_units[i];
        }
    const int total = s_total_n;
    if (tid == kBThreads - 1) s_upref[total] = pu;   // the last thread ends on the total
    __syncthreads();
    return total;
}

__device__ __forceinline__ int find_running(const int *s_upref, int nrun, int u)
{
    int lo = 0, hi = nrun;     // s_upref[lo] <= u < s_upref[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_upref[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

namespace cg = cooperative_groups;

// A Jacobi instance run by one thread-block cluster of cs CTAs with the grid
// in their shared memory: CTA r holds the rows (2D) or planes (3D)
// [r * per, (r + 1) * per) of both states and of f, in the compute type.  A
// sweep updates the CTA's own cells, reading neighbours held by the other
// CTAs through distributed shared memory, with the same operations in the
// same order as jacobi_unit; the CTA's max |delta| goes to a per-parity
// shared word; one cluster barrier then makes the new states and the maxima
// visible, and every CTA reads the cs maxima and takes the same decision, so
// the CTAs stop together at the sweep the instance would stop at in the
// batch-wide loop.  The final state goes back to a (parity 0).  No CTA
// leaves before the others are done reading its shared memory.
template <class T, int DIM>
__device__ void cluster_run(BInst &Ig, int cs, long long sweeps, unsigned char *smem)
{
    using C = typename St<T>::C;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ unsigned long long s_wmax[2][kBThreads / 32];   // per sweep parity, one word per warp
    const BInst I = Ig;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = (int)cl.block_rank();
    const C ghost = sizeof(C) == 8 ? (C)I.ghost : (C)I.ghostf;
    const C h2 = sizeof(C) == 8 ? (C)I.h2 : (C)I.h2f;
    const C d = sizeof(C) == 8 ? (C)I.d : (C)I.df;
    const int nx = (int)I.nx, ny = (int)I.ny, nz = (int)I.nz;
    const bool wrap = I.wrap != 0;
    const int planes = DIM == 3 ? nz : ny, pc = DIM == 3 ? nx * ny : nx;   // partition unit and its cells
    const int per = (planes + cs - 1) / cs;
    const int p0 = min(rank * per, planes), p1 = min(p0 + per, planes);
    const int own = (p1 - p0) * pc;
    C *buf0 = (C *)smem, *buf1 = buf0 + (size_t)per * pc, *fs = buf1 + (size_t)per * pc;
    const int par0 = I.parity;
    const void *g0 = par0 ? I.b : I.a;
    for (int c = tid; c < own; c += kBThreads) {
        buf0[c] = St<T>::ld(g0, (long long)p0 * pc + c);
        fs[c] = St<T>::ldf(I.aux, (long long)p0 * pc + c);
    }
    cl.sync();                                        // every CTA's part is loaded
    // row (k, i) of the buffer whose local copy is `base`, in whichever CTA
    // holds plane k (row i in 2D); null outside the grid unless it wraps
    auto row_at = [&](const C *base, int k, int i) -> const C * {
        if (i < 0 || i >= ny || k < 0 || k >= nz) {
            if (!wrap) return nullptr;
            i = i < 0 ? i + ny : (i >= ny ? i - ny : i);
            k = k < 0 ? k + nz : (k >= nz ? k - nz : k);
        }
        const int pl = DIM == 3 ? k : i;
        if (pl >= p0 && pl < p1)
            return base + (DIM == 3 ? ((k - p0) * ny + i) * nx : (i - p0) * nx);
        const int r = pl / per;
        return cl.map_shared_rank((C *)base, r) + (DIM == 3 ? ((k - r * per) * ny + i) * nx : (i - r * per) * nx);
    };
    long long it = I.iters;
    int cur = 0;
    bool stop = false;
    Decision dcs;
    dcs.value = 0.0; dcs.count = 0ull; dcs.changed = 0; dcs.converged = 0;
    for (long long s = 0; s < sweeps && !stop; ++s) {
        C *v = cur ? buf0 : buf1;
        const C *u = cur ? buf1 : buf0;
        typename MaxBits<C>::type mx = 0;
        // one cell: the neighbours in the order of jacobi_unit
        auto cell = [&](const C *rc, const C *fr, C *vr, int j, C n, C so, C bl, C ab) {
            const C uc = rc[j];
            // the x-neighbours by index (wrapped, or the cell itself where the ghost goes)
            C w = rc[j > 0 ? j - 1 : (wrap ? nx - 1 : j)];
            C e = rc[j + 1 < nx ? j + 1 : (wrap ? 0 : j)];
            if (!wrap) {
                w = j > 0 ? w : ghost;
                e = j + 1 < nx ? e : ghost;
            }
            C sum;
            if (DIM == 2)
                sum = add_rn(add_rn(add_rn(n, so), w), e);
            else
                sum = add_rn(add_rn(add_rn(add_rn(add_rn(w, e), n), so), bl), ab);
            const C tt = mul_rn(h2, fr[j]);
            // the value rounded to the storage type, widened back (exact)
            const C stored = St<T>::rnd(div_rn(add_rn(tt, sum), d));
            vr[j] = stored;
            max_bits(mx, sub_rn(stored, uc));
        };
        // warp per row of the CTA's part (rows of its planes in 3D), lanes
        // across x; rows whose neighbouring rows are all this CTA's and inside
        // the grid read them at fixed offsets, the others find them once per row
        const int nrows = (p1 - p0) * (DIM == 3 ? ny : 1);
        for (int row = warp; row < nrows; row += kBThreads / 32) {
            const int k = DIM == 3 ? p0 + row / ny : 0;
            const int i = DIM == 3 ? row - (row / ny) * ny : p0 + row;
            const C *rc = u + row * nx;
            const C *fr = fs + row * nx;
            C *vr = v + row * nx;
            const bool inner = DIM == 2 ? (i - 1 >= p0 && i + 1 < p1)
                                        : (k - 1 >= p0 && k + 1 < p1 && i >= 1 && i + 1 < ny);
            if (inner) {
                const int pz = ny * nx;
                for (int j = lane; j < nx; j += 32)
                    cell(rc, fr, vr, j, rc[j - nx], rc[j + nx], DIM == 3 ? rc[j - pz] : ghost,
                         DIM == 3 ? rc[j + pz] : ghost);
            } else {
                const C *rn = row_at(u, k, i - 1), *rs = row_at(u, k, i + 1);
                const C *rb = DIM == 3 ? row_at(u, k - 1, i) : nullptr, *ra = DIM == 3 ? row_at(u, k + 1, i) : nullptr;
                for (int j = lane; j < nx; j += 32)
                    cell(rc, fr, vr, j, rn ? rn[j] : ghost, rs ? rs[j] : ghost, rb ? rb[j] : ghost,
                         ra ? ra[j] : ghost);
            }
        }
        unsigned long long m = widen_bits(mx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
            m = t > m ? t : m;
        }
        if (lane == 0) s_wmax[s & 1][warp] = m;
        // the new states and every warp's maximum, cluster-wide; the words of
        // this parity are written again two sweeps on, after the next barrier,
        // which no CTA passes before all have read them
        cl.sync();
        unsigned long long b = 0ull;
        for (int x = lane; x < cs * (kBThreads / 32); x += 32) {
            const unsigned long long y = *cl.map_shared_rank(&s_wmax[s & 1][x % (kBThreads / 32)], x / (kBThreads / 32));
            b = y > b ? y : b;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
            b = t > b ? t : b;
        }
        Slot sl;
        memset(&sl, 0, sizeof(sl));
        sl.maxbits = b;
        sl.changed = b != 0ull;
        dcs = decide(I.reduce, sl, I.tol);
        it += 1;
        cur ^= 1;
        stop = dcs.converged || it >= I.max_iters;
    }
    const C *fin = cur ? buf1 : buf0;
    for (int c = tid; c < own; c += kBThreads) St<T>::put(I.a, (long long)p0 * pc + c, fin[c]);
    if (rank == 0 && tid == 0) {
        Ig.iters = it;
        Ig.parity = 0;
        Ig.done = stop;
        if (stop) {
            Ig.value = dcs.value;
            Ig.count = dcs.count;
            Ig.converged = dcs.converged;
        }
    }
    cl.sync();                                        // the others' last reads of this CTA's memory are done
}

// A defect-correction instance run by one thread-block cluster, phase by
// phase as dc_unit runs it in the batch-wide loop (the same operations in the
// same order): the binary32 defect r32 and the corrections e0, e1 of the
// CTA's rows or planes live in its shared memory for the launch (loaded at
// its start and stored at its end, so that a later launch resumes at the same
// phase), the binary64 state and f in global memory.  One cluster barrier per
// phase orders both; the scaled defect's maximum is taken over the cluster at
// the correction phases, where the test runs.
template <int DIM>
__device__ void cluster_dc_run(BInst &Ig, int cs, long long sweeps, unsigned char *smem)
{
    cg::cluster_group cl = cg::this_cluster();
    __shared__ unsigned long long s_wmax[2][kBThreads / 32];   // per phase parity, one word per warp
    const BInst I = Ig;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = (int)cl.block_rank();
    const int nx = (int)I.nx, ny = (int)I.ny, nz = (int)I.nz;
    const int planes = DIM == 3 ? nz : ny, pc = DIM == 3 ? nx * ny : nx;
    const int per = (planes + cs - 1) / cs;
    const int p0 = min(rank * per, planes), p1 = min(p0 + per, planes);
    const int own = (p1 - p0) * pc;
    const long long base = (long long)p0 * pc;
    float *sr = (float *)smem, *se0 = sr + (size_t)per * pc, *se1 = se0 + (size_t)per * pc;
    for (int c = tid; c < own; c += kBThreads) {
        sr[c] = __ldcg(I.r32 + base + c);
        se0[c] = __ldcg(I.e0 + base + c);
        se1[c] = __ldcg(I.e1 + base + c);
    }
    cl.sync();
    // cell (k, i, j) of one of the shared arrays, wherever it is held
    auto at = [&](float *arr, long long k, long long i, long long j) -> float {
        const int pl = (int)(DIM == 3 ? k : i);
        if (pl >= p0 && pl < p1)                     // held by this CTA: no division
            return arr[DIM == 3 ? (int)(((k - p0) * ny + i) * nx + j) : (int)((i - p0) * nx + j)];
        const int r = pl / per;
        const int off = DIM == 3 ? (int)(((k - r * per) * ny + i) * nx + j) : (int)((i - r * per) * nx + j);
        return cl.map_shared_rank(arr, r)[off];
    };
    // row (k, i) of one of the shared arrays in whichever CTA holds it; null
    // outside the grid (the corrections' ghost is 0)
    auto row_of = [&](float *arr, int k, int i) -> const float * {
        if (i < 0 || i >= ny || k < 0 || k >= nz) return nullptr;
        const int pl = DIM == 3 ? k : i;
        if (pl >= p0 && pl < p1) return arr + (DIM == 3 ? ((k - p0) * ny + i) * nx : (i - p0) * nx);
        const int r = pl / per;
        return cl.map_shared_rank(arr, r) + (DIM == 3 ? ((k - r * per) * ny + i) * nx : (i - r * per) * nx);
    };
    const long long P = I.inner + 1, q0 = I.phase;
    const float *ec = (I.inner & 1) ? se1 : se0;            // e after the inner sweeps
    bool stop = false;
    long long s = 0;
    Decision dcs;
    dcs.value = 0.0; dcs.count = 0ull; dcs.changed = 0; dcs.converged = 0;
    for (; s < sweeps && !stop; ++s) {
        const long long q = q0 + s;
        const long long n = q >= 1 ? (q - 1) / P : 0;
        const int ph = q >= 1 ? (int)((q - 1) % P) : -1;
        const double *uo = (const double *)((n & 1) ? I.b : I.a);
        double *un = (double *)((n & 1) ? I.a : I.b);
        float *es = (ph & 1) ? se1 : se0;
        float *ed = (ph & 1) ? se0 : se1;
        unsigned long long mx = 0ull;
        // warp per row of the CTA's part (rows of its planes in 3D), lanes across x
        const int nrows = (p1 - p0) * (DIM == 3 ? ny : 1);
        for (int row = warp; row < nrows; row += kBThreads / 32) {
            if (ph >= 0 && ph < I.inner) {
                // an inner binary32 sweep: the neighbouring rows of e found once per row
                const int kk = DIM == 3 ? p0 + row / ny : 0;
                const int ii = DIM == 3 ? row - (row / ny) * ny : p0 + row;
                const float *rc = es + row * nx, *rr = sr + row * nx;
                float *rd = ed + row * nx;
                const bool sum = ph > 0;
                const float *rn = sum ? row_of(es, kk, ii - 1) : nullptr, *rs = sum ? row_of(es, kk, ii + 1) : nullptr;
                const float *rb = sum && DIM == 3 ? row_of(es, kk - 1, ii) : nullptr;
                const float *ra = sum && DIM == 3 ? row_of(es, kk + 1, ii) : nullptr;
                for (int j = lane; j < nx; j += 32) {
                    float sn = 0.0f;
                    if (sum) {
                        // the neighbours in the order of dc_sum; 0 outside the grid
                        float w = rc[j > 0 ? j - 1 : j], e = rc[j + 1 < nx ? j + 1 : j];
                        w = j > 0 ? w : 0.0f;
                        e = j + 1 < nx ? e : 0.0f;
                        const float n = rn ? rn[j] : 0.0f, so = rs ? rs[j] : 0.0f;
                        if (DIM == 2) {
                            sn = __fadd_rn(__fadd_rn(__fadd_rn(n, so), w), e);
                        } else {
                            const float bl = rb ? rb[j] : 0.0f, ab = ra ? ra[j] : 0.0f;
                            sn = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(w, e), n), so), bl), ab);
                        }
                    }
                    const float t = __fmul_rn(I.h2f, rr[j]);
                    rd[j] = __fdiv_rn(__fadd_rn(t, sn), I.df);
                }
                continue;
            }
            for (int jj = lane; jj < nx; jj += 32) {
                const long long k = DIM == 3 ? p0 + row / ny : 0;
                const long long i = DIM == 3 ? row - (row / ny) * ny : p0 + row;
                const long long j = jj;
                const int c = row * nx + jj;
                const long long idx = base + c;
                if (ph < 0) {
                    const double rv = dc_defect<DIM>(I, k, i, j, [&](long long z, long long y, long long x) {
                        return dc_outside(I, z, y, x) ? 0.0 : __ldcg(uo + (z * I.ny + y) * I.nx + x);
                    });
                    sr[c] = (float)rv;
                } else {
                    un[idx] = __dadd_rn(__ldcg(uo + idx), (double)ec[c]);
                    const double rv = dc_defect<DIM>(I, k, i, j, [&](long long z, long long y, long long x) {
                        if (dc_outside(I, z, y, x)) return 0.0;
                        return __dadd_rn(__ldcg(uo + (z * I.ny + y) * I.nx + x), (double)at((float *)ec, z, y, x));
                    });
                    sr[c] = (float)rv;
                    const unsigned long long b =
                        (unsigned long long)__double_as_longlong(fabs(__ddiv_rn(__dmul_rn(I.h2, rv), I.d)));
                    mx = b > mx ? b : mx;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = t > mx ? t : mx;
        }
        if (lane == 0) s_wmax[s & 1][warp] = mx;
        // this phase's values (shared and global) and every warp's maximum,
        // cluster-wide; the words of this parity are written again two phases
        // on, after the next barrier, which no CTA passes before all have read them
        cl.sync();
        const bool tested = q >= 1 && ph == I.inner;
        if (tested) {
            unsigned long long b = 0ull;
            for (int x = lane; x < cs * (kBThreads / 32); x += 32) {
                const unsigned long long y =
                    *cl.map_shared_rank(&s_wmax[s & 1][x % (kBThreads / 32)], x / (kBThreads / 32));
                b = y > b ? y : b;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
                b = t > b ? t : b;
            }
            Slot sl;
            memset(&sl, 0, sizeof(sl));
            sl.maxbits = b;
            dcs = decide(I.reduce, sl, I.tol);
            stop = dcs.converged || dc_corrections(I, q + 1) >= I.max_iters;
        }
    }
    const long long phase = q0 + s;
    const long long iters = dc_corrections(I, phase);
    for (int c = tid; c < own; c += kBThreads) {
        I.r32[base + c] = sr[c];
        I.e0[base + c] = se0[c];
        I.e1[base + c] = se1[c];
    }
    if (stop && (iters & 1)) {
        // the final state is in b: into a
        for (int c = tid; c < own; c += kBThreads) ((double *)I.a)[base + c] = __ldcg((const double *)I.b + base + c);
    }
    if (rank == 0 && tid == 0) {
        Ig.phase = phase;
        Ig.iters = iters;
        Ig.parity = stop ? 0 : (int)(iters & 1);
        Ig.done = stop;
        if (stop) {
            Ig.value = dcs.value;
            Ig.count = dcs.count;
            Ig.converged = dcs.converged;
        }
    }
    cl.sync();                                        // the others' last reads of this CTA's memory are done
}

__global__ void __launch_bounds__(kBThreads, 4) batch_cluster_kernel(ClusterArgs ca)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = align_up(smem_raw, 16);
    BInst &I = ca.inst[ca.list[blockIdx.x / ca.cs]];
    const bool d3 = I.stencil == SLR_J3D7;
    if (I.dc) {
        d3 ? cluster_dc_run<3>(I, ca.cs, ca.sweeps, smem) : cluster_dc_run<2>(I, ca.cs, ca.sweeps, smem);
        return;
    }
    switch (I.storage) {
    case SLR_F64: d3 ? cluster_run<double, 3>(I, ca.cs, ca.sweeps, smem) : cluster_run<double, 2>(I, ca.cs, ca.sweeps, smem); break;
    case SLR_F32: d3 ? cluster_run<float, 3>(I, ca.cs, ca.sweeps, smem) : cluster_run<float, 2>(I, ca.cs, ca.sweeps, smem); break;
    case SLR_BF16:
        d3 ? cluster_run<__nv_bfloat16, 3>(I, ca.cs, ca.sweeps, smem) : cluster_run<__nv_bfloat16, 2>(I, ca.cs, ca.sweeps, smem);
        break;
    default: d3 ? cluster_run<__half, 3>(I, ca.cs, ca.sweeps, smem) : cluster_run<__half, 2>(I, ca.cs, ca.sweeps, smem); break;
    }
}

__global__ void __launch_bounds__(kBThreads, 2) batch_kernel(BatchArgs ba)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *stage = smem_raw + (size_t)(threadIdx.x >> 5) * kStageBytesPerWarp;
    unsigned char *tail = smem_raw + (size_t)(kBThreads / 32) * kStageBytesPerWarp;
    const int n = ba.nact;
    long long *s_iters0 = (long long *)tail;                      // [n]
    long long *s_phase0 = s_iters0 + n;                           // [n]: defect correction's phases so far
    int *s_stop = (int *)(s_phase0 + n);                          // [n]: sweep index of the stop, -1 running
    int *s_units = s_stop + n;                                    // [n]
    int *s_aidx = s_units + n;                                    // [n]: running instances (positions in act)
    int *s_upref = s_aidx + n;                                    // [n + 1]: unit prefix of s_aidx
    unsigned char *s_par0 = (unsigned char *)(s_upref + n + 1);   // [n]
    __shared__ int s_alive;

    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < n; i += kBThreads) {
        const BInst &I = ba.inst[ba.act[i]];
        s_iters0[i] = I.iters;
        s_phase0[i] = I.phase;
        s_par0[i] = (unsigned char)I.parity;
        s_stop[i] = I.done ? -2 : -1;
        s_units[i] = (int)I.units;
    }
    __syncthreads();
    int nrun = compact_running(n, s_stop, s_units, s_aidx, s_upref);
    const int G = (int)gridDim.x;                      // CTAs of the batch-wide loop
    // warps interleave across CTAs so that consecutive units land on different SMs
    const int warps = G * (kBThreads / 32);
    const int gw = (tid >> 5) * G + (int)blockIdx.x;
    long long s = 0;
    for (; s < ba.sweeps; ++s) {
        const int U = s_upref[nrun];
        for (int u = gw; u < U; u += warps) {
            const int ri = find_running(s_upref, nrun, u);
            const int ai = s_aidx[ri];
            const BInst &I = ba.inst[ba.act[ai]];
            const long long unit = u - s_upref[ri];
            const int par = (s_par0[ai] + (int)s) & 1;
            const void *src = par ? I.b : I.a;
            void *dst = par ? I.a : I.b;
            Slot *slot = &ba.slots[(size_t)ba.act[ai] * kSlots + (size_t)(s % kSlots)];
            if (I.dc) {
                unsigned long long mx = I.stencil == SLR_J3D7 ? dc_unit<3>(I, unit, s_phase0[ai] + s)
                                                              : dc_unit<2>(I, unit, s_phase0[ai] + s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
                    mx = m2 > mx ? m2 : mx;
                }
                if (lane == 0 && mx) atomicMax(&slot->maxbits, mx);
            } else if (I.stencil == SLR_RESTORE8) {
                unsigned long long sum = 0ull, cnt = 0ull;
                restore_unit(I, unit, src, dst, stage, sum, cnt);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sum += __shfl_xor_sync(0xffffffffu, sum, o);
                    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                }
                if (lane == 0) {
                    if (sum) atomicAdd(&slot->sum, sum);
                    if (cnt) atomicAdd(&slot->cnt, cnt);
                    if (sum) atomicOr(&slot->changed, 1u);
                }
            } else {
                unsigned long long mx = 0ull;
                const bool d3 = I.stencil == SLR_J3D7;
                switch (I.storage) {
                case SLR_F64: mx = d3 ? jacobi_unit<double, 3>(I, unit, src, dst, stage) : jacobi_unit<double, 2>(I, unit, src, dst, stage); break;
                case SLR_F32: mx = d3 ? jacobi_unit<float, 3>(I, unit, src, dst, stage) : jacobi_unit<float, 2>(I, unit, src, dst, stage); break;
                case SLR_BF16:
                    mx = d3 ? jacobi_unit<__nv_bfloat16, 3>(I, unit, src, dst, stage) : jacobi_unit<__nv_bfloat16, 2>(I, unit, src, dst, stage);
                    break;
                default: mx = d3 ? jacobi_unit<__half, 3>(I, unit, src, dst, stage) : jacobi_unit<__half, 2>(I, unit, src, dst, stage); break;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
                    mx = m2 > mx ? m2 : mx;
                }
                if (lane == 0 && mx) {
                    atomicMax(&slot->maxbits, mx);
                    atomicOr(&slot->changed, 1u);
                }
            }
        }
        if (!grid_barrier(ba.ctl, (unsigned long long)(s + 1) * (unsigned long long)G, ba.limit_ns))
            return;
        // every CTA takes the same per-instance decision
        if (tid == 0) s_alive = 0;
        __syncthreads();
        int alive = 0;
        for (int r = tid; r < nrun; r += kBThreads) {
            const int i = s_aidx[r];
            const int gi = ba.act[i];
            const Slot sl = read_slot(&ba.slots[(size_t)gi * kSlots + (size_t)(s % kSlots)]);
            BInst &I = ba.inst[gi];
            const Decision dcs = decide(I.reduce, sl, I.tol);
            long long it = s_iters0[i] + s + 1;
            bool tested = true;
            if (I.dc) {
                // the test follows the corrections only
                const long long q = s_phase0[i] + s;
                tested = q >= 1 && (q - 1) % (I.inner + 1) == I.inner;
                it = dc_corrections(I, q + 1);
            }
            if (tested && (dcs.converged || it >= I.max_iters)) {
                s_stop[i] = (int)s;
                if (blockIdx.x == 0) {
                    I.value = dcs.value;
                    I.count = dcs.count;
                    I.converged = dcs.converged;
                }
            } else {
                alive = 1;
            }
            if (blockIdx.x == 0) zero_slot(&ba.slots[(size_t)gi * kSlots + (size_t)((s + 2) % kSlots)]);
        }
        if (alive) s_alive = 1;
        __syncthreads();
        if (!s_alive) { ++s; break; }
        nrun = compact_running(n, s_stop, s_units, s_aidx, s_upref);
    }
    const long long ran = s < ba.sweeps ? s : ba.sweeps;
    // results (CTA 0) and the write-back of stopped instances whose state is in b
    if (blockIdx.x == 0) {
        for (int i = tid; i < n; i += kBThreads) {
            if (s_stop[i] == -2) continue;
            BInst &I = ba.inst[ba.act[i]];
            const long long done_sweeps = s_stop[i] >= 0 ? s_stop[i] + 1 : ran;
            if (I.dc) {
                I.phase = s_phase0[i] + done_sweeps;
                I.iters = dc_corrections(I, I.phase);
                I.parity = (int)(I.iters & 1);
            } else {
                I.iters = s_iters0[i] + done_sweeps;
                I.parity = (s_par0[i] + (int)done_sweeps) & 1;
            }
            I.done = s_stop[i] >= 0;
        }
    }
    const long long U0 = __ldg(ba.prefix + n);
    for (long long u = gw; u < U0; u += warps) {
        const int ai = find_instance(ba.prefix, n, u);
        if (s_stop[ai] < 0) continue;
        const BInst &I = ba.inst[ba.act[ai]];
        if (I.dc) {
            if ((dc_corrections(I, s_phase0[ai] + s_stop[ai] + 1) & 1) == 0) continue;   // final state in a
        } else if (((s_par0[ai] + s_stop[ai] + 1) & 1) == 0) {
            continue;                                                // final state already in a
        }
        unit_copy(I, u - __ldg(ba.prefix + ai), I.b, I.a);
    }
}

}  // namespace
}  // namespace slr

using slr::BInst;

struct slr_batch_ctx {
    int max_inst;
    unsigned char *ws;
    cudaStream_t stream;
    std::vector<BInst> inst;     // host mirror
    std::vector<int> used;       // slot in use
    std::vector<int> reported;   // finished and already returned by poll
    std::string err;
    bool dirty;                  // host mirror newer than the device table
    // side streams of the cluster launches (one per cluster size, created on
    // first use) and their completion events, which `stream` waits for
    cudaStream_t side[slr::kClusterGroups] = {};
    cudaEvent_t done[slr::kClusterGroups] = {};
    ~slr_batch_ctx()
    {
        for (int i = 0; i < slr::kClusterGroups; ++i) {
            if (done[i]) cudaEventDestroy(done[i]);
            if (side[i]) cudaStreamDestroy(side[i]);
        }
    }
};

namespace {

thread_local std::string g_batch_create_error = "no error";

size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }
size_t off_inst() { return rup(sizeof(slr::Ctl), 256); }
size_t off_slots(int m) { return off_inst() + rup((size_t)m * sizeof(BInst), 256); }
size_t off_act(int m) { return off_slots(m) + rup((size_t)m * slr::kSlots * sizeof(slr::Slot), 256); }
size_t off_prefix(int m) { return off_act(m) + rup((size_t)m * sizeof(int), 256); }
size_t ws_total(int m) { return off_prefix(m) + rup((size_t)(m + 1) * sizeof(long long), 256); }

slr_status bfail(slr_batch b, slr_status s, const std::string &m)
{
    if (b) b->err = m; else g_batch_create_error = m;
    return s;
}

slr_status bcuda(slr_batch b, cudaError_t e, const char *where)
{
    return bfail(b, SLR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Bring the host mirror up to date with the device results.
slr_status sync_mirror(slr_batch b)
{
    cudaError_t e = cudaMemcpyAsync(b->inst.data(), b->ws + off_inst(), (size_t)b->max_inst * sizeof(BInst),
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "read batch table");
    return SLR_OK;
}

}  // namespace

extern "C" {

size_t slr_batch_workspace_size(int32_t max_instances)
{
    if (max_instances < 1 || max_instances > slr::kMaxBatch) return 0;
    return ws_total(max_instances);
}

size_t slr_batch_scratch_size(const slr_desc *d)
{
    bool unsup = false;
    if (!slr::describe_invalid(d, &unsup).empty()) return 0;
    if (d->stencil == SLR_LIFE) return 0;
    const slr::Problem p = slr::problem_of(d);
    // the second state buffer, and for defect correction the binary32 defect and two corrections
    return rup(p.state_bytes, 256) + (d->defect_correction ? slr::dc_workspace_bytes(p.nx, p.ny, p.nz) : 0);
}

slr_status slr_batch_create(int32_t max_instances, void *workspace, size_t workspace_bytes, void *stream,
                            slr_batch *out)
{
    if (!out) return bfail(nullptr, SLR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_instances < 1 || max_instances > slr::kMaxBatch)
        return bfail(nullptr, SLR_ERR_INVALID_ARG, "max_instances must be in [1, 1024]");
    if (!workspace || ((uintptr_t)workspace & 255u))
        return bfail(nullptr, SLR_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
    if (workspace_bytes < ws_total(max_instances)) return bfail(nullptr, SLR_ERR_WORKSPACE, "workspace too small");
    slr_batch_ctx *b = new (std::nothrow) slr_batch_ctx();
    if (!b) return bfail(nullptr, SLR_ERR_INVALID_ARG, "host allocation failed");
    b->max_inst = max_instances;
    b->ws = (unsigned char *)workspace;
    b->stream = (cudaStream_t)stream;
    b->inst.assign((size_t)max_instances, BInst());
    memset(b->inst.data(), 0, sizeof(BInst) * (size_t)max_instances);
    b->used.assign((size_t)max_instances, 0);
    b->reported.assign((size_t)max_instances, 0);
    b->err = "no error";
    b->dirty = true;
    cudaError_t e = cudaMemsetAsync(b->ws, 0, ws_total(max_instances), b->stream);
    if (e != cudaSuccess) {
        delete b;
        return bcuda(nullptr, e, "clear batch workspace");
    }
    *out = b;
    return SLR_OK;
}

slr_status slr_batch_add(slr_batch b, const slr_desc *d, void *u, const void *aux, void *scratch, int64_t max_iters,
                         int32_t *slot)
{
    if (!b) return bfail(nullptr, SLR_ERR_INVALID_ARG, "batch is NULL");
    bool unsup = false;
    const std::string why = slr::describe_invalid(d, &unsup);
    if (!why.empty()) return bfail(b, unsup ? SLR_ERR_UNSUPPORTED : SLR_ERR_INVALID_ARG, why);
    if (d->stencil == SLR_LIFE)
        return bfail(b, SLR_ERR_UNSUPPORTED, "batches run the Jacobi and restoration stencils");
    if (d->stencil == SLR_RESTORE8 && d->math != SLR_MATH_EXACT)
        return bfail(b, SLR_ERR_UNSUPPORTED, "batched restoration runs EXACT math");
    if (!u || !aux || !scratch || ((uintptr_t)u & 15u) || ((uintptr_t)scratch & 15u))
        return bfail(b, SLR_ERR_INVALID_ARG, "u, aux and scratch must be device pointers (u, scratch 16-byte aligned)");
    if (max_iters < 1) return bfail(b, SLR_ERR_INVALID_ARG, "max_iters must be >= 1");
    int s = -1;
    for (int i = 0; i < b->max_inst; ++i)
        if (!b->used[(size_t)i]) { s = i; break; }
    if (s < 0) return bfail(b, SLR_ERR_WORKSPACE, "batch is full");
    if (!b->dirty) {
        slr_status st = sync_mirror(b);
        if (st != SLR_OK) return st;
    }
    const slr::Problem p = slr::problem_of(d);
    BInst I;
    memset(&I, 0, sizeof(I));
    I.stencil = p.stencil; I.storage = p.storage; I.wrap = p.wrap; I.reduce = p.reduce;
    I.nx = p.nx; I.ny = p.ny; I.nz = p.nz;
    I.ghost = p.ghost; I.h2 = p.h2; I.d = p.d; I.tol = p.tol;
    I.ghostf = p.ghostf; I.h2f = p.h2f; I.df = p.df; I.alpha = p.alpha;
    I.a = u; I.b = scratch; I.aux = aux;
    I.max_iters = max_iters;
    I.tiles_x = (p.nx + slr::kTileW - 1) / slr::kTileW;
    I.tiles_y = (p.ny + slr::kTileH - 1) / slr::kTileH;
    I.units = I.tiles_x * I.tiles_y * p.nz;
    I.dc = d->defect_correction ? 1 : 0;
    I.cs = slr::cluster_size(I);
    if (d->defect_correction) {
        const size_t blk = rup((size_t)p.nx * (size_t)p.ny * (size_t)p.nz * 4, 256);
        unsigned char *f32 = (unsigned char *)scratch + rup(p.state_bytes, 256);
        I.dc = 1;
        I.inner = d->inner_sweeps > 0 ? d->inner_sweeps : 50;
        I.r32 = (float *)f32;
        I.e0 = (float *)(f32 + blk);
        I.e1 = (float *)(f32 + 2 * blk);
        I.phase = 0;
    }
    b->inst[(size_t)s] = I;
    b->used[(size_t)s] = 1;
    b->reported[(size_t)s] = 0;
    b->dirty = true;
    if (slot) *slot = s;
    return SLR_OK;
}

slr_status slr_batch_remove(slr_batch b, int32_t slot)
{
    if (!b || slot < 0 || slot >= b->max_inst || !b->used[(size_t)slot])
        return bfail(b, SLR_ERR_INVALID_ARG, "no such slot");
    if (!b->dirty) {
        slr_status st = sync_mirror(b);
        if (st != SLR_OK) return st;
    }
    b->used[(size_t)slot] = 0;
    memset(&b->inst[(size_t)slot], 0, sizeof(BInst));
    b->dirty = true;
    return SLR_OK;
}

slr_status slr_batch_run(slr_batch b, int64_t sweeps)
{
    if (!b) return bfail(nullptr, SLR_ERR_INVALID_ARG, "batch is NULL");
    if (sweeps < 1) return bfail(b, SLR_ERR_INVALID_ARG, "sweeps must be >= 1");
    if (!b->dirty) {
        slr_status st = sync_mirror(b);
        if (st != SLR_OK) return st;
    }
    // the running instances: the batch-wide launch's, then those run by
    // clusters, grouped by cluster size (1, 2, 4, 8, 16), all in one list
    std::vector<int> act, grp[slr::kClusterGroups];
    std::vector<long long> prefix(1, 0);
    for (int i = 0; i < b->max_inst; ++i) {
        const BInst &I = b->inst[(size_t)i];
        if (!b->used[(size_t)i] || I.done || I.iters >= I.max_iters) continue;
        if (I.cs) {
            grp[__builtin_ctz((unsigned)I.cs)].push_back(i);
        } else {
            act.push_back(i);
            prefix.push_back(prefix.back() + I.units);
        }
    }
    const size_t nact = act.size();
    for (auto &g : grp) act.insert(act.end(), g.begin(), g.end());
    cudaError_t e = cudaMemcpyAsync(b->ws + off_inst(), b->inst.data(), (size_t)b->max_inst * sizeof(BInst),
                                    cudaMemcpyHostToDevice, b->stream);
    b->dirty = false;
    if (e != cudaSuccess) return bcuda(b, e, "write batch table");
    if (act.empty()) return cudaStreamSynchronize(b->stream) == cudaSuccess ? SLR_OK : bcuda(b, cudaGetLastError(), "sync");
    e = cudaMemcpyAsync(b->ws + off_act(b->max_inst), act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->ws + off_prefix(b->max_inst), prefix.data(), prefix.size() * sizeof(long long),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->ws + off_slots(b->max_inst), 0, (size_t)b->max_inst * slr::kSlots * sizeof(slr::Slot),
                            b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ws, 0, sizeof(slr::Ctl), b->stream);
    // the host vectors must outlive the asynchronous copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "stage batch run");
    slr::BatchArgs ba;
    ba.inst = (BInst *)(b->ws + off_inst());
    ba.slots = (slr::Slot *)(b->ws + off_slots(b->max_inst));
    ba.act = (const int *)(b->ws + off_act(b->max_inst));
    ba.prefix = (const long long *)(b->ws + off_prefix(b->max_inst));
    ba.nact = (int)nact;
    ba.sweeps = sweeps;
    ba.ctl = (slr::Ctl *)b->ws;
    ba.limit_ns = 2000000000ll;
    // the clusters' instances: one launch per cluster size, each on a side
    // stream of its own so that they run together (the staging above is
    // complete: the stream was synchronised); the batch-wide launch follows on
    // `stream` once they are all done
    size_t off = nact;
    for (int gi = 0; gi < slr::kClusterGroups; ++gi) {
        const size_t ng = grp[gi].size();
        if (ng == 0) continue;
        if (!b->side[gi]) {
            e = cudaStreamCreateWithFlags(&b->side[gi], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[gi], cudaEventDisableTiming);
            if (e != cudaSuccess) return bcuda(b, e, "cluster stream");
        }
        slr::ClusterArgs ca;
        ca.inst = ba.inst;
        ca.list = ba.act + off;
        ca.cs = 1 << gi;
        ca.sweeps = sweeps;
        size_t csm = 0;
        for (int i : grp[gi]) csm = std::max(csm, slr::cluster_smem(b->inst[(size_t)i], ca.cs));
        off += ng;
        e = cudaFuncSetAttribute(slr::batch_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
        if (e == cudaSuccess && ca.cs > 8)
            e = cudaFuncSetAttribute(slr::batch_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return bcuda(b, e, "cluster kernel attributes");
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(ng * (size_t)ca.cs));
        cfg.blockDim = dim3(slr::kBThreads);
        cfg.dynamicSmemBytes = csm;
        cfg.stream = b->side[gi];
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = (unsigned)ca.cs;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, slr::batch_cluster_kernel, ca);
        if (e == cudaSuccess) e = cudaEventRecord(b->done[gi], b->side[gi]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->done[gi], 0);
        if (e != cudaSuccess) return bcuda(b, e, "cluster kernel launch");
    }
    if (nact == 0) return SLR_OK;
    const size_t smem = (size_t)(slr::kBThreads / 32) * slr::kStageBytesPerWarp + (size_t)ba.nact * 16 +
                        (size_t)ba.nact * 4 * 4 + 4 + (size_t)ba.nact;
    e = cudaFuncSetAttribute(slr::batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return bcuda(b, e, "batch kernel attributes");
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, slr::batch_kernel, slr::kBThreads, smem);
    if (e != cudaSuccess || per_sm < 1) return bcuda(b, e == cudaSuccess ? cudaErrorCooperativeLaunchTooLarge : e, "occupancy");
    if (per_sm > 4) per_sm = 4;
    ba.nblocks = sms * per_sm;
    void *args[] = {&ba};
    e = cudaLaunchCooperativeKernel((const void *)slr::batch_kernel, dim3(ba.nblocks), dim3(slr::kBThreads), args,
                                    smem, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch kernel launch");
    return SLR_OK;
}

slr_status slr_batch_poll(slr_batch b, int32_t *finished, int32_t max_finished, int32_t *n_finished,
                          int32_t *n_running)
{
    if (!b) return bfail(nullptr, SLR_ERR_INVALID_ARG, "batch is NULL");
    slr_status st = sync_mirror(b);
    if (st != SLR_OK) return st;
    slr::Ctl c;
    cudaError_t e = cudaMemcpyAsync(&c, b->ws, sizeof(c), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "read batch control");
    int nf = 0, nr = 0;
    for (int i = 0; i < b->max_inst; ++i) {
        if (!b->used[(size_t)i]) continue;
        const BInst &I = b->inst[(size_t)i];
        const bool fin = I.done || I.iters >= I.max_iters;
        if (fin && !b->reported[(size_t)i]) {
            if (finished && nf < max_finished) {
                finished[nf++] = i;
                b->reported[(size_t)i] = 1;
            }
        } else if (!fin) {
            ++nr;
        }
    }
    if (n_finished) *n_finished = nf;
    if (n_running) *n_running = nr;
    if (c.err & slr::DEV_ERR_TIMEOUT) return bfail(b, SLR_ERR_TIMEOUT, "a device-side grid barrier wait ran out its limit");
    return SLR_OK;
}

slr_status slr_batch_result(slr_batch b, int32_t slot, double *value, int64_t *iters, int32_t *converged,
                            uint64_t *count)
{
    if (!b || slot < 0 || slot >= b->max_inst || !b->used[(size_t)slot])
        return bfail(b, SLR_ERR_INVALID_ARG, "no such slot");
    const BInst &I = b->inst[(size_t)slot];
    if (value) *value = I.value;
    if (iters) *iters = I.iters;
    if (converged) *converged = I.converged;
    if (count) *count = I.count;
    return I.converged ? SLR_OK : SLR_NOT_CONVERGED;
}

slr_status slr_batch_destroy(slr_batch b)
{
    delete b;
    return SLR_OK;
}

const char *slr_batch_last_error(slr_batch b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

}  // extern "C"
