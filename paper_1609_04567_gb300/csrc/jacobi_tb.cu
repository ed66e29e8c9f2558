// jacobi_tb.cu -- temporal-blocked 2D Helmholtz Jacobi: up to 8 sweeps per pass
// over HBM.
//
// The loop-of-stencil-reduce-d of Sec. 3.1 with the five-point update of
// Sec. 4.1, u' = (h^2 f + ((u_N + u_S) + u_W) + u_E) / (4 + sigma h^2), in
// binary32 arithmetic with the state stored as binary32, bfloat16 or binary16
// (every new value rounded to the storage type, the change taken between
// stored values), a Dirichlet ghost value, reduce max |u' - u|, stop at the first
// sweep whose reduced value is below tol or at the iteration cap.
//
// Tiles.  A pass cuts the grid into tiles of 240 owned columns by H - 16 owned
// rows (H = 112 rows for 4-byte storage, 224 for 2-byte storage).  A CTA
// loads a tile's state and f with a halo of 8 cells on every side, 256 x H
// cells each, by two TMA boxes (the hardware fills the cells outside the
// grid with 0; for another Dirichlet ghost value, which must be exact in the
// storage type, the border tiles then set them to it), runs k <= 8 sweeps on
// them in shared memory, and stores the owned cells to the other state
// buffer.  Sweep s updates the tile rows s .. H-1-s; cells within s of the
// tile's edge are out of date after s sweeps, the owned cells never are.
// Cells outside the grid are never written and keep the ghost value.
//
// Threads.  16 warps; warp w owns tile rows [w R, (w+1) R) (R = H / 16) and
// updates them in place, top to bottom, keeping the old rows y-1, y, y+1 of
// its 8 cells per lane in registers (a lane holds two 16-byte groups of 4
// cells, 128 columns apart, for binary32 storage, one group of 8 for 2-byte
// storage, so every warp access is 512 contiguous bytes); x-neighbours by
// shuffles.  The old rows just above and below a warp's rows, which the
// neighbouring warps overwrite during the sweep, are read before a CTA
// barrier; a second barrier ends the sweep.  Arithmetic per cell: the same
// operations in the same order as the one-sweep-per-pass kernels, two cells
// per paired binary32 instruction, the division by the constant 4 + sigma h^2
// by Markstein's corrected reciprocal (exact, checked exhaustively on the
// device) with the IEEE division for numerators outside its range.
//
// Reduce and decision.  The max |delta| over each tile's owned cells is taken
// per sweep (warp, then CTA in shared memory, then one slot per sweep of the
// pass).  After a pass a grid barrier publishes the slots and every CTA takes
// the same decision: the first sweep of the pass whose value is below tol
// stops the loop.  If that is not the pass's last sweep, the pass is run
// again from its input, which it did not overwrite (the two state buffers
// alternate), with only the sweeps up to the stopping one, so the state, the
// reduced value and the iteration count are those of the one-sweep-per-pass
// loop.  The caller's buffer receives the final state.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>

#include "crmath.cuh"
#include "jacobi_tb.h"
#include "slr_internal.cuh"
#include "tma.cuh"

namespace slr {
namespace {

constexpr int kTThreads = 512;
constexpr int kTWarps = kTThreads / 32;
constexpr int kTHalo = kJacobiTbMaxK;          // halo cells per side
constexpr int kTW = 256;                       // tile columns, halo included
constexpr int kTOwnW = kTW - 2 * kTHalo;       // 240 owned columns

template <class T>
struct TbShape {
    static constexpr int kVG = 16 / (int)sizeof(T);          // cells per 16-byte group
    static constexpr int kNG = 8 / kVG;                      // groups per lane (2 or 1)
    static constexpr int kGStride = kTW / kNG;               // columns between a lane's groups
    static constexpr int kH = sizeof(T) == 4 ? 112 : 224;    // tile rows, halo included
    static constexpr int kR = kH / kTWarps;                  // rows per warp
    static constexpr int kOwnH = kH - 2 * kTHalo;
    static constexpr size_t kPlane = (size_t)kTW * kH * sizeof(T);
    static constexpr size_t kSmem = 128 + 2 * kPlane + 16 + kTHalo * 4;
    static_assert(kR * kTWarps == kH, "warps tile the rows");
    static_assert(kPlane % 128 == 0, "TMA destinations stay 128-byte aligned");
    static_assert(kNG * kVG == 8 && kVG % 2 == 0, "eight cells per lane in whole pairs");
};

template <class T>
struct JTb {
    CUtensorMap umap[2];        // state buffers A (caller's u) and B, box 256 x H
    CUtensorMap fmap;           // f, box 256 x H
    T *buf[2];
    int nx, ny;
    int tiles_x, tiles_y;
    int K;                      // sweeps per pass
    float h2, d, yd;            // h^2, 4 + sigma h^2, RN(1 / d)
    int dconst;                 // d in the range of the corrected quotient
    T ghost;                    // the Dirichlet ghost value in storage form
    int ghost_fill;             // the ghost is not +0: cells outside the grid are set to it
};

// ---- the eight cells of a lane in a row ------------------------------------
template <class T> struct Lane8;
template <> struct Lane8<float> {
    __device__ __forceinline__ static void widen(const uint4 (&w)[2], float (&v)[8])
    {
        v[0] = __uint_as_float(w[0].x); v[1] = __uint_as_float(w[0].y);
        v[2] = __uint_as_float(w[0].z); v[3] = __uint_as_float(w[0].w);
        v[4] = __uint_as_float(w[1].x); v[5] = __uint_as_float(w[1].y);
        v[6] = __uint_as_float(w[1].z); v[7] = __uint_as_float(w[1].w);
    }
    // q rounded to storage (exact for binary32) into w; o = the stored values
    __device__ __forceinline__ static void round(const float (&q)[8], uint4 (&w)[2], float (&o)[8])
    {
        w[0] = make_uint4(__float_as_uint(q[0]), __float_as_uint(q[1]), __float_as_uint(q[2]), __float_as_uint(q[3]));
        w[1] = make_uint4(__float_as_uint(q[4]), __float_as_uint(q[5]), __float_as_uint(q[6]), __float_as_uint(q[7]));
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = q[k];
    }
};
template <> struct Lane8<__nv_bfloat16> {
    __device__ __forceinline__ static float2 w2(uint32_t w)
    {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
    }
    __device__ __forceinline__ static void widen(const uint4 (&w)[1], float (&v)[8])
    {
        float2 t;
        t = w2(w[0].x); v[0] = t.x; v[1] = t.y;
        t = w2(w[0].y); v[2] = t.x; v[3] = t.y;
        t = w2(w[0].z); v[4] = t.x; v[5] = t.y;
        t = w2(w[0].w); v[6] = t.x; v[7] = t.y;
    }
    __device__ __forceinline__ static uint32_t pack(float a, float b)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *(const uint32_t *)&h;
    }
    __device__ __forceinline__ static void round(const float (&q)[8], uint4 (&w)[1], float (&o)[8])
    {
        w[0] = make_uint4(pack(q[0], q[1]), pack(q[2], q[3]), pack(q[4], q[5]), pack(q[6], q[7]));
        widen(w, o);
    }
};
template <> struct Lane8<__half> {
    __device__ __forceinline__ static float2 w2(uint32_t w) { return __half22float2(*(const __half2 *)&w); }
    __device__ __forceinline__ static void widen(const uint4 (&w)[1], float (&v)[8])
    {
        float2 t;
        t = w2(w[0].x); v[0] = t.x; v[1] = t.y;
        t = w2(w[0].y); v[2] = t.x; v[3] = t.y;
        t = w2(w[0].z); v[4] = t.x; v[5] = t.y;
        t = w2(w[0].w); v[6] = t.x; v[7] = t.y;
    }
    __device__ __forceinline__ static uint32_t pack(float a, float b)
    {
        const __half2 h = __floats2half2_rn(a, b);
        return *(const uint32_t *)&h;
    }
    __device__ __forceinline__ static void round(const float (&q)[8], uint4 (&w)[1], float (&o)[8])
    {
        w[0] = make_uint4(pack(q[0], q[1]), pack(q[2], q[3]), pack(q[4], q[5]), pack(q[6], q[7]));
        widen(w, o);
    }
};

// the lane's cells of tile row `row` (shared memory), widened
template <class T>
__device__ __forceinline__ void load8(const T *row, int lane, float (&v)[8])
{
    using S = TbShape<T>;
    uint4 w[S::kNG];
#pragma unroll
    for (int g = 0; g < S::kNG; ++g) w[g] = *(const uint4 *)(row + g * S::kGStride + lane * S::kVG);
    Lane8<T>::widen(w, v);
}

// One row of a sweep: the new values of row y of the lane's cells from the old
// rows above (a), at (c) and below (b) and f of row y; stored in place for the
// groups inside the grid; max |delta| over the reduced groups into mx.
template <class T, bool REDUCE>
__device__ __forceinline__ void row_update(const JTb<T> &tp, T *srow, const float (&a)[8], const float (&c)[8],
                                           const float (&b)[8], const T *frow, int lane, const bool (&gin)[2],
                                           const bool (&red)[2], bool own_row, float &mx)
{
    using S = TbShape<T>;
    constexpr int VG = S::kVG, NG = S::kNG;
    float f[8];
    load8<T>(frow, lane, f);
    // x-neighbours of each group's first and last cell
    float left[NG], right[NG];
    if constexpr (NG == 1) {
        left[0] = __shfl_up_sync(0xffffffffu, c[7], 1);        // lane 0: outside the tile (not used)
        right[0] = __shfl_down_sync(0xffffffffu, c[0], 1);     // lane 31: outside the tile
    } else {
        // groups at columns 4l and 128 + 4l: lane 31's second group follows lane 0's first
        left[0] = __shfl_up_sync(0xffffffffu, c[3], 1);
        left[1] = __shfl_sync(0xffffffffu, lane == 31 ? c[3] : c[7], (lane + 31) & 31);
        right[0] = __shfl_sync(0xffffffffu, lane == 0 ? c[4] : c[0], (lane + 1) & 31);
        right[1] = __shfl_down_sync(0xffffffffu, c[4], 1);
    }
    float q[8];
    float amin = INFINITY, amax = 0.0f;            // |numerator| over the groups inside the grid
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        const int g = k / VG, i = k % VG;
        const float2 w = make_float2(i == 0 ? left[g] : c[k - 1], c[k]);
        const float2 e = make_float2(c[k + 1], i + 2 == VG ? right[g] : c[k + 2]);
        const float2 sum = __fadd2_rn(__fadd2_rn(__fadd2_rn(make_float2(a[k], a[k + 1]), make_float2(b[k], b[k + 1])),
                                                 w), e);
        // h^2 f by the scalar operation: a paired product feeding a paired sum
        // may be contracted into one fused operation
        const float2 t = make_float2(__fmul_rn(tp.h2, f[k]), __fmul_rn(tp.h2, f[k + 1]));
        const float2 num = __fadd2_rn(t, sum);
        if (gin[g]) {
            amin = min3f(amin, fabsf(num.x), fabsf(num.y));
            amax = max3f(amax, fabsf(num.x), fabsf(num.y));
        }
        q[k] = num.x;
        q[k + 1] = num.y;
    }
    if (tp.dconst && amin >= 0x1p-40f && amax < 0x1p40f) {
        const float2 y2 = make_float2(tp.yd, tp.yd), nd2 = make_float2(-tp.d, -tp.d);
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            // Markstein's corrected quotient; fma(q, -d, a) is the residual a - q d
            const float2 num = make_float2(q[k], q[k + 1]);
            const float2 q0 = __fmul2_rn(num, y2);
            const float2 q1 = __ffma2_rn(__ffma2_rn(q0, nd2, num), y2, q0);
            const float2 qq = __ffma2_rn(__ffma2_rn(q1, nd2, num), y2, q1);
            q[k] = qq.x;
            q[k + 1] = qq.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            q[k] = tp.dconst ? div_const_rn(q[k], tp.d, tp.yd) : div_ieee(q[k], tp.d);
    }
    uint4 w[NG];
    float o[8];
    Lane8<T>::round(q, w, o);
#pragma unroll
    for (int g = 0; g < NG; ++g)
        if (gin[g]) *(uint4 *)(srow + g * S::kGStride + lane * VG) = w[g];
    if (REDUCE && own_row) {
        const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            if (red[k / VG]) {
                // |old - new|: fma(new, -1, old) is the rounded difference
                const float2 dl = __ffma2_rn(make_float2(o[k], o[k + 1]), m1, make_float2(c[k], c[k + 1]));
                mx = max3f(mx, fabsf(dl.x), fabsf(dl.y));
            }
        }
    }
}

template <class T>
__device__ __forceinline__ void copy8(float (&dst)[8], const float (&src)[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[k] = src[k];
}

// One sweep s (1-based) of the tile in shared memory (state S, f F).  Rows
// [yin_lo, yin_hi) of the tile lie inside the grid.
template <class T, bool REDUCE>
__device__ __forceinline__ void tile_sweep(const JTb<T> &tp, T *S, const T *F, int s, int yin_lo, int yin_hi,
                                           const bool (&gin)[2], const bool (&red)[2], float &mx)
{
    using Sh = TbShape<T>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ra = warp * Sh::kR, rb = ra + Sh::kR;
    int ylo = ra > s ? ra : s, yhi = rb < Sh::kH - s ? rb : Sh::kH - s;
    ylo = ylo > yin_lo ? ylo : yin_lo;
    yhi = yhi < yin_hi ? yhi : yin_hi;
    // the old rows just outside the warp's rows, which the neighbouring warps
    // overwrite during this sweep (ylo == ra implies ra >= s >= 1, yhi == rb
    // implies rb <= H - s - 1 < H)
    float up[8], dn[8];
    if (ylo < yhi && ylo == ra) load8<T>(S + (ra - 1) * kTW, lane, up);
    if (ylo < yhi && yhi == rb) load8<T>(S + rb * kTW, lane, dn);
    __syncthreads();
    if (ylo < yhi) {
        float a[8], c[8], b[8];
        if (ylo == ra) copy8<T>(a, up);
        else load8<T>(S + (ylo - 1) * kTW, lane, a);
        load8<T>(S + ylo * kTW, lane, c);
        // rows rotate through a, c, b: three rows per turn, no register copies
        for (int y = ylo; y < yhi; y += 3) {
            if (y + 1 == rb) copy8<T>(b, dn);
            else load8<T>(S + (y + 1) * kTW, lane, b);
            row_update<T, REDUCE>(tp, S + y * kTW, a, c, b, F + y * kTW, lane, gin, red,
                                  y >= kTHalo && y < Sh::kH - kTHalo, mx);
            if (y + 1 >= yhi) break;
            if (y + 2 == rb) copy8<T>(a, dn);
            else load8<T>(S + (y + 2) * kTW, lane, a);
            row_update<T, REDUCE>(tp, S + (y + 1) * kTW, c, b, a, F + (y + 1) * kTW, lane, gin, red,
                                  y + 1 >= kTHalo && y + 1 < Sh::kH - kTHalo, mx);
            if (y + 2 >= yhi) break;
            if (y + 3 == rb) copy8<T>(c, dn);
            else load8<T>(S + (y + 3) * kTW, lane, c);
            row_update<T, REDUCE>(tp, S + (y + 2) * kTW, b, a, c, F + (y + 2) * kTW, lane, gin, red,
                                  y + 2 >= kTHalo && y + 2 < Sh::kH - kTHalo, mx);
        }
    }
    __syncthreads();
}

// One pass: every tile of this CTA, kp sweeps each, from buf[cur] to
// buf[cur ^ 1]; with REDUCE the per-sweep max |delta| of the CTA's owned cells
// into s_red[0 .. kp).  False if a TMA wait ran out.
template <class T, bool REDUCE>
__device__ bool tb_pass(const JTb<T> &tp, unsigned char *smem, uint64_t *bar, unsigned *s_red, unsigned &phase,
                        int cur, int kp, const LoopArgs &la)
{
    using Sh = TbShape<T>;
    T *S = (T *)smem;
    T *F = (T *)(smem + Sh::kPlane);
    T *dst = tp.buf[cur ^ 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntiles = tp.tiles_x * tp.tiles_y;
    for (int t = (int)blockIdx.x; t < ntiles; t += (int)gridDim.x) {
        const int tx = t % tp.tiles_x, ty = t / tp.tiles_x;
        const int x0 = tx * kTOwnW - kTHalo, y0 = ty * Sh::kOwnH - kTHalo;   // tile origin in the grid
        if (tid == 0) {
            tma::mbar_expect_tx(bar, (uint32_t)(2 * Sh::kPlane));
            tma::load_2d(S, &tp.umap[cur], x0, y0, bar);
            tma::load_2d(F, &tp.fmap, x0, y0, bar);
        }
        const bool ok = tma::bounded_wait(bar, phase & 1u, tma::kLoadWaitNs, &la.ctl->err);
        ++phase;
        if (!__syncthreads_and(ok)) return false;
        if (tp.ghost_fill && (x0 < 0 || x0 + kTW > tp.nx || y0 < 0 || y0 + Sh::kH > tp.ny)) {
            // the copy filled the cells outside the grid with +0: they hold the ghost
            for (int i = tid; i < kTW * Sh::kH; i += kTThreads) {
                const int gy = y0 + i / kTW, gx = x0 + i % kTW;
                if (gy < 0 || gy >= tp.ny || gx < 0 || gx >= tp.nx) S[i] = tp.ghost;
            }
            __syncthreads();
        }
        const int yin_lo = y0 < 0 ? -y0 : 0;
        const int yin_hi = tp.ny - y0 < Sh::kH ? tp.ny - y0 : Sh::kH;
        bool gin[2] = {false, false}, red[2] = {false, false};
#pragma unroll
        for (int g = 0; g < Sh::kNG; ++g) {
            const int col = g * Sh::kGStride + lane * Sh::kVG;
            gin[g] = x0 + col >= 0 && x0 + col < tp.nx;
            red[g] = gin[g] && col >= kTHalo && col + Sh::kVG <= kTW - kTHalo;
        }
        for (int s = 1; s <= kp; ++s) {
            float mx = 0.0f;
            tile_sweep<T, REDUCE>(tp, S, F, s, yin_lo, yin_hi, gin, red, mx);
            if (REDUCE) {
                // non-negative binary32 values order as their bits
                const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
                if (lane == 0 && m != 0u) atomicMax(&s_red[s - 1], m);
            }
        }
        // the owned cells inside the grid to the output buffer
        const int ra = warp * Sh::kR;
        for (int y = ra; y < ra + Sh::kR; ++y) {
            if (y < kTHalo || y >= Sh::kH - kTHalo || y < yin_lo || y >= yin_hi) continue;
            const long long gy = (long long)y0 + y;
#pragma unroll
            for (int g = 0; g < Sh::kNG; ++g) {
                if (!red[g]) continue;
                const int col = g * Sh::kGStride + lane * Sh::kVG;
                *(uint4 *)(dst + gy * tp.nx + (x0 + col)) = *(const uint4 *)(S + y * kTW + col);
            }
        }
        // this tile's shared-memory accesses before the next tile's copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    // this pass's stores before the copies of later passes (after a grid barrier)
    tma::fence_proxy_async_global();
    return true;
}

template <class T>
__global__ void __launch_bounds__(kTThreads, 1) jacobi_tb_kernel(const __grid_constant__ JTb<T> tp, LoopArgs la)
{
    extern __shared__ unsigned char smem_dyn[];
    using Sh = TbShape<T>;
    unsigned char *smem = align_up(smem_dyn, 128);
    uint64_t *bar = (uint64_t *)(smem + 2 * Sh::kPlane);
    unsigned *s_red = (unsigned *)(bar + 2);
    __shared__ int s_stop, s_rewind;
    __shared__ long long s_it;
    const int tid = threadIdx.x;
    Ctl *ctl = la.ctl;
    const long long it0 = ctl->iters;
    if (ctl->converged || it0 >= la.max_iters || ctl->err) return;
    if ((la.debug_flags & SLR_DEBUG_SKIP_ARRIVAL) && blockIdx.x == gridDim.x - 1) return;
    if (tid == 0) {
        tma::mbar_init(bar, 1);
        tma::mbar_init_fence();
        tma::fence_proxy_async_global();   // earlier stores to the state before this launch's copies
    }
    if (tid < kTHalo) s_red[tid] = 0u;
    __syncthreads();

    unsigned phase = 0;
    unsigned long long bar_target = 0;
    long long it = it0;
    int cur = 0;
    __shared__ int s_kpn;                     // length of the next pass
    if (tid == 0) s_kpn = tp.K;
    __syncthreads();
    for (long long p = 0;; ++p) {
        const long long left = la.max_iters - it;
        const int kp = (int)((long long)s_kpn < left ? (long long)s_kpn : left);
        if (!tb_pass<T, true>(tp, smem, bar, s_red, phase, cur, kp, la)) return;
        __syncthreads();
        if (tid < kp) {
            // the binary32 maximum as binary64 bits (non-negative: bits order as values)
            if (s_red[tid])
                atomicMax(&ctl->sub[p % kSlots][tid].maxbits,
                          (unsigned long long)__double_as_longlong((double)__uint_as_float(s_red[tid])));
            s_red[tid] = 0u;
        }
        bar_target += (unsigned long long)la.nblocks;
        if (!grid_barrier(ctl, bar_target, la.limit_ns)) return;
        if (tid < 32) {
            if (blockIdx.x == 0) zero_slot(&ctl->sub[(p + 2) % kSlots][tid]);
            // lane j decides sweep j of the pass; the first one below tol stops
            Slot sl;
            sl.maxbits = tid < kp ? ld_relaxed_u64(&ctl->sub[p % kSlots][tid].maxbits) : 0ull;
            sl.sum = sl.cnt = 0ull;
            sl.changed = 0u;
            const Decision dj = decide(la.reduce, sl, la.tol);
            const unsigned conv = __ballot_sync(0xffffffffu, tid < kp && dj.converged);
            const int jstop = conv ? __ffs(conv) - 1 : -1;
            const int jlast = jstop >= 0 ? jstop : kp - 1;
            const double value = __shfl_sync(0xffffffffu, dj.value, jlast);
            const long long itn = it + jlast + 1;
            const double v0 = __shfl_sync(0xffffffffu, dj.value, 0);
            if (tid == 0) {
                s_kpn = predict_pass(v0, value, kp, la.tol, tp.K);
                const int stop = jstop >= 0 || itn >= la.max_iters;
                s_stop = stop;
                s_rewind = jstop >= 0 && jstop + 1 < kp ? jstop + 1 : 0;
                s_it = itn;
                if (stop && blockIdx.x == 0) {
                    ctl->iters = itn;
                    ctl->value = value;
                    ctl->count = 0ull;
                    ctl->changed = value > 0.0;
                    ctl->converged = jstop >= 0;
                }
            }
        }
        __syncthreads();
        it = s_it;
        if (s_stop) {
            if (s_rewind) {
                // the pass again from its input, up to the stopping sweep
                if (tid == 0) tma::fence_proxy_async_global();
                if (!tb_pass<T, false>(tp, smem, bar, s_red, phase, cur, s_rewind, la)) return;
                bar_target += (unsigned long long)la.nblocks;
                if (!grid_barrier(ctl, bar_target, la.limit_ns)) return;
            }
            if ((cur ^ 1) == 1) grid_copy(tp.buf[1], tp.buf[0], (size_t)tp.nx * tp.ny * sizeof(T));
            return;
        }
        cur ^= 1;
        if (tid == 0) tma::fence_proxy_async_global();
    }
}

template <class T> CUtensorMapDataType tb_type();
template <> CUtensorMapDataType tb_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> CUtensorMapDataType tb_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
template <> CUtensorMapDataType tb_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

template <class T>
cudaError_t run_tb(const Problem &p, LoopArgs la, int K, cudaStream_t st)
{
    using Sh = TbShape<T>;
    JTb<T> tp;
    memset(&tp, 0, sizeof(tp));
    const CUtensorMapDataType dt = tb_type<T>();
    bool ok = tma::make_map_2d(&tp.umap[0], la.a, dt, sizeof(T), p.nx, p.ny, kTW, Sh::kH) &&
              tma::make_map_2d(&tp.umap[1], la.b, dt, sizeof(T), p.nx, p.ny, kTW, Sh::kH) &&
              tma::make_map_2d(&tp.fmap, la.aux, dt, sizeof(T), p.nx, p.ny, kTW, Sh::kH);
    if (!ok) return cudaErrorNotSupported;
    tp.buf[0] = (T *)la.a;
    tp.buf[1] = (T *)la.b;
    tp.nx = (int)p.nx;
    tp.ny = (int)p.ny;
    tp.tiles_x = (int)((p.nx + kTOwnW - 1) / kTOwnW);
    tp.tiles_y = (int)((p.ny + Sh::kOwnH - 1) / Sh::kOwnH);
    tp.K = K;
    tp.h2 = p.h2f;
    tp.d = p.df;
    tp.yd = host_rcp_rn(p.df);
    tp.dconst = div_const_ok(p.df);
    tp.ghost = (T)p.ghostf;
    tp.ghost_fill = p.ghostf != 0.0f || std::signbit(p.ghostf);
    auto kern = jacobi_tb_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::kSmem);
    if (e != cudaSuccess) return e;
    return launch_cooperative(kern, kTThreads, Sh::kSmem, 1, la, &tp, st);
}

size_t elem_bytes(int storage)
{
    switch (storage) {
    case SLR_F32: return 4;
    case SLR_BF16:
    case SLR_F16: return 2;
    default: return 0;
    }
}

}  // namespace

// The ghost value as the tile holds it (storage form) must be the value the
// update reads: exactly representable in the storage type.
bool jacobi_tb_ghost_exact(const Problem &p)
{
    const float g = p.ghostf;
    if (g != g) return false;
    switch (p.storage) {
    case SLR_F32: return true;
    case SLR_BF16: {
        uint32_t b;
        memcpy(&b, &g, 4);
        return (b & 0xFFFFu) == 0u;
    }
    case SLR_F16: return __half2float(__float2half_rn(g)) == g && (g != 0.0f || !std::signbit(g) ||
                                                                    std::signbit(__half2float(__float2half_rn(g))));
    default: return false;
    }
}

bool jacobi_tb_supported(const Problem &p, const void *a, const void *b, const void *f)
{
    if (p.stencil == SLR_J3D7) return jacobi_tb3_supported(p, a, b, f);
    const size_t es = elem_bytes(p.storage);
    if (p.stencil != SLR_J2D5 || es == 0 || p.wrap || !jacobi_tb_ghost_exact(p)) return false;
    if ((p.nx * (long long)es) % 16 != 0 || p.nx >= (1ll << 31) - 4096 || p.ny >= (1ll << 31) - 4096) return false;
    if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)f) % 16 != 0) return false;
    return tma::encode_fn() != nullptr;
}

int jacobi_tb_resolve_k(const Problem &p, const void *a, const void *b, const void *f)
{
    if (p.k == 1 || !jacobi_tb_supported(p, a, b, f)) return 1;
    const bool d3 = p.stencil == SLR_J3D7;
    const int most = d3 ? kJacobiTb3MaxK : kJacobiTbMaxK;
    // the library's choice unless a staging of the one-sweep kernel was asked for
    if (p.k == 0) return p.tiling == SLR_TILING_AUTO ? (d3 ? kJacobiTb3DefaultK : kJacobiTbMaxK) : 1;
    return p.k > most ? most : p.k;
}

cudaError_t jacobi_tb_persistent(const Problem &p, LoopArgs la, cudaStream_t st)
{
    const int K = jacobi_tb_resolve_k(p, la.a, la.b, la.aux);
    if (K < 2) return cudaErrorNotSupported;
    if (p.stencil == SLR_J3D7) return jacobi_tb3_persistent(p, la, K, st);
    switch (p.storage) {
    case SLR_F32: return run_tb<float>(p, la, K, st);
    case SLR_BF16: return run_tb<__nv_bfloat16>(p, la, K, st);
    case SLR_F16: return run_tb<__half>(p, la, K, st);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace slr
