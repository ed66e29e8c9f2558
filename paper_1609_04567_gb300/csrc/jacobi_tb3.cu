// jacobi_tb3.cu -- temporal-blocked 3D Helmholtz Jacobi: up to 4 sweeps per
// pass over HBM.
//
// The loop-of-stencil-reduce-d of Sec. 3.1 with the seven-point form of the
// Sec. 4.1 update, u' = (h^2 f + ((((u_W + u_E) + u_N) + u_S) + u_D) + u_U) /
// (6 + sigma h^2), in binary32 arithmetic with the state stored as binary32,
// bfloat16 or binary16 (every new value rounded to the storage type, the
// change taken between stored values), a Dirichlet ghost value, reduce
// max |u' - u|, stop at the first sweep whose value is below tol or at the cap.
//
// Work units.  A pass cuts the grid into columns of 48 owned x by 24 - 2K
// owned y cells (K = the pipeline depth, 2 or 4), and each column into chunks
// of 64 owned planes along z; a unit is one chunk of one column.  Units are
// handed out by a per-pass counter, the x-y neighbours of a chunk first, so
// that concurrent units share their halo planes in the L2.
//
// The z march.  A CTA loads the 64 x 24 box of u and f around its column
// (8 halo columns on each side in x, which keeps the box's x origin on a
// 16-byte boundary, and K halo rows in y) one plane at a time by TMA into a
// ring of 8 planes, from K planes below its chunk to K planes above.  With kp
// sweeps in the pass, step z of the march computes level L = 1 .. kp at plane
// z - L: the state after L sweeps, from level L - 1 at planes z - L - 1,
// z - L and z - L + 1, which the thread keeps in registers (its own two
// cells of the plane; the newest came from this very step), and from level
// L - 1's x-y neighbours of plane z - L, which the previous step published in
// shared memory (level 0: the loaded box itself).  Level L's new plane goes to
// registers and to the other of its two shared planes; level kp's owned cells
// go to the other state buffer in global memory.  One CTA barrier per step
// orders all of it.  Level L is correct in the rows [L, 24 - L) of the box,
// which covers the rows its successors read; the planes below 0 and from nz
// on, and the cells outside the grid, hold the ghost value at every level.
//
// Threads.  24 warps: warp w is box row w, lane l its columns 2l and 2l + 1
// (one paired binary32 instruction per operation for the two cells);
// x-neighbours by shuffles.  Arithmetic per cell: the same operations in the
// same order as the one-sweep kernels, the division by the constant
// 6 + sigma h^2 by Markstein's corrected reciprocal (exact, checked on the
// device) with the IEEE division for numerators outside its range.
//
// Reduce and decision.  As for the 2D blocked loop: one slot per sweep of the
// pass (max over each unit's owned cells); after the pass a grid barrier, the
// first sweep below tol stops the loop, and a stop inside the pass reruns the
// pass from its untouched input up to that sweep, so the state, the value and
// the iteration count equal those of one sweep per pass.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <type_traits>

#include "crmath.cuh"
#include "jacobi_tb.h"
#include "slr_internal.cuh"
#include "tma.cuh"

namespace slr {
namespace {

constexpr int kW = 64;                 // box columns
constexpr int kXH = 8;                 // halo columns per side
constexpr int kOwnW = kW - 2 * kXH;    // 48 owned columns
constexpr int kH = 24;                 // box rows (K halo rows per side)
constexpr int kRing = 8;               // loaded planes in flight or in use (a power of two)
constexpr int kChunk = 64;             // owned planes per unit
constexpr int kThreads = 32 * kH;      // warp w = box row w

template <class T>
struct Shape3 {
    static constexpr size_t kPlane = (size_t)kW * kH * sizeof(T);        // one loaded box
    static constexpr size_t kSlot = 2 * kPlane;                           // u and f
    static constexpr size_t kPub = (size_t)kW * kH * sizeof(float);      // one published plane
    static constexpr size_t kPubBytes = 2 * (kJacobiTb3MaxK - 1) * kPub;
    static constexpr size_t kSmem = 128 + kRing * kSlot + kPubBytes + kRing * 8;
    static_assert(kPlane % 128 == 0 && kPub % 128 == 0, "TMA destinations stay 128-byte aligned");
    static_assert(kRing >= kJacobiTb3MaxK + 3 && (kRing & (kRing - 1)) == 0, "ring covers the oldest level's f");
};

template <class T>
struct JTb3 {
    CUtensorMap umap[2];        // state buffers A (caller's u) and B, box 64 x 24 x 1
    CUtensorMap fmap;           // f, box 64 x 24 x 1
    T *buf[2];
    int nx, ny, nz;
    int tiles_x, tiles_y, chunks;
    int K;                      // sweeps per pass (at most the pipeline depth)
    float h2, d, yd;            // h^2, 6 + sigma h^2, RN(1 / d)
    int dconst;                 // d in the range of the corrected quotient
    float ghost;                // the Dirichlet ghost value (exact in T)
};

// two cells of storage type T as binary32 values, and back (rounded)
template <class T> struct Pair2;
template <> struct Pair2<float> {
    __device__ __forceinline__ static float2 load(const float *p) { return *(const float2 *)p; }
    __device__ __forceinline__ static float2 round(float2 q, float2 &bits) { bits = q; return q; }
    __device__ __forceinline__ static void store(float *p, float2 bits) { *(float2 *)p = bits; }
};
template <> struct Pair2<__nv_bfloat16> {
    __device__ __forceinline__ static float2 widen(uint32_t w)
    {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
    }
    __device__ __forceinline__ static float2 load(const __nv_bfloat16 *p) { return widen(*(const uint32_t *)p); }
    __device__ __forceinline__ static float2 round(float2 q, uint32_t &bits)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(q.x, q.y);
        bits = *(const uint32_t *)&h;
        return widen(bits);
    }
    __device__ __forceinline__ static void store(__nv_bfloat16 *p, uint32_t bits) { *(uint32_t *)p = bits; }
};
template <> struct Pair2<__half> {
    __device__ __forceinline__ static float2 widen(uint32_t w) { return __half22float2(*(const __half2 *)&w); }
    __device__ __forceinline__ static float2 load(const __half *p) { return widen(*(const uint32_t *)p); }
    __device__ __forceinline__ static float2 round(float2 q, uint32_t &bits)
    {
        const __half2 h = __floats2half2_rn(q.x, q.y);
        bits = *(const uint32_t *)&h;
        return widen(bits);
    }
    __device__ __forceinline__ static void store(__half *p, uint32_t bits) { *(uint32_t *)p = bits; }
};
template <class T> using Bits2 = typename std::conditional<sizeof(T) == 4, float2, uint32_t>::type;

// register slot of plane x of a level: planes rotate through three slots
template <int ROT, int OFF>
__device__ __forceinline__ constexpr int rs() { return ((ROT + OFF) % 3 + 3) % 3; }

// Everything a unit's steps share.
template <class T, int KD>
struct Unit {
    const T *ring;              // kRing slots of (u box, f box)
    const T *ucell;             // this thread's cells in slot 0's u box
    float *pub;                 // published planes: level L (1 .. KD-1), parity of the plane
    float *pubcell;             // this thread's cells in the first published plane
    uint64_t *bars;
    T *dcell;                   // this thread's cells of plane 0 in the output buffer
    size_t pstride;             // elements per plane
    int z0, z1, zl0, zl1, zs;   // owned planes, loaded planes, first step
    unsigned qb;                // load index of plane zl0
    int kp;
    int lane, w;
    bool gin, own_xy, rin_n, rin_s;
    float2 ghost2;
};

// this thread's cells of slot `slot` (u box, then f box)
template <class T>
__device__ __forceinline__ const T *slot_cell(const T *cell, int slot)
{
    return (const T *)((const unsigned char *)cell + (size_t)slot * Shape3<T>::kSlot);
}

template <class T>
__device__ __forceinline__ const T *ring_u(const T *ring, int slot)
{
    return (const T *)((const unsigned char *)ring + (size_t)slot * Shape3<T>::kSlot);
}
template <class T>
__device__ __forceinline__ const T *ring_f(const T *ring, int slot)
{
    return (const T *)((const unsigned char *)ring + (size_t)slot * Shape3<T>::kSlot + Shape3<T>::kPlane);
}

// Level L at step z: plane p = z - L from level L - 1 (see the header).  FULL:
// a step at which every level's plane lies in the grid and in its range.
template <class T, int KD, int ROT, int L, bool REDUCE, bool FULL>
__device__ __forceinline__ void level(const JTb3<T> &tp, const Unit<T, KD> &U, float2 (&R)[KD][3], float (&mx)[KD],
                                      int z, unsigned slot_z)
{
    if (L > U.kp) return;
    const int p = z - L;
    const int reach = U.kp - L;                   // planes this level serves beyond the chunk
    if (!FULL && (p < U.z0 - reach || p >= U.z1 + reach)) return;
    float2 nv = U.ghost2;
    if (FULL || (p >= 0 && p < tp.nz)) {
        if (U.w < L || U.w >= kH - L) return;     // rows no later level reads
        const float2 c = R[L - 1][rs<ROT, -L>()];
        const float2 dn = R[L - 1][rs<ROT, -L - 1>()];
        const float2 up = R[L - 1][rs<ROT, -L + 1>()];
        float2 n, s;
        const int slot = (int)((slot_z - (unsigned)L) & (kRing - 1));        // plane p's slot
        const T *uc = slot_cell<T>(U.ucell, slot);
        if (L == 1) {
            n = U.rin_n ? Pair2<T>::load(uc - kW) : U.ghost2;
            s = U.rin_s ? Pair2<T>::load(uc + kW) : U.ghost2;
        } else {
            const float *src = U.pubcell + (2 * (L - 2) + (p & 1)) * (kW * kH);
            n = *(const float2 *)(src - kW);
            s = *(const float2 *)(src + kW);
        }
        const float wl = __shfl_up_sync(0xffffffffu, c.y, 1);      // lane 0: outside the box (unused)
        const float er = __shfl_down_sync(0xffffffffu, c.x, 1);    // lane 31: outside the box (unused)
        const float2 f = Pair2<T>::load(uc + kW * kH);
        float2 sum = __fadd2_rn(make_float2(wl, c.x), make_float2(c.y, er));
        sum = __fadd2_rn(sum, n);
        sum = __fadd2_rn(sum, s);
        sum = __fadd2_rn(sum, dn);
        sum = __fadd2_rn(sum, up);
        // h^2 f by the scalar operation: a paired product feeding a paired sum
        // may be contracted into one fused operation
        const float2 t = make_float2(__fmul_rn(tp.h2, f.x), __fmul_rn(tp.h2, f.y));
        // cells outside the grid (their result is dropped) divide 1, which
        // keeps the warp on the paired quotient
        const float2 num = U.gin ? __fadd2_rn(t, sum) : make_float2(1.0f, 1.0f);
        float2 q;
        if (tp.dconst) {
            q = div_const_rn2(num, tp.d, tp.yd);
        } else {
            q = make_float2(div_ieee(num.x, tp.d), div_ieee(num.y, tp.d));
        }
        Bits2<T> bits;
        const float2 o = Pair2<T>::round(q, bits);
        // cells outside the grid stay at the ghost value
        nv = make_float2(U.gin ? o.x : U.ghost2.x, U.gin ? o.y : U.ghost2.y);
        const bool owned = U.own_xy && p >= U.z0 && p < U.z1;
        if (REDUCE) {
            // |old - new|: fma(new, -1, old) is the rounded difference
            const float2 dl = __ffma2_rn(o, make_float2(-1.0f, -1.0f), c);
            mx[L - 1] = max3f(mx[L - 1], owned ? fabsf(dl.x) : 0.0f, owned ? fabsf(dl.y) : 0.0f);
        }
        if (L == U.kp) {
            if (owned) Pair2<T>::store(U.dcell + (size_t)p * U.pstride, bits);
            return;
        }
    }
    if constexpr (L < KD) {
        if (L < U.kp) {
            R[L][rs<ROT, -L>()] = nv;
            if (FULL || (p >= 0 && p < tp.nz)) *(float2 *)(U.pubcell + (2 * (L - 1) + (p & 1)) * (kW * kH)) = nv;
        }
    }
}

// Thread 0: the next planes of the unit into the ring, up to plane `upto`.
template <class T, int KD>
__device__ __forceinline__ void refill(const JTb3<T> &tp, const Unit<T, KD> &U, int &nxt, int upto, int cur, int x0,
                                       int y0)
{
    for (; nxt < U.zl1 && nxt <= upto; ++nxt) {
        const int slot = (int)((U.qb + (unsigned)(nxt - U.zl0)) & (kRing - 1));
        tma::mbar_expect_tx(U.bars + slot, (uint32_t)Shape3<T>::kSlot);
        tma::load_3d((void *)ring_u<T>(U.ring, slot), &tp.umap[cur], x0, y0, nxt, U.bars + slot);
        tma::load_3d((void *)ring_f<T>(U.ring, slot), &tp.fmap, x0, y0, nxt, U.bars + slot);
    }
}

// One step of the march (plane z of level 0 arrives; levels 1 .. kp advance).
template <class T, int KD, int ROT, bool REDUCE, bool FULL>
__device__ __forceinline__ bool step(const JTb3<T> &tp, const Unit<T, KD> &U, float2 (&R)[KD][3], float (&mx)[KD],
                                     int z, const LoopArgs &la, int &nxt, int cur, int x0, int y0)
{
    bool ok = true;
    float2 v0 = U.ghost2;
    // plane z's load index (modulo 2^32, which kRing divides): its slot and phase
    const unsigned qi = U.qb + (unsigned)(z - U.zl0);
    if (z >= U.zl0 && z < U.zl1) {
        const int slot = (int)(qi & (kRing - 1));
        // the plane was asked for several steps ago: usually there already
        if (!tma::mbar_try_wait(U.bars + slot, (qi / kRing) & 1u))
            ok = tma::bounded_wait(U.bars + slot, (qi / kRing) & 1u, tma::kLoadWaitNs, &la.ctl->err);
        if (ok && U.gin) v0 = Pair2<T>::load(slot_cell<T>(U.ucell, slot));
    }
    R[0][rs<ROT, 0>()] = v0;
    level<T, KD, ROT, 1, REDUCE, FULL>(tp, U, R, mx, z, qi);
    level<T, KD, ROT, 2, REDUCE, FULL>(tp, U, R, mx, z, qi);
    if constexpr (KD > 2) {
        level<T, KD, ROT, 3, REDUCE, FULL>(tp, U, R, mx, z, qi);
        level<T, KD, ROT, 4, REDUCE, FULL>(tp, U, R, mx, z, qi);
    }
    // this step's shared-memory accesses before later copies into the slots
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(ok)) return false;
    // the planes up to z - kp are used up: their slots take the next ones
    if (threadIdx.x == 0) refill<T, KD>(tp, U, nxt, z - U.kp + kRing, cur, x0, y0);
    return true;
}

// One pass: the units handed out to this CTA, kp sweeps each, from buf[cur]
// to buf[cur ^ 1]; with REDUCE the per-sweep max |delta| of the owned cells
// into s_red[0 .. kp).  False if a TMA wait ran out.
template <class T, int KD, bool REDUCE>
__device__ bool tb3_pass(const JTb3<T> &tp, unsigned char *smem, uint64_t *bars, unsigned *s_red, int *s_unit,
                         unsigned &q, int cur, int kp, const LoopArgs &la, unsigned int *next)
{
    using Sh = Shape3<T>;
    constexpr int kOwnH = kH - 2 * KD;
    const int tid = threadIdx.x;
    const int units = tp.tiles_x * tp.tiles_y * tp.chunks;
    Unit<T, KD> U;
    U.ring = (const T *)smem;
    U.pub = (float *)(smem + kRing * Sh::kSlot);
    U.bars = bars;
    U.pstride = (size_t)tp.ny * (size_t)tp.nx;
    U.kp = kp;
    U.lane = tid & 31;
    U.w = tid >> 5;
    U.ucell = U.ring + U.w * kW + 2 * U.lane;
    U.pubcell = U.pub + U.w * kW + 2 * U.lane;
    U.ghost2 = make_float2(tp.ghost, tp.ghost);
    float mx[KD];
#pragma unroll
    for (int l = 0; l < KD; ++l) mx[l] = 0.0f;
    for (;;) {
        if (tid == 0) *s_unit = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int t = *s_unit;
        if (t >= units) break;
        const int xy = t % (tp.tiles_x * tp.tiles_y), c = t / (tp.tiles_x * tp.tiles_y);
        const int tx = xy % tp.tiles_x, ty = xy / tp.tiles_x;
        const int x0 = tx * kOwnW - kXH, y0 = ty * kOwnH - KD;        // box origin in the grid
        U.z0 = c * kChunk;
        U.z1 = min(tp.nz, U.z0 + kChunk);
        U.zl0 = max(0, U.z0 - kp);
        U.zl1 = min(tp.nz, U.z1 + kp);
        U.zs = U.z0 - kp;
        U.qb = q;
        const int gx = x0 + 2 * U.lane, gy = y0 + U.w;
        const bool xin = gx >= 0 && gx < tp.nx;                       // nx is even: pairs lie wholly inside
        U.gin = xin && gy >= 0 && gy < tp.ny;
        U.rin_n = xin && gy - 1 >= 0 && gy - 1 < tp.ny;
        U.rin_s = xin && gy + 1 >= 0 && gy + 1 < tp.ny;
        U.own_xy = U.gin && U.w >= KD && U.w < kH - KD && 2 * U.lane >= kXH && 2 * U.lane < kXH + kOwnW;
        U.dcell = tp.buf[cur ^ 1] + ((long long)gy * tp.nx + gx);
        // the first loads; the rest follow as slots free up
        int nxt = U.zl0;
        if (tid == 0) refill<T, KD>(tp, U, nxt, U.zl0 + kRing - 1, cur, x0, y0);
        float2 R[KD][3];
#pragma unroll
        for (int l = 0; l < KD; ++l)
#pragma unroll
            for (int j = 0; j < 3; ++j) R[l][j] = U.ghost2;
        const int zend = U.z1 + kp;
        // steps in threes: the register slots of the planes rotate with the
        // step.  Steps [zf0, zf1) have every level's plane in the grid and in
        // its range (level kp: z - kp in [z0, z1); level 1: z - 1 < min(nz, z1 + kp - 1)).
        const int zf0 = max(U.z0, 0) + kp, zf1 = min(U.z1 + kp, tp.nz + 1);
        for (int z = U.zs; z < zend; z += 3) {
            bool ok;
            if (z >= zf0 && z + 2 < zf1) {
                ok = step<T, KD, 0, REDUCE, true>(tp, U, R, mx, z, la, nxt, cur, x0, y0);
                if (ok) ok = step<T, KD, 1, REDUCE, true>(tp, U, R, mx, z + 1, la, nxt, cur, x0, y0);
                if (ok) ok = step<T, KD, 2, REDUCE, true>(tp, U, R, mx, z + 2, la, nxt, cur, x0, y0);
            } else {
                ok = step<T, KD, 0, REDUCE, false>(tp, U, R, mx, z, la, nxt, cur, x0, y0);
                if (ok && z + 1 < zend) ok = step<T, KD, 1, REDUCE, false>(tp, U, R, mx, z + 1, la, nxt, cur, x0, y0);
                if (ok && z + 2 < zend) ok = step<T, KD, 2, REDUCE, false>(tp, U, R, mx, z + 2, la, nxt, cur, x0, y0);
            }
            if (!ok) return false;
        }
        q += (unsigned)(U.zl1 - U.zl0);
        __syncthreads();
    }
    if (REDUCE) {
#pragma unroll
        for (int l = 0; l < KD; ++l) {
            // non-negative binary32 values order as their bits
            const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(mx[l]));
            if (U.lane == 0 && m != 0u && l < kp) atomicMax(&s_red[l], m);
        }
    }
    // this pass's stores before the copies of later passes (after a grid barrier)
    tma::fence_proxy_async_global();
    return true;
}

template <class T, int KD>
__global__ void __launch_bounds__(kThreads, 1) jacobi_tb3_kernel(const __grid_constant__ JTb3<T> tp, LoopArgs la)
{
    extern __shared__ unsigned char smem_dyn[];
    using Sh = Shape3<T>;
    unsigned char *smem = align_up(smem_dyn, 128);
    uint64_t *bars = (uint64_t *)(smem + kRing * Sh::kSlot + Sh::kPubBytes);
    __shared__ unsigned s_red[kJacobiTb3MaxK];
    __shared__ int s_stop, s_rewind, s_unit, s_kpn;
    __shared__ long long s_it;
    const int tid = threadIdx.x;
    Ctl *ctl = la.ctl;
    const long long it0 = ctl->iters;
    if (ctl->converged || it0 >= la.max_iters || ctl->err) return;
    if ((la.debug_flags & SLR_DEBUG_SKIP_ARRIVAL) && blockIdx.x == gridDim.x - 1) return;
    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) tma::mbar_init(bars + i, 1);
        tma::mbar_init_fence();
        tma::fence_proxy_async_global();   // earlier stores to the state before this launch's copies
        s_kpn = tp.K;
    }
    if (tid < kJacobiTb3MaxK) s_red[tid] = 0u;
    __syncthreads();

    unsigned q = 0;                        // TMA plane loads issued by this CTA (mbarrier phases)
    unsigned long long bar_target = 0;
    long long it = it0;
    int cur = 0;
    for (long long p = 0;; ++p) {
        const long long left = la.max_iters - it;
        const int kp = (int)((long long)s_kpn < left ? (long long)s_kpn : left);
        if (!tb3_pass<T, KD, true>(tp, smem, bars, s_red, &s_unit, q, cur, kp, la, &ctl->next_tile[p % kSlots]))
            return;
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
            if (blockIdx.x == 0) {
                zero_slot(&ctl->sub[(p + 2) % kSlots][tid]);
                if (tid == 0) ctl->next_tile[(p + 2) % kSlots] = 0u;
            }
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
                if (!tb3_pass<T, KD, false>(tp, smem, bars, s_red, &s_unit, q, cur, s_rewind, la,
                                            &ctl->next_tile[(p + 1) % kSlots]))
                    return;
                bar_target += (unsigned long long)la.nblocks;
                if (!grid_barrier(ctl, bar_target, la.limit_ns)) return;
            }
            if ((cur ^ 1) == 1)
                grid_copy(tp.buf[1], tp.buf[0], (size_t)tp.nx * tp.ny * (size_t)tp.nz * sizeof(T));
            return;
        }
        cur ^= 1;
        if (tid == 0) tma::fence_proxy_async_global();
    }
}

template <class T> CUtensorMapDataType tb3_type();
template <> CUtensorMapDataType tb3_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> CUtensorMapDataType tb3_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
template <> CUtensorMapDataType tb3_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

template <class T, int KD>
cudaError_t run_tb3(const Problem &p, LoopArgs la, int K, cudaStream_t st)
{
    using Sh = Shape3<T>;
    JTb3<T> tp;
    memset(&tp, 0, sizeof(tp));
    const CUtensorMapDataType dt = tb3_type<T>();
    bool ok = tma::make_map_3d(&tp.umap[0], la.a, dt, sizeof(T), p.nx, p.ny, p.nz, kW, kH, 1) &&
              tma::make_map_3d(&tp.umap[1], la.b, dt, sizeof(T), p.nx, p.ny, p.nz, kW, kH, 1) &&
              tma::make_map_3d(&tp.fmap, la.aux, dt, sizeof(T), p.nx, p.ny, p.nz, kW, kH, 1);
    if (!ok) return cudaErrorNotSupported;
    tp.buf[0] = (T *)la.a;
    tp.buf[1] = (T *)la.b;
    tp.nx = (int)p.nx;
    tp.ny = (int)p.ny;
    tp.nz = (int)p.nz;
    tp.tiles_x = (int)((p.nx + kOwnW - 1) / kOwnW);
    tp.tiles_y = (int)((p.ny + (kH - 2 * KD) - 1) / (kH - 2 * KD));
    tp.chunks = (int)((p.nz + kChunk - 1) / kChunk);
    tp.K = K;
    tp.h2 = p.h2f;
    tp.d = p.df;
    tp.yd = host_rcp_rn(p.df);
    tp.dconst = div_const_ok(p.df);
    tp.ghost = p.ghostf;
    auto kern = jacobi_tb3_kernel<T, KD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::kSmem);
    if (e != cudaSuccess) return e;
    return launch_cooperative(kern, kThreads, Sh::kSmem, 1, la, &tp, st);
}

template <class T>
cudaError_t run_tb3_depth(const Problem &p, LoopArgs la, int K, cudaStream_t st)
{
    return K <= 2 ? run_tb3<T, 2>(p, la, K, st) : run_tb3<T, 4>(p, la, K, st);
}

}  // namespace

bool jacobi_tb3_supported(const Problem &p, const void *a, const void *b, const void *f)
{
    size_t es = 0;
    switch (p.storage) {
    case SLR_F32: es = 4; break;
    case SLR_BF16:
    case SLR_F16: es = 2; break;
    default: return false;
    }
    if (p.stencil != SLR_J3D7 || p.wrap || !jacobi_tb_ghost_exact(p)) return false;
    if ((p.nx * (long long)es) % 16 != 0 || p.nx >= (1ll << 31) - 4096 || p.ny >= (1ll << 31) - 4096 ||
        p.nz >= (1ll << 31) - 4096)
        return false;
    if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)f) % 16 != 0) return false;
    return tma::encode_fn() != nullptr;
}

cudaError_t jacobi_tb3_persistent(const Problem &p, LoopArgs la, int K, cudaStream_t st)
{
    if (K < 2 || K > kJacobiTb3MaxK) return cudaErrorNotSupported;
    switch (p.storage) {
    case SLR_F32: return run_tb3_depth<float>(p, la, K, st);
    case SLR_BF16: return run_tb3_depth<__nv_bfloat16>(p, la, K, st);
    case SLR_F16: return run_tb3_depth<__half>(p, la, K, st);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace slr
