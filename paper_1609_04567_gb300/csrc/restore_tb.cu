// restore_tb.cu -- temporal-blocked restoration (Sec. 4.3): up to 8 sweeps per
// pass over HBM.
//
// The loop-of-stencil-reduce-d of Sec. 3.1 with the restoration update of the
// two-phase denoiser: every noisy pixel becomes the weighted mean of its
// in-range 8-neighbours, w_j = 1 / sqrt(alpha + (u - u_j)^2) (restore_math.cuh),
// clean pixels never change; reduce = mean |u' - u| over the noisy pixels
// (each |delta| truncated to a multiple of 2^-24 and added as an integer), stop
// at the first sweep whose mean is below tol or at the iteration cap.
//
// Tiles.  A pass cuts the grid into tiles of 64 x 64 owned pixels.  A CTA
// loads a tile's state with a halo of 8 pixels on every side (80 x 80 floats)
// into two shared-memory buffers and its mask (96 x 80 bytes, from 16 columns
// to the left so that the copy starts on a 16-byte boundary), three TMA boxes
// on one mbarrier; the hardware fills what lies outside the grid with zeros,
// which no update reads.  The noisy pixels of the loaded region are listed
// once per tile, ordered by their depth: the distance to the nearest edge of
// the loaded region behind which the grid continues (edges on the grid's own
// border do not count, nothing is missing there), capped at 8.  A pixel of
// depth d is up to date after any sweep s <= d, so a pass of kp sweeps runs
// sweep s over the pixels of depth >= s + 8 - kp: a prefix of the list, which
// shrinks by one ring per sweep and ends on the owned pixels (depth 8).  Each
// sweep reads one buffer and writes the other (clean pixels are in both), so
// the update sees only old values, as the Jacobi form of the method requires.
// After kp sweeps the 64 x 64 owned pixels go to the other state buffer in
// global memory with 16-byte stores.
//
// Row pitch.  The tensor maps need rows that start on 16-byte boundaries:
// the mask's (bytes) when nx is a multiple of 16, the state's (floats) when nx
// is a multiple of 4.  Otherwise the run works on copies in the workspace
// whose rows are padded to the next such multiple: the mask copied in at the
// start of a run, the state copied in and, after the loop, back out.  The
// padding columns lie outside the maps' extent (nx), so no copy reads them.
//
// Lists across passes.  The mask does not change, so a tile's list does not
// either: the first pass of a launch lists every noisy pixel of depth >= 1
// and stores the list, its per-depth counts and its owned count in the
// workspace (one fixed-size record per tile); later passes read the record
// while the state arrives, and load no mask.
//
// Reduce and decision.  Each sweep's sum of truncated |delta| over the owned
// noisy pixels goes to a per-sweep slot (warp, then CTA in shared memory,
// then one 64-bit atomic per CTA and sweep), with the count of owned noisy
// pixels.  After a pass a grid barrier publishes the slots; every CTA takes
// the same decision: the first sweep of the pass whose mean is below tol
// stops the loop, and when it is not the pass's last sweep the pass runs
// again from its untouched input up to that sweep, so the state, the value,
// the count and the iteration count equal those of one sweep per pass.
#include <string.h>

#include "restore_math.cuh"
#include "slr_internal.cuh"
#include "tma.cuh"

namespace slr {
namespace {

constexpr int kK = 8;                        // most sweeps per pass: the tile halo
constexpr int kOwn = 64;                     // owned pixels per tile side
constexpr int kW = kOwn + 2 * kK;            // 80: loaded columns (x0 - 8 .. x0 + 71)
constexpr int kH = kOwn + 2 * kK;            // 80: loaded rows
constexpr int kMX = 16;                      // mask halo columns (16-byte aligned start)
constexpr int kMW = kOwn + 2 * kMX;          // 96 mask bytes per row
constexpr int kThreads = 256;
constexpr int kPlane = kW * kH * 4;                                   // 25600
constexpr int kMaskBytes = kMW * kH;                                  // 7680
constexpr int kMaxList = (kW - 2) * (kH - 2);                         // pixels that can be updated
constexpr int kListBytes = (kMaxList * 2 + 127) / 128 * 128;
constexpr size_t kSmem = 128 + 2 * (size_t)kPlane + kMaskBytes + kListBytes + 16;
constexpr uint32_t kTxBytes = 2u * kPlane + kMaskBytes;               // what the three boxes deliver
static_assert(kPlane % 128 == 0 && kMaskBytes % 128 == 0, "TMA destinations stay 128-byte aligned");
static_assert(kW * kH < (1 << 14), "a list entry keeps the position in 14 bits");
static_assert(kK <= kMaxK, "per-sweep slots");
static_assert((kW * kH) % kThreads == 0, "the listing loops run whole warps");
// a tile's stored list: counts (nge[0 .. kK + 1], owned) in 64 bytes, then the entries
constexpr int kRecHead = 64;
constexpr size_t kRecBytes = kRecHead + (size_t)kListBytes;
static_assert(kListBytes % 16 == 0 && (kK + 3) * 4 <= kRecHead, "record layout");

struct RTb {
    CUtensorMap umap[2];       // state buffers A (caller's u) and B, box 80 x 80
    CUtensorMap mmap;          // mask, box 96 x 80
    float *buf[2];
    long long pitch;           // floats per row of buf[0] and buf[1]
    int nx, ny;
    int tiles_x, tiles_y;
    int K;                     // sweeps per pass
    float alpha;
    int alpha_in_range;        // restore_alpha_in_range(alpha)
    unsigned char *lists;      // one kRecBytes record per tile (workspace)
};

// Per-CTA bookkeeping in static shared memory.
struct RTbShared {
    int cnt[kK + 1];                    // noisy pixels per depth
    int next[kK + 1];                   // placement cursor per depth
    int nge[kK + 2];                    // listed pixels of depth >= d
    unsigned owned;                     // owned noisy pixels of the tile
    int tile;                           // the tile this CTA works on
    unsigned long long sum[kK];         // per-sweep sum over the CTA's tiles
    unsigned long long own_total;       // owned noisy pixels over the CTA's tiles
};

__device__ __forceinline__ int tile_depth(int ly, int lx, bool top, bool bottom, bool left, bool right)
{
    int d = kK;
    if (top) d = min(d, ly);
    if (bottom) d = min(d, kH - 1 - ly);
    if (left) d = min(d, lx);
    if (right) d = min(d, kW - 1 - lx);
    return d;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One pass: kp sweeps of every tile, from buf[cur] to buf[cur ^ 1]; the
// CTAs take tiles from the counter *next as they finish the previous one, so
// tiles with more noisy pixels even out.  With REDUCE the per-sweep sums go
// to sh.sum and the owned noisy pixels to sh.own_total.  False if a TMA wait
// ran out.
template <bool FAST, bool REDUCE>
__device__ bool rtb_pass(const RTb &tp, unsigned char *smem, uint64_t *bar, RTbShared &sh, unsigned &phase, int cur,
                         int kp, const LoopArgs &la, unsigned int *next, bool cached)
{
    float *S0 = (float *)smem;
    float *S1 = (float *)(smem + kPlane);
    const unsigned char *M = smem + 2 * kPlane;
    unsigned short *L = (unsigned short *)(smem + 2 * kPlane + kMaskBytes);
    float *dst = tp.buf[cur ^ 1];
    const int tid = threadIdx.x, lane = tid & 31;
    const int ntiles = tp.tiles_x * tp.tiles_y;
    for (;;) {
        if (tid == 0) sh.tile = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int t = sh.tile;
        if (t >= ntiles) break;
        const int x0 = (t % tp.tiles_x) * kOwn, y0 = (t / tp.tiles_x) * kOwn;
        const int X0 = x0 - kK, Y0 = y0 - kK;    // origin of the loaded region in the grid
        unsigned char *rec = tp.lists + (size_t)t * kRecBytes;
        if (tid == 0) {
            tma::mbar_expect_tx(bar, cached ? 2u * kPlane : kTxBytes);
            tma::load_2d(S0, &tp.umap[cur], X0, Y0, bar);
            tma::load_2d(S1, &tp.umap[cur], X0, Y0, bar);
            if (!cached) tma::load_2d((void *)M, &tp.mmap, x0 - kMX, Y0, bar);
        }
        if (cached) {
            // the stored record, read while the state arrives
            const int *head = (const int *)rec;
            if (tid < kK + 2) sh.nge[tid] = __ldcg(head + tid);
            if (tid == kK + 2) sh.owned = (unsigned)__ldcg(head + kK + 2);
            const int n = __ldcg(head + 1);
            const uint4 *src = (const uint4 *)(rec + kRecHead);
            for (int i = tid; i < (2 * n + 15) / 16; i += kThreads) ((uint4 *)L)[i] = __ldcg(src + i);
        } else {
            if (tid <= kK) sh.cnt[tid] = 0;
            if (tid == 0) sh.owned = 0u;
        }
        const bool ok = tma::bounded_wait(bar, phase & 1u, tma::kLoadWaitNs, &la.ctl->err);
        ++phase;
        if (!__syncthreads_and(ok)) return false;
        // edges of the loaded region behind which the grid continues; a
        // tile that reaches none of the grid's borders has all its pixels'
        // neighbours in the grid
        const bool top = Y0 > 0, bottom = Y0 + kH < tp.ny, left = X0 > 0, right = X0 + kW < tp.nx;
        const bool edge_tile = !(top && bottom && left && right);
        // list the noisy pixels by depth: count, place (the lanes of a warp
        // that share a depth add once, by their first lane)
        // and check that every loaded value is below 2^60 in magnitude: the
        // pass's weighted means then stay below 2^61 and the weights can skip
        // their range checks (restore_interior_in_range)
        const unsigned lt = (1u << lane) - 1u;
        bool small = true;
        if (cached) {
            for (int i = tid; i < kW * kH; i += kThreads) small = small && fabsf(S0[i]) < 0x1p60f;
        } else {
            for (int i = tid; i < kW * kH; i += kThreads) {
                const int ly = i / kW, lx = i - ly * kW;
                const int gy = Y0 + ly, gx = X0 + lx;
                const bool noisy = gy >= 0 && gy < tp.ny && gx >= 0 && gx < tp.nx && M[ly * kMW + lx + (kMX - kK)];
                const int d = tile_depth(ly, lx, top, bottom, left, right);
                const bool listed = noisy && d >= 1;
                const unsigned peers = __match_any_sync(0xffffffffu, listed ? d : -1);
                if (listed && (peers & lt) == 0u) atomicAdd(&sh.cnt[d], __popc(peers));
                small = small && fabsf(S0[i]) < 0x1p60f;           // false for a NaN
            }
        }
        const bool in_range = __syncthreads_and(small) && tp.alpha_in_range;
        if (!cached) {
        if (tid == 0) {
            int pos = 0;
            sh.nge[kK + 1] = 0;
            for (int d = kK; d >= 1; --d) {
                sh.next[d] = pos;
                pos += sh.cnt[d];
                sh.nge[d] = pos;
            }
            sh.nge[0] = pos;
        }
        __syncthreads();
        for (int i = tid; i < kW * kH; i += kThreads) {
            const int ly = i / kW, lx = i - ly * kW;
            const int gy = Y0 + ly, gx = X0 + lx;
            const bool noisy = gy >= 0 && gy < tp.ny && gx >= 0 && gx < tp.nx && M[ly * kMW + lx + (kMX - kK)];
            const int d = tile_depth(ly, lx, top, bottom, left, right);
            const bool listed = noisy && d >= 1;
            const unsigned peers = __match_any_sync(0xffffffffu, listed ? d : -1);
            const int first = __ffs(peers) - 1;
            int base = 0;
            if (listed && lane == first) base = atomicAdd(&sh.next[d], __popc(peers));
            base = __shfl_sync(0xffffffffu, base, first);
            const bool own = listed && ly >= kK && ly < kK + kOwn && lx >= kK && lx < kK + kOwn;
            const bool border = gy == 0 || gy == tp.ny - 1 || gx == 0 || gx == tp.nx - 1;
            if (listed)
                L[base + __popc(peers & lt)] = (unsigned short)(i | (own ? 1 << 14 : 0) | (border ? 1 << 15 : 0));
            const unsigned owners = __ballot_sync(0xffffffffu, own);
            if (lane == 0 && owners) atomicAdd(&sh.owned, (unsigned)__popc(owners));
        }
        __syncthreads();
        // store the record for the later passes of this launch
        int *head = (int *)rec;
        if (tid < kK + 2) head[tid] = sh.nge[tid];
        if (tid == kK + 2) head[kK + 2] = (int)sh.owned;
        const int nl = sh.nge[1];
        for (int i = tid; i < (2 * nl + 15) / 16; i += kThreads) ((uint4 *)(rec + kRecHead))[i] = ((const uint4 *)L)[i];
        }
        for (int s = 1; s <= kp; ++s) {
            const float *In = (s & 1) ? S0 : S1;
            float *Out = (s & 1) ? S1 : S0;
            const int n = sh.nge[s + kK - kp];
            unsigned long long sum = 0ull;
            if (!FAST && in_range && !edge_tile) {
                // the common case, with no branch per pixel: no pixel on the
                // grid's border, weights without range checks
                for (int e = tid; e < n; e += kThreads) {
                    const unsigned ent = L[e];
                    const int pos = (int)(ent & 0x3FFFu);
                    const float *C = In + pos;
                    const float nv = restore_interior_in_range(C, kW, tp.alpha);
                    Out[pos] = nv;
                    if (REDUCE) {
                        const unsigned long long fx = fixed_2m24_nb(__fsub_rn(nv, *C));
                        sum += (ent & 0x4000u) ? fx : 0ull;
                    }
                }
            } else {
                for (int e = tid; e < n; e += kThreads) {
                    const unsigned ent = L[e];
                    const int pos = (int)(ent & 0x3FFFu);
                    const float *C = In + pos;
                    float nv;
                    if (ent & 0x8000u) {
                        const int gy = Y0 + pos / kW, gx = X0 + pos % kW;
                        nv = restore_border<FAST>(C, kW, tp.alpha, gy > 0, gy + 1 < tp.ny, gx > 0, gx + 1 < tp.nx);
                    } else if (!FAST && in_range) {
                        nv = restore_interior_in_range(C, kW, tp.alpha);
                    } else {
                        nv = restore_interior<FAST>(C, kW, tp.alpha);
                    }
                    Out[pos] = nv;
                    if (REDUCE && (ent & 0x4000u)) sum += fixed_2m24(__fsub_rn(nv, *C));
                }
            }
            if (REDUCE) {
                sum = warp_sum_u64(sum);
                if (lane == 0 && sum) atomicAdd(&sh.sum[s - 1], sum);
            }
            __syncthreads();
        }
        if (REDUCE && tid == 0) sh.own_total += sh.owned;
        // the owned pixels inside the grid to the output buffer
        const float *Fin = (kp & 1) ? S1 : S0;
        for (int i = tid; i < kOwn * (kOwn / 4); i += kThreads) {
            const int r = i / (kOwn / 4), c4 = i % (kOwn / 4);
            const int gy = y0 + r, gx = x0 + 4 * c4;
            if (gy < tp.ny && gx < tp.nx)
                *(float4 *)(dst + (size_t)gy * (size_t)tp.pitch + gx) = *(const float4 *)(Fin + (r + kK) * kW + kK + 4 * c4);
        }
        // this tile's shared-memory accesses before the next tile's copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    // this pass's stores before the copies of later passes (after a grid barrier)
    tma::fence_proxy_async_global();
    return true;
}

template <bool FAST>
__global__ void __launch_bounds__(kThreads, 3) restore_tb_kernel(const __grid_constant__ RTb tp, LoopArgs la)
{
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem = align_up(smem_dyn, 128);
    uint64_t *bar = (uint64_t *)(smem + 2 * kPlane + kMaskBytes + kListBytes);
    __shared__ RTbShared sh;
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
        sh.own_total = 0ull;
    }
    if (tid < kK) sh.sum[tid] = 0ull;
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
        if (!rtb_pass<FAST, true>(tp, smem, bar, sh, phase, cur, kp, la, &ctl->next_tile[p % kSlots], p > 0)) return;
        __syncthreads();
        if (tid < kp) {
            Slot *sl = &ctl->sub[p % kSlots][tid];
            if (sh.sum[tid]) atomicAdd(&sl->sum, sh.sum[tid]);
            if (sh.own_total) atomicAdd(&sl->cnt, sh.own_total);
            sh.sum[tid] = 0ull;
        }
        __syncthreads();
        if (tid == 0) sh.own_total = 0ull;
        bar_target += (unsigned long long)la.nblocks;
        if (!grid_barrier(ctl, bar_target, la.limit_ns)) return;
        if (tid < 32) {
            if (blockIdx.x == 0) {
                zero_slot(&ctl->sub[(p + 2) % kSlots][tid]);
                if (tid == 0) ctl->next_tile[(p + 2) % kSlots] = 0u;
            }
            // lane j decides sweep j of the pass; the first one below tol stops
            Slot sl;
            sl.maxbits = 0ull;
            sl.sum = tid < kp ? ld_relaxed_u64(&ctl->sub[p % kSlots][tid].sum) : 0ull;
            sl.cnt = tid < kp ? ld_relaxed_u64(&ctl->sub[p % kSlots][tid].cnt) : 0ull;
            sl.changed = sl.sum != 0ull;
            const Decision dj = decide(la.reduce, sl, la.tol);
            const unsigned conv = __ballot_sync(0xffffffffu, tid < kp && dj.converged);
            const int jstop = conv ? __ffs(conv) - 1 : -1;
            const int jlast = jstop >= 0 ? jstop : kp - 1;
            const double value = __shfl_sync(0xffffffffu, dj.value, jlast);
            const unsigned long long count = __shfl_sync(0xffffffffu, dj.count, jlast);
            const int changed = __shfl_sync(0xffffffffu, dj.changed, jlast);
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
                    ctl->count = count;
                    ctl->changed = changed;
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
                if (!rtb_pass<FAST, false>(tp, smem, bar, sh, phase, cur, s_rewind, la,
                                           &ctl->next_tile[(p + 1) % kSlots], true))
                    return;
                bar_target += (unsigned long long)la.nblocks;
                if (!grid_barrier(ctl, bar_target, la.limit_ns)) return;
            }
            if ((cur ^ 1) == 1) grid_copy(tp.buf[1], tp.buf[0], (size_t)tp.pitch * tp.ny * sizeof(float));
            return;
        }
        cur ^= 1;
        if (tid == 0) tma::fence_proxy_async_global();
    }
}

// state buffers la.a / la.b with `pitch` floats per row, mask rows `mpitch` bytes
template <bool FAST>
cudaError_t run_rtb(const Problem &p, LoopArgs la, int K, void *lists, const void *mask, long long pitch,
                    long long mpitch, cudaStream_t st)
{
    RTb tp;
    memset(&tp, 0, sizeof(tp));
    const auto none = CU_TENSOR_MAP_SWIZZLE_NONE;
    if (!tma::make_map_2d(&tp.umap[0], la.a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p.nx, p.ny, kW, kH, none, 4 * pitch) ||
        !tma::make_map_2d(&tp.umap[1], la.b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p.nx, p.ny, kW, kH, none, 4 * pitch) ||
        !tma::make_map_2d(&tp.mmap, mask, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, p.nx, p.ny, kMW, kH, none, mpitch))
        return cudaErrorNotSupported;
    tp.buf[0] = (float *)la.a;
    tp.buf[1] = (float *)la.b;
    tp.pitch = pitch;
    tp.nx = (int)p.nx;
    tp.ny = (int)p.ny;
    tp.tiles_x = (int)((p.nx + kOwn - 1) / kOwn);
    tp.tiles_y = (int)((p.ny + kOwn - 1) / kOwn);
    tp.K = K;
    tp.alpha = p.alpha;
    tp.alpha_in_range = restore_alpha_in_range(p.alpha);
    tp.lists = (unsigned char *)lists;
    auto kern = restore_tb_kernel<FAST>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    return launch_cooperative(kern, kThreads, kSmem, 3, la, &tp, st);
}

}  // namespace

namespace {
// padded row pitches (see the header comment)
bool mask_padded(long long nx) { return nx % 16 != 0; }
bool state_padded(long long nx) { return nx % 4 != 0; }
long long mask_pitch(long long nx) { return (nx + 15) / 16 * 16; }
long long state_pitch(long long nx) { return (nx + 3) / 4 * 4; }
size_t up256(size_t x) { return (x + 255) / 256 * 256; }
size_t records_bytes(long long nx, long long ny)
{
    return up256((size_t)((nx + kOwn - 1) / kOwn) * (size_t)((ny + kOwn - 1) / kOwn) * kRecBytes);
}
size_t mask_copy_bytes(long long nx, long long ny)
{
    return mask_padded(nx) ? up256((size_t)mask_pitch(nx) * (size_t)ny) : 0;
}
size_t state_copy_bytes(long long nx, long long ny)      // one of the two buffers
{
    return state_padded(nx) ? up256((size_t)state_pitch(nx) * (size_t)ny * sizeof(float)) : 0;
}
}  // namespace

bool restore_tb_supported(const Problem &p, const void *a, const void *b, const void *mask)
{
    if (p.stencil != SLR_RESTORE8 || p.nx >= (1ll << 31) - 4096 || p.ny >= (1ll << 31) - 4096) return false;
    // buffers the maps read in place must start on 16-byte boundaries
    if (!state_padded(p.nx) && (((uintptr_t)a | (uintptr_t)b) % 16) != 0) return false;
    if (!mask_padded(p.nx) && ((uintptr_t)mask % 16) != 0) return false;
    if ((double)p.nx * (double)p.ny >= 4.0e18) return false;
    return tma::encode_fn() != nullptr;
}

int restore_tb_resolve_k(const Problem &p, const void *a, const void *b, const void *mask)
{
    if (p.k == 1 || !restore_tb_supported(p, a, b, mask)) return 1;
    if (p.k == 0) return p.tiling == SLR_TILING_AUTO ? kRestoreTbDefaultK : 1;
    return p.k > kK ? kK : p.k;
}

size_t restore_tb_list_bytes(long long nx, long long ny)
{
    return records_bytes(nx, ny) + mask_copy_bytes(nx, ny) + 2 * state_copy_bytes(nx, ny);
}

cudaError_t restore_tb_persistent(const Problem &p, LoopArgs la, void *lists, cudaStream_t st)
{
    const int K = restore_tb_resolve_k(p, la.a, la.b, la.aux);
    if (K < 2 || !lists || ((uintptr_t)lists % 256) != 0) return cudaErrorNotSupported;
    unsigned char *scratch = (unsigned char *)lists + records_bytes(p.nx, p.ny);
    const void *mask = la.aux;
    long long mpitch = p.nx, pitch = p.nx;
    cudaError_t e = cudaSuccess;
    if (mask_padded(p.nx)) {
        mpitch = mask_pitch(p.nx);
        e = cudaMemcpy2DAsync(scratch, (size_t)mpitch, la.aux, (size_t)p.nx, (size_t)p.nx, (size_t)p.ny,
                              cudaMemcpyDeviceToDevice, st);
        mask = scratch;
        scratch += mask_copy_bytes(p.nx, p.ny);
    }
    LoopArgs lp = la;
    const size_t row = (size_t)p.nx * sizeof(float);
    if (state_padded(p.nx)) {
        pitch = state_pitch(p.nx);
        lp.a = scratch;
        lp.b = scratch + state_copy_bytes(p.nx, p.ny);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(lp.a, (size_t)pitch * sizeof(float), la.a, row, row, (size_t)p.ny,
                                  cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess) return e;
    e = p.math == SLR_MATH_FAST ? run_rtb<true>(p, lp, K, lists, mask, pitch, mpitch, st)
                                : run_rtb<false>(p, lp, K, lists, mask, pitch, mpitch, st);
    // the loop leaves its state in lp.a
    if (e == cudaSuccess && state_padded(p.nx))
        e = cudaMemcpy2DAsync(la.a, row, lp.a, (size_t)pitch * sizeof(float), row, (size_t)p.ny,
                              cudaMemcpyDeviceToDevice, st);
    return e;
}

}  // namespace slr
