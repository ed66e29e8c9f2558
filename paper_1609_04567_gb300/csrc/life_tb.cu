// life_tb.cu -- temporal-blocked Game of Life: K generations per pass over a
// bit-packed grid.
//
// The loop-of-stencil-reduce of Sec. 3.1 with the Fig. 1 elemental function
// (B3/S23), restructured for GB300.  One cooperative persistent launch does:
//
//  P. Pack: the caller's uint8 grid (any non-zero byte is a live cell) is
//     staged through shared memory by TMA
//     (cp.async.bulk.tensor.2d, 32-row x 128-byte boxes with the 128B swizzle,
//     double buffered) and packed to 1 bit per cell (bit b of word w = column
//     32w + b) into a workspace buffer.  Boxes wholly outside the grid are not
//     loaded; the hardware fills the outside of partly-outside boxes with
//     zeros.
//  G. Passes: each pass reads the packed grid, runs up to K generations on
//     chip, and writes the packed grid to the other workspace buffer.  A tile
//     is 1024 owned columns (plus one 32-cell word of halo on each side) by
//     482 - 2K owned rows (plus K halo rows above and below); K generations
//     stay exact inside it.  Thread (w, l) of the 16 warps holds tile row
//     30w + l as 34 words in registers, so warps overlap by two rows: lanes
//     1..30 are the warp's own rows, lanes 0 and 31 are copies of the
//     neighbour warps' edge rows, refreshed through shared memory after every
//     generation.  Per generation every thread forms its row's horizontal
//     2-bit sums (left + self + right, and left + right) with two funnel shifts
//     and four logic operations, takes the rows above and below by shuffle,
//     and finishes the B3/S23 rule with six more logic operations: twelve per
//     32 cells.  "Any cell changed" is reduced over the owned cells in the
//     pass's last generation, the live count too (see the decision below).
//  U. Unpack: the final packed grid is expanded back into the caller's uint8
//     grid.
//
// After each pass a bounded grid barrier publishes the reduces and every CTA
// takes the same decision: stop at the first generation that changed nothing
// (a still state is a fixed point, so the packed state at the end of the pass
// equals it), or at the iteration cap (the last pass runs only the generations
// left).  A pass whose last generation changed nothing reached its still state
// at some generation of the pass; it runs again from its input with a
// "changed" flag per generation to find the first.  The dead border stays dead: cells of a tile
// outside the grid are cleared after every generation.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "slr_internal.cuh"
#include "tma.cuh"

namespace slr {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kRowsPerWarp = 30;                      // own rows of a warp (lanes 1..30)
constexpr int kTileRows = kWarps * kRowsPerWarp + 2;  // 482 distinct tile rows
constexpr int kWords = 34;                            // 1 halo + 32 owned + 1 halo
constexpr int kOwnWords = 32;
constexpr int kOwnCols = 32 * kOwnWords;              // 1024
constexpr int kXchStride = 36;                        // exchange row stride in words (16-byte aligned rows)
constexpr int kXchWords = 2 * kWarps * 2 * kXchStride; // [parity][warp][lane 1 row, lane 30 row][word]
// pack phase: 32 rows x 1024 columns per unit, 8 swizzled boxes of 128 bytes
constexpr int kPackRows = 32;
constexpr int kBoxW = 128;
constexpr int kBoxes = kOwnCols / kBoxW;              // 8
constexpr int kBoxBytes = kBoxW * kPackRows;          // 4096
constexpr int kStageBytes = kBoxes * kBoxBytes;       // 32768
constexpr size_t kSmemBytes = 1024 + 2 * kStageBytes + kXchWords * 4 + 2 * 8 + kMaxK * 8 + kMaxK * 4;
static_assert((kXchWords * 4) % 16 == 0 && (2 * kStageBytes) % 16 == 0, "exchange rows and mbarriers stay aligned");
static_assert(kMaxK == 32, "one lane per generation in the per-pass decision");

struct TbParams {
    CUtensorMap cells;           // uint8 view of the caller's grid (box 128 x 32, 128B swizzle)
    unsigned int *bits[2];       // packed ping-pong buffers (workspace)
    long long nx, ny;            // grid extents (nx % 32 == 0)
    long long nxw, pitch;        // words per row, row pitch in words (multiple of 4)
    int wrap, K, own_rows, tiles_x, tiles_y;
};

// ---- cell packing -----------------------------------------------------------
// Four 0/1 bytes -> 4 bits (byte i -> bit i): the partial products land on
// distinct bit positions 24..27, so the multiply adds no carries.
__device__ __forceinline__ uint32_t pack4(uint32_t w) { return (w * 0x01020408u) >> 24; }

// Any non-zero byte reads as a live cell: fold each byte's bits into its bit 0
// (shifts by 4, 2, 1 stay inside the byte for the low bits kept).
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t w)
{
    w |= w >> 4;
    w |= w >> 2;
    w |= w >> 1;
    return w & 0x01010101u;
}

__device__ __forceinline__ uint32_t pack16(const uint4 v)
{
    return pack4(nonzero_bytes(v.x)) | (pack4(nonzero_bytes(v.y)) << 4) | (pack4(nonzero_bytes(v.z)) << 8) |
           (pack4(nonzero_bytes(v.w)) << 12);
}

// 4 bits -> four 0/1 bytes (bit i -> byte i): copies of the nibble at shifts
// 0, 7, 14, 21 do not overlap, so bit i lands alone at bit 8i.
__device__ __forceinline__ uint32_t unpack4(uint32_t n) { return (n * 0x00204081u) & 0x01010101u; }

__device__ __forceinline__ uint4 unpack16(uint32_t h)
{
    return make_uint4(unpack4(h & 15u), unpack4((h >> 4) & 15u), unpack4((h >> 8) & 15u), unpack4((h >> 12) & 15u));
}

__device__ __forceinline__ long long wrap_mod(long long v, long long n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// ---- phase P: uint8 -> bits ---------------------------------------------------
__device__ __forceinline__ void issue_pack_unit(const TbParams &tp, int unit, unsigned char *stage, uint64_t *bar)
{
    const int cbs = (int)((tp.nx + kOwnCols - 1) / kOwnCols);
    const long long y = (long long)(unit / cbs) * kPackRows;
    const long long x0 = (long long)(unit % cbs) * kOwnCols;
    uint32_t bytes = 0;
    for (int b = 0; b < kBoxes; ++b)
        if (x0 + (long long)b * kBoxW < tp.nx) bytes += kBoxBytes;
    tma::mbar_expect_tx(bar, bytes);
    for (int b = 0; b < kBoxes; ++b)
        if (x0 + (long long)b * kBoxW < tp.nx)
            tma::load_2d(stage + b * kBoxBytes, &tp.cells, (int)(x0 + (long long)b * kBoxW), (int)y, bar);
}

__device__ bool pack_phase(const TbParams &tp, unsigned char *stage, uint64_t *mbar, int *s_ok, int *err)
{
    const int tid = threadIdx.x;
    const int cbs = (int)((tp.nx + kOwnCols - 1) / kOwnCols);
    const int units = (int)((tp.ny + kPackRows - 1) / kPackRows) * cbs;
    const int mine = (int)blockIdx.x < units ? (units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    unsigned int *dst = tp.bits[0];
    // unit i of this CTA uses staging buffer i & 1, phase (i >> 1) & 1 of its mbarrier
    if (tid == 0)
        for (int i = 0; i < 2 && i < mine; ++i)
            issue_pack_unit(tp, (int)blockIdx.x + i * (int)gridDim.x, stage + (i & 1) * kStageBytes, &mbar[i & 1]);
    for (int i = 0; i < mine; ++i) {
        const int unit = (int)blockIdx.x + i * (int)gridDim.x;
        const int sb = i & 1;
        if (tid == 0) *s_ok = tma::bounded_wait(&mbar[sb], (uint32_t)(i >> 1) & 1u, tma::kLoadWaitNs, err);
        __syncthreads();
        if (!*s_ok) return false;
        const long long y0 = (long long)(unit / cbs) * kPackRows;
        const long long xw0 = (long long)(unit % cbs) * kOwnWords;
        const unsigned char *sbase = stage + sb * kStageBytes;
#pragma unroll
        for (int it = 0; it < (kPackRows * kOwnWords) / kThreads; ++it) {   // 32 rows x 32 words
            const int item = tid + it * kThreads;
            const int rr = item >> 5, w = item & 31;                        // one warp = one row
            const int box = w >> 2, c0 = (w & 3) * 2;                       // 4 words per 128-byte box row
            const long long y = y0 + rr, xw = xw0 + w;
            if (y >= tp.ny || xw >= tp.nxw) continue;
            const unsigned char *row = sbase + box * kBoxBytes + rr * kBoxW;
            const uint4 lo = *(const uint4 *)(row + ((c0 ^ (rr & 7)) << 4));
            const uint4 hi = *(const uint4 *)(row + (((c0 + 1) ^ (rr & 7)) << 4));
            dst[y * tp.pitch + xw] = pack16(lo) | (pack16(hi) << 16);
        }
        __syncthreads();
        const int nxt = i + 2;
        if (tid == 0 && nxt < mine)
            issue_pack_unit(tp, (int)blockIdx.x + nxt * (int)gridDim.x, stage + sb * kStageBytes, &mbar[sb]);
    }
    return true;
}

// ---- phase G: one tile of one pass ---------------------------------------------
// Word xw of a packed row, with wrap-around or the dead border in x.
__device__ __forceinline__ uint32_t load_word(const TbParams &tp, const unsigned int *row, long long xw)
{
    if (xw < 0 || xw >= tp.nxw) {
        if (!tp.wrap) return 0u;
        xw = wrap_mod(xw, tp.nxw);
    }
    return __ldcg(row + xw);
}

// Named barrier `id` (1..kWarps-1) for the two warps id - 1 and id.
__device__ __forceinline__ void pair_sync(int id)
{
    asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// One generation of a thread's row (34 words in registers, updated in place):
// horizontal 2-bit sums by funnel shifts and logic, the rows above and below
// by shuffle, the B3/S23 rule.  With TRACK `changed` collects owned cells that
// changed; in the pass's last generation (LAST) `cnt` counts the owned live
// cells.
template <bool WRAP, bool FULL, bool LAST, bool TRACK>
__device__ __forceinline__ void generation(uint32_t (&cur)[kWords], bool own, int own_words, bool row_in, int wlo,
                                           int whi, uint32_t &changed, uint32_t &cnt)
{
    uint32_t prevC = 0u, C = cur[0];
#pragma unroll
    for (int w = 0; w < kWords; ++w) {
        const uint32_t nextC = w + 1 < kWords ? cur[w + 1] : 0u;
        const uint32_t L = __funnelshift_l(prevC, C, 1);   // left neighbours (bit b-1)
        const uint32_t R = __funnelshift_r(C, nextC, 1);   // right neighbours (bit b+1)
        const uint32_t s0 = L ^ C ^ R, s1 = (L & C) | (L & R) | (C & R);   // L + C + R
        const uint32_t m0 = L ^ R, m1 = L & R;                              // L + R
        const uint32_t u0 = __shfl_up_sync(0xffffffffu, s0, 1), u1 = __shfl_up_sync(0xffffffffu, s1, 1);
        const uint32_t d0 = __shfl_down_sync(0xffffffffu, s0, 1), d1 = __shfl_down_sync(0xffffffffu, s1, 1);
        // n = (u0 + m0 + d0) + 2 (u1 + m1 + d1) = bit0 + 2 (c0 + u1 + m1 + d1)
        const uint32_t bit0 = u0 ^ m0 ^ d0, c0 = (u0 & m0) | (u0 & d0) | (m0 & d0);
        const uint32_t x = u1 ^ m1 ^ d1, yy = (u1 & m1) | (u1 & d1) | (m1 & d1);
        uint32_t nw = ((x ^ c0) & ~yy) & (C | bit0);       // n == 3, or n == 2 and alive
        if (!WRAP && !(row_in && w >= wlo && w <= whi)) nw = 0u;
        if (w >= 1 && w <= kOwnWords && own && (FULL || w <= own_words)) {
            if (TRACK) changed |= nw ^ C;
            if (LAST) cnt += (uint32_t)__popc(nw);
        }
        prevC = C;
        cur[w] = nw;
        C = nextC;
    }
}

// `exact`: track "changed" in every generation, else in the last one only
template <bool WRAP>
__device__ __forceinline__ void run_tile(const TbParams &tp, int tile, int kp, int exact, const unsigned int *src,
                                         unsigned int *dst, uint32_t *xch, unsigned long long *s_cnt,
                                         unsigned int *s_ch)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tile % tp.tiles_x, ty = tile / tp.tiles_x;
    const long long xw0 = (long long)tx * kOwnWords;
    const int trow = warp * kRowsPerWarp + lane;                     // tile row of this thread
    const long long yf = (long long)ty * tp.own_rows - tp.K + trow;  // grid row before wrapping
    long long y = yf;
    bool row_in = true;
    if (WRAP) y = wrap_mod(yf, tp.ny);
    else row_in = yf >= 0 && yf < tp.ny;

    // load the row: 32 owned words and one halo word on each side
    uint32_t cur[kWords];
    if (row_in) {
        const unsigned int *row = src + y * tp.pitch;
        if (xw0 + kOwnWords <= tp.nxw) {
            const uint4 *v = (const uint4 *)(row + xw0);
#pragma unroll
            for (int i = 0; i < kOwnWords / 4; ++i) {
                const uint4 q4 = __ldcg(v + i);
                cur[1 + 4 * i] = q4.x; cur[2 + 4 * i] = q4.y; cur[3 + 4 * i] = q4.z; cur[4 + 4 * i] = q4.w;
            }
        } else {
#pragma unroll
            for (int w = 1; w <= kOwnWords; ++w) cur[w] = load_word(tp, row, xw0 + w - 1);
        }
        cur[0] = load_word(tp, row, xw0 - 1);
        cur[kWords - 1] = load_word(tp, row, xw0 + kOwnWords);
    } else {
#pragma unroll
        for (int w = 0; w < kWords; ++w) cur[w] = 0u;
    }
    // word w of the tile holds grid word xw0 + w - 1; with the dead border only
    // words [wlo, whi] lie inside the grid
    const long long wmax = tp.nxw - xw0;
    const int wlo = (WRAP || xw0 > 0) ? 0 : 1;
    const int whi = WRAP ? kWords - 1 : (int)(wmax < kWords - 1 ? wmax : kWords - 1);
    // reduce and store ownership: the warp's own lanes, owned tile rows, rows
    // inside the grid (the last band of tiles may reach past it)
    const bool own = lane >= 1 && lane <= kRowsPerWarp && trow >= tp.K && trow < kTileRows - tp.K &&
                     (long long)ty * tp.own_rows + (trow - tp.K) < tp.ny;
    const int own_words = (int)(wmax < kOwnWords ? wmax : kOwnWords);

    for (int j = 0; j < kp; ++j) {
        uint32_t changed = 0u, cnt = 0u;
        // full tiles (every owned word inside the grid) drop the per-word
        // bound; the live count is taken in the pass's last generation only
        if (own_words == kOwnWords) {
            if (j == kp - 1) generation<WRAP, true, true, true>(cur, own, own_words, row_in, wlo, whi, changed, cnt);
            else if (exact) generation<WRAP, true, false, true>(cur, own, own_words, row_in, wlo, whi, changed, cnt);
            else generation<WRAP, true, false, false>(cur, own, own_words, row_in, wlo, whi, changed, cnt);
        } else {
            if (j == kp - 1) generation<WRAP, false, true, true>(cur, own, own_words, row_in, wlo, whi, changed, cnt);
            else if (exact) generation<WRAP, false, false, true>(cur, own, own_words, row_in, wlo, whi, changed, cnt);
            else generation<WRAP, false, false, false>(cur, own, own_words, row_in, wlo, whi, changed, cnt);
        }
        // refresh the two copied rows from the neighbour warps (exchange rows
        // double buffered by generation parity; 16-byte shared-memory
        // accesses).  Each warp synchronises with its two neighbours only:
        // named barrier w + 1 joins warps w and w + 1; even warps take the one
        // below first, odd warps the one above, so pairs never wait in a chain
        uint32_t *xb = xch + (j & 1) * kWarps * 2 * kXchStride;
        if (lane == 1 || lane == kRowsPerWarp) {
            uint32_t *row = xb + (warp * 2 + (lane == 1 ? 0 : 1)) * kXchStride;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                ((uint4 *)row)[i] = make_uint4(cur[4 * i], cur[4 * i + 1], cur[4 * i + 2], cur[4 * i + 3]);
            ((uint2 *)row)[16] = make_uint2(cur[32], cur[33]);
        }
        // warp reduces: one vote for "changed", the count (last generation only) by one reduction
        const bool any_changed = __any_sync(0xffffffffu, changed != 0u);
        if (j == kp - 1) cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) {
            if (cnt) atomicAdd(&s_cnt[kp - 1], (unsigned long long)cnt);
            if (any_changed) atomicOr(&s_ch[j], 1u);
        }
        if (warp & 1) {
            pair_sync(warp);                                   // with warp - 1
            if (warp < kWarps - 1) pair_sync(warp + 1);        // with warp + 1
        } else {
            if (warp < kWarps - 1) pair_sync(warp + 1);
            if (warp > 0) pair_sync(warp);
        }
        if ((lane == 0 && warp > 0) || (lane == 31 && warp < kWarps - 1)) {
            // lane 0 takes lane 30 of the warp above, lane 31 lane 1 of the warp below
            const uint32_t *row = xb + (lane == 0 ? (warp - 1) * 2 + 1 : (warp + 1) * 2) * kXchStride;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint4 v = ((const uint4 *)row)[i];
                cur[4 * i] = v.x; cur[4 * i + 1] = v.y; cur[4 * i + 2] = v.z; cur[4 * i + 3] = v.w;
            }
            const uint2 t = ((const uint2 *)row)[16];
            cur[32] = t.x;
            cur[33] = t.y;
        }
    }
    __syncthreads();   // the last exchange buffer is read before the next tile writes it
    // store the owned words of the owned rows
    if (own) {
        unsigned int *row = dst + y * tp.pitch + xw0;
        if (own_words == kOwnWords) {
            uint4 *v = (uint4 *)row;
#pragma unroll
            for (int i = 0; i < kOwnWords / 4; ++i)
                v[i] = make_uint4(cur[1 + 4 * i], cur[2 + 4 * i], cur[3 + 4 * i], cur[4 + 4 * i]);
        } else {
#pragma unroll
            for (int w = 1; w <= kOwnWords; ++w)
                if (w <= own_words) row[w - 1] = cur[w];
        }
    }
}

template <bool WRAP>
__global__ void __launch_bounds__(kThreads, 1) life_tb_kernel(const __grid_constant__ TbParams tp, LoopArgs la)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = align_up(smem_raw, 1024);
    unsigned char *stage = base;                                   // [2][kStageBytes]
    uint32_t *xch = (uint32_t *)(base + 2 * kStageBytes);          // [2][8][2][36]
    uint64_t *mbar = (uint64_t *)(xch + kXchWords);                // [2]
    unsigned long long *s_cnt = (unsigned long long *)(mbar + 2);  // [kMaxK]
    unsigned int *s_ch = (unsigned int *)(s_cnt + kMaxK);          // [kMaxK]
    __shared__ int s_ok, s_stop, s_rerun;
    __shared__ long long s_it;

    const int tid = threadIdx.x;
    Ctl *ctl = la.ctl;
    const long long it0 = ctl->iters;
    if (ctl->converged || it0 >= la.max_iters || ctl->err) return;
    if ((la.debug_flags & SLR_DEBUG_SKIP_ARRIVAL) && blockIdx.x == gridDim.x - 1) return;

    if (tid == 0) {
        tma::mbar_init(&mbar[0], 1);
        tma::mbar_init(&mbar[1], 1);
        tma::mbar_init_fence();
    }
    if (tid < kMaxK) { s_cnt[tid] = 0ull; s_ch[tid] = 0u; }
    __syncthreads();

    // ---- P: pack the caller's cells into bits[0]
    if (!pack_phase(tp, stage, mbar, &s_ok, &ctl->err)) return;
    unsigned long long bar_target = (unsigned long long)la.nblocks;
    if (!grid_barrier(ctl, bar_target, la.limit_ns)) return;

    // ---- G: passes
    const int ntiles = tp.tiles_x * tp.tiles_y;
    long long it = it0;
    int cur = 0;
    for (long long p = 0;; ++p) {
        const long long left = la.max_iters - it;
        const int kp = (int)((long long)tp.K < left ? (long long)tp.K : left);
        // A pass tracks "changed" in its last generation only.  A still state
        // stays still, so the last generation changed nothing exactly when some
        // generation of the pass did; the pass then runs again from its input
        // (untouched: the buffers alternate) with a flag per generation, into
        // the next pass's slots, to find the first.
        int exact = 0;
        int slot = (int)(p % kSlots);
        for (;;) {
            for (int t = (int)blockIdx.x; t < ntiles; t += (int)gridDim.x)
                run_tile<WRAP>(tp, t, kp, exact, tp.bits[cur], tp.bits[cur ^ 1], xch, s_cnt, s_ch);
            __syncthreads();
            if (tid < kp) {
                Slot *s = &ctl->sub[slot][tid];
                if (s_cnt[tid]) atomicAdd(&s->cnt, s_cnt[tid]);
                if (s_ch[tid]) atomicOr(&s->changed, 1u);
                s_cnt[tid] = 0ull;
                s_ch[tid] = 0u;
            }
            bar_target += (unsigned long long)la.nblocks;
            if (!grid_barrier(ctl, bar_target, la.limit_ns)) return;
            if (tid < 32) {
                if (blockIdx.x == 0 && !exact) zero_slot(&ctl->sub[(p + 2) % kSlots][tid]);
                // a generation that changed nothing is a still state, a fixed
                // point: the state (and live count) at the end of the pass equal
                // it.  Lane j reads generation j's flag; the first unchanged one wins.
                const bool unchanged = tid < kp && (exact || tid == kp - 1) &&
                                       ld_relaxed_u32(&ctl->sub[slot][tid].changed) == 0u;
                const unsigned still = __ballot_sync(0xffffffffu, unchanged);
                const int jstop = still ? __ffs(still) - 1 : -1;
                const int rerun = !exact && jstop >= 0;
                const unsigned long long cnt = ld_relaxed_u64(&ctl->sub[slot][kp - 1].cnt);
                const long long itn = jstop >= 0 ? it + jstop + 1 : it + kp;
                const int conv = jstop >= 0;
                if (tid == 0) {
                    s_rerun = rerun;
                    s_stop = !rerun && (conv || itn >= la.max_iters);
                    s_it = itn;
                    if (!rerun && (conv || itn >= la.max_iters) && blockIdx.x == 0) {
                        ctl->iters = itn;
                        ctl->value = (double)cnt;
                        ctl->count = cnt;
                        ctl->changed = !conv;
                        ctl->converged = conv;
                    }
                }
            }
            __syncthreads();
            if (!s_rerun) break;
            exact = 1;
            slot = (int)((p + 1) % kSlots);
        }
        cur ^= 1;
        it = s_it;
        if (s_stop) break;
    }

    // ---- U: unpack bits[cur] into the caller's cells
    const unsigned int *fin = tp.bits[cur];
    unsigned char *cells = (unsigned char *)la.a;
    const long long total = tp.ny * tp.nxw;
    for (long long i = (long long)blockIdx.x * kThreads + tid; i < total; i += (long long)gridDim.x * kThreads) {
        const long long y = i / tp.nxw, xw = i - y * tp.nxw;
        const uint32_t word = __ldcg(fin + y * tp.pitch + xw);
        uint4 *o = (uint4 *)(cells + y * tp.nx + 32 * xw);
        o[0] = unpack16(word & 0xFFFFu);
        o[1] = unpack16(word >> 16);
    }
}

bool make_cells_map(CUtensorMap *m, void *base, long long nx, long long ny)
{
    auto fn = tma::encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)nx};
    cuuint32_t box[2] = {(cuuint32_t)kBoxW, (cuuint32_t)kPackRows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

long long pitch_words(long long nx) { return ((nx / 32) + 3) / 4 * 4; }

}  // namespace

bool life_tb_supported(const Problem &p)
{
    if (p.nx % 32 != 0 || p.nx < 32 || p.ny < 1) return false;
    if (p.nx >= (1ll << 31) || p.ny >= (1ll << 31)) return false;
    return tma::encode_fn() != nullptr;
}

size_t life_tb_bits_bytes(long long nx, long long ny) { return (size_t)(pitch_words(nx) * ny * 4); }

// Generations per pass when the caller leaves it to the library: the largest K
// (up to kMaxK) whose tiling needs no more tiles than the CTAs resident at
// once, so every pass is one wave of tiles.
int life_tb_default_k(const Problem &p, int nblocks)
{
    const long long tx = (p.nx + kOwnCols - 1) / kOwnCols;
    for (int k = kMaxK; k >= 4; --k) {
        const long long own = kTileRows - 2 * k;
        if (tx * ((p.ny + own - 1) / own) <= nblocks) return k;
    }
    return 16;
}

// CTAs of the persistent launch (at most 2 per SM, capped by `request`).
static cudaError_t tb_grid(const Problem &p, int request, int *nblocks)
{
    auto kern = p.wrap ? life_tb_kernel<true> : life_tb_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, kSmemBytes)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    *nblocks = grid_ctas(sms, per_sm > 2 ? 2 : per_sm, request);
    return cudaSuccess;
}

int life_tb_resolve_k(const Problem &p, int grid_request)
{
    if (p.k > 1) return p.k > kMaxK ? kMaxK : p.k;
    int nblocks = 0;
    if (tb_grid(p, grid_request, &nblocks) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return life_tb_default_k(p, nblocks);
}

cudaError_t life_tb_persistent(const Problem &p, LoopArgs la, void *bits0, void *bits1, cudaStream_t st)
{
    if (!life_tb_supported(p)) return cudaErrorNotSupported;
    TbParams tp;
    memset(&tp, 0, sizeof(tp));
    if (!make_cells_map(&tp.cells, la.a, p.nx, p.ny)) return cudaErrorInvalidValue;
    tp.bits[0] = (unsigned int *)bits0;
    tp.bits[1] = (unsigned int *)bits1;
    tp.nx = p.nx;
    tp.ny = p.ny;
    tp.nxw = p.nx / 32;
    tp.pitch = pitch_words(p.nx);
    tp.wrap = p.wrap;
    auto kern = p.wrap ? life_tb_kernel<true> : life_tb_kernel<false>;
    int nblocks = 0;
    cudaError_t e = tb_grid(p, la.nblocks, &nblocks);
    if (e != cudaSuccess) return e;
    tp.K = p.k > 1 ? (p.k > kMaxK ? kMaxK : p.k) : life_tb_default_k(p, nblocks);
    tp.own_rows = kTileRows - 2 * tp.K;
    tp.tiles_x = (int)((p.nx + kOwnCols - 1) / kOwnCols);
    tp.tiles_y = (int)((p.ny + tp.own_rows - 1) / tp.own_rows);
    return launch_cooperative(kern, kThreads, kSmemBytes, 2, la, &tp, st);
}

}  // namespace slr
