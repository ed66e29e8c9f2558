// life_tb.cu -- temporal-blocked Game of Life: K generations per HBM pass.
//
// The loop-of-stencil-reduce of Sec. 3.1 with the Fig. 1 elemental function
// (B3/S23) on a uint8 grid, restructured for GB300: every pass reads each cell
// from HBM once, runs up to K generations on chip, and writes each cell once,
// so HBM traffic per generation is 2/K bytes per cell instead of 2.
//
// Tile: 256 rows x 1088 columns loaded (1024 owned columns plus one 32-cell
// word of halo on each side; 224 owned rows plus 16 halo rows above and
// below), so up to 16 generations stay exact inside the owned region (each
// generation invalidates one more cell ring from the outside).
//
//  1. Load: the tile arrives in 8 chunks of 32 rows, each chunk as ten TMA
//     boxes (cp.async.bulk.tensor.2d) into a double-buffered staging area:
//     eight 128-byte-wide boxes with the 128B swizzle (so that the packing
//     reads below are bank-conflict free) and two 32-byte halo boxes.  An
//     out-of-range box reads zeros (the dead border for free); on the torus
//     every box is placed at its wrapped coordinate (tiles are laid out so no
//     box straddles the grid edge).  Threads pack the bytes into a bit-tile in
//     shared memory, 32 cells per 32-bit word, bit b = column b.
//  2. Evolve: thread t takes tile row t into 34 registers.  Vertical
//     neighbours come from the adjacent lanes by shuffle (and from the adjacent
//     warps through a small shared exchange row, one barrier per generation);
//     horizontal neighbours by funnel shifts across the word boundary.  The
//     8-neighbour count is a bit-sliced adder tree of 18 logic operations per
//     32 cells.  The two reduces of the generation (live count, any cell
//     changed) are taken over the owned region only, per generation.
//  3. Store: rows go back through the bit-tile, are expanded to bytes and
//     written with coalesced 16-byte stores.
//
// After each pass a bounded grid barrier publishes the per-generation
// reduces; every CTA takes the same decision: stop at the first generation
// that changed nothing (a still state is a fixed point, so the stored state
// after the pass equals that generation) or at the iteration cap (the last
// pass runs only the generations left).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "slr_internal.cuh"

namespace slr {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTileRows = 256;
constexpr int kHaloRows = 16;
constexpr int kOwnRows = kTileRows - 2 * kHaloRows;  // 224
constexpr int kWords = 34;                            // 1 halo + 32 owned + 1 halo
constexpr int kOwnCols = 1024;
constexpr int kBitStride = 35;                        // odd: conflict-free row loads
constexpr int kChunkRows = 32;
constexpr int kChunks = kTileRows / kChunkRows;       // 8
constexpr int kMidBoxW = 128;                         // bytes (= cells) per swizzled box row
constexpr int kMidBoxes = kOwnCols / kMidBoxW;        // 8
constexpr int kMidBoxBytes = kMidBoxW * kChunkRows;   // 4096
constexpr int kHaloBoxW = 32;
constexpr int kHaloBoxBytes = kHaloBoxW * kChunkRows; // 1024
constexpr int kStageBytes = kMidBoxes * kMidBoxBytes + 2 * kHaloBoxBytes;  // 34816 = 34 KiB
constexpr int kBitsBytes = kTileRows * kBitStride * 4;                      // 35840
constexpr int kXchWords = 2 * kWarps * 2 * kWords;    // [parity][warp][top,bottom][word]
constexpr size_t kSmemBytes = 1024 /*alignment slack*/ + 2 * kStageBytes + kBitsBytes + kXchWords * 4 +
                              kWords * 4 /*zero row*/ + 2 * 8 /*mbarriers*/ + kMaxK * 8 + kMaxK * 4;
static_assert(kStageBytes % 1024 == 0, "staging buffers must keep 1024-byte alignment for the swizzle");

struct TbParams {
    CUtensorMap mid[2];   // [0] reads buffer A (the caller's u), [1] reads buffer B
    CUtensorMap halo[2];
    long long nx, ny;
    int wrap, K, tiles_x, tiles_y;
};

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ---- cell packing -----------------------------------------------------------
// Four 0/1 bytes -> 4 bits (byte i -> bit i): the products land on distinct bit
// positions 24..27, so the multiply adds no carries.
__device__ __forceinline__ uint32_t pack4(uint32_t w) { return (w * 0x01020408u) >> 24; }

__device__ __forceinline__ uint32_t pack16(const uint4 v)
{
    return pack4(v.x) | (pack4(v.y) << 4) | (pack4(v.z) << 8) | (pack4(v.w) << 12);
}

// 4 bits -> four 0/1 bytes (bit i -> byte i): copies of the nibble at shifts
// 0, 7, 14, 21 do not overlap, so bit i lands alone at bit 8i.
__device__ __forceinline__ uint32_t unpack4(uint32_t n) { return (n * 0x00204081u) & 0x01010101u; }

__device__ __forceinline__ uint4 unpack16(uint32_t h)
{
    return make_uint4(unpack4(h & 15u), unpack4((h >> 4) & 15u), unpack4((h >> 8) & 15u), unpack4((h >> 12) & 15u));
}

// ---- the B3/S23 step on 32 cells --------------------------------------------
// U*, C*, D*: the row above, the row itself, the row below; m/c/n: the word to
// the left, the word, the word to the right.  Bit b of a word is column b, so
// the left neighbour of bit b is bit b-1 (or bit 31 of the word to the left).
__device__ __forceinline__ uint32_t life_word(uint32_t Um, uint32_t Uc, uint32_t Un, uint32_t Cm, uint32_t Cc,
                                              uint32_t Cn, uint32_t Dm, uint32_t Dc, uint32_t Dn)
{
    const uint32_t UL = __funnelshift_l(Um, Uc, 1), UR = __funnelshift_r(Uc, Un, 1);
    const uint32_t CL = __funnelshift_l(Cm, Cc, 1), CR = __funnelshift_r(Cc, Cn, 1);
    const uint32_t DL = __funnelshift_l(Dm, Dc, 1), DR = __funnelshift_r(Dc, Dn, 1);
    // 2-bit sums: above (a1 a0) = UL+Uc+UR, below (b1 b0), middle (m1 m0) = CL+CR
    const uint32_t a0 = UL ^ Uc ^ UR, a1 = (UL & Uc) | (UL & UR) | (Uc & UR);
    const uint32_t b0 = DL ^ Dc ^ DR, b1 = (DL & Dc) | (DL & DR) | (Dc & DR);
    const uint32_t m0 = CL ^ CR, m1 = CL & CR;
    // n = bit0 + 2*H with H = c0 + a1 + m1 + b1; alive next <=> H == 1 and (bit0 or self)
    const uint32_t bit0 = a0 ^ m0 ^ b0, c0 = (a0 & m0) | (a0 & b0) | (m0 & b0);
    const uint32_t x = a1 ^ m1 ^ b1, y = (a1 & m1) | (a1 & b1) | (m1 & b1);
    const uint32_t one = (x ^ c0) & ~y;  // exactly one of {a1, m1, b1, c0}
    return one & (Cc | bit0);
}

// ---- tile geometry ----------------------------------------------------------
struct Tile {
    long long x0;        // first owned column
    long long frame0;    // frame row of tile row 0 (owned frame rows: [frame0 + 16, frame0 + 240))
    long long real0;     // real (unwrapped) row of tile row 0
};

__device__ __forceinline__ Tile tile_of(const TbParams &tp, int t)
{
    Tile g;
    const int tx = t % tp.tiles_x, ty = t / tp.tiles_x;
    g.x0 = (long long)tx * kOwnCols;
    g.frame0 = (long long)ty * kOwnRows - kHaloRows;
    // on the torus the frame is rotated by 16 rows so that every 32-row chunk
    // starts on a multiple of 32 and never straddles the grid edge
    g.real0 = g.frame0 - (tp.wrap ? kHaloRows : 0);
    return g;
}

__device__ __forceinline__ long long wrap_mod(long long v, long long n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Box b of a chunk (b < 8: owned columns, 8: left halo, 9: right halo): its
// column, width and whether any of it lies inside the grid.  On the torus every
// box is placed at its wrapped coordinate and is always inside; with the dead
// border a box wholly outside the grid is not loaded at all and reads as zeros
// (a box partly outside is loaded and the hardware fills the outside with
// zeros).
struct Box {
    long long x;
    int w;
    bool in;
};

__device__ __forceinline__ long long chunk_row(const TbParams &tp, const Tile &g, int c)
{
    long long y = g.real0 + (long long)c * kChunkRows;
    return tp.wrap ? wrap_mod(y, tp.ny) : y;
}

__device__ __forceinline__ Box box_of(const TbParams &tp, const Tile &g, long long y, int b)
{
    Box bx;
    if (b < kMidBoxes) { bx.x = g.x0 + (long long)b * kMidBoxW; bx.w = kMidBoxW; }
    else { bx.x = b == kMidBoxes ? g.x0 - kHaloBoxW : g.x0 + kOwnCols; bx.w = kHaloBoxW; }
    if (tp.wrap) {
        bx.x = wrap_mod(bx.x, tp.nx);
        bx.in = true;
    } else {
        bx.in = bx.x < tp.nx && bx.x + bx.w > 0 && y < tp.ny && y + kChunkRows > 0;
    }
    return bx;
}

// Thread 0: enqueue the in-grid boxes of chunk c of tile g into a staging buffer.
__device__ __forceinline__ void issue_chunk(const TbParams &tp, int srcbuf, const Tile &g, int c,
                                           unsigned char *stage, uint64_t *bar)
{
    const long long y = chunk_row(tp, g, c);
    uint32_t bytes = 0;
    Box bx[kMidBoxes + 2];
#pragma unroll
    for (int b = 0; b < kMidBoxes + 2; ++b) {
        bx[b] = box_of(tp, g, y, b);
        if (bx[b].in) bytes += (uint32_t)(bx[b].w * kChunkRows);
    }
    mbar_expect_tx(bar, bytes);
#pragma unroll
    for (int b = 0; b < kMidBoxes; ++b)
        if (bx[b].in) tma_load_2d(stage + b * kMidBoxBytes, &tp.mid[srcbuf], (int)bx[b].x, (int)y, bar);
#pragma unroll
    for (int s = 0; s < 2; ++s)
        if (bx[kMidBoxes + s].in)
            tma_load_2d(stage + kMidBoxes * kMidBoxBytes + s * kHaloBoxBytes, &tp.halo[srcbuf],
                        (int)bx[kMidBoxes + s].x, (int)y, bar);
}

// WRAP: torus (every tile cell is a real, wrapped cell).  !WRAP: dead border;
// cells of the tile that lie outside the grid are cleared after every
// generation, because the border stays dead at every step.
template <bool WRAP>
__global__ void __launch_bounds__(kThreads, 2) life_tb_kernel(const __grid_constant__ TbParams tp, LoopArgs la)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stage = base;                                   // [2][kStageBytes]
    uint32_t *bits = (uint32_t *)(base + 2 * kStageBytes);         // [256][35]
    uint32_t *xch = bits + kTileRows * kBitStride;                 // [2][8][2][34]
    uint32_t *zrow = xch + kXchWords;                              // [34] zeros
    uint64_t *mbar = (uint64_t *)(zrow + kWords);                  // [2] (8-byte aligned: offsets are even words)
    unsigned long long *s_cnt = (unsigned long long *)(mbar + 2);  // [kMaxK]
    unsigned int *s_ch = (unsigned int *)(s_cnt + kMaxK);          // [kMaxK]
    __shared__ int s_ok, s_stop, s_conv;
    __shared__ long long s_it;
    __shared__ double s_val;
    __shared__ unsigned long long s_count;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Ctl *ctl = la.ctl;
    const long long it0 = ctl->iters;
    if (ctl->converged || it0 >= la.max_iters || ctl->err) return;
    if ((la.debug_flags & SLR_DEBUG_SKIP_ARRIVAL) && blockIdx.x == gridDim.x - 1) return;

    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (tid < kWords) zrow[tid] = 0u;
    if (tid < kMaxK) { s_cnt[tid] = 0ull; s_ch[tid] = 0u; }
    __syncthreads();

    const int ntiles = tp.tiles_x * tp.tiles_y;
    const int mine = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int nchunks = mine * kChunks;
    // chunks consumed so far by this CTA; chunk q uses staging buffer q & 1 and
    // completes phase (q >> 1) & 1 of that buffer's mbarrier
    uint32_t q = 0;
    long long it = it0;

    for (long long p = 0;; ++p) {
        const int srcbuf = (int)(p & 1);                         // pass p reads A (p even) or B
        unsigned char *dst = (unsigned char *)(srcbuf ? la.a : la.b);
        const long long left = la.max_iters - it;
        const int kp = (int)((long long)tp.K < left ? (long long)tp.K : left);

        if (tid == 0) {
            // after the grid barrier: make other CTAs' generic stores of the
            // previous pass visible to this CTA's TMA (async proxy) reads
            fence_proxy_async_global();
            for (int ci = 0; ci < 2 && ci < nchunks; ++ci)
                issue_chunk(tp, srcbuf, tile_of(tp, (int)blockIdx.x + (ci / kChunks) * (int)gridDim.x),
                            ci % kChunks, stage + ((q + ci) & 1u) * kStageBytes, &mbar[(q + ci) & 1u]);
        }
        for (int ti = 0; ti < mine; ++ti) {
            const Tile g = tile_of(tp, (int)blockIdx.x + ti * (int)gridDim.x);
            // ---- 1. load: wait for each chunk, pack it into the bit-tile -----------
            for (int c = 0; c < kChunks; ++c, ++q) {
                const uint32_t sb = q & 1u;
                if (tid == 0) {
                    int ok = 1;
                    long long t0 = 0;
                    unsigned spins = 0;
                    while (!mbar_try_wait(&mbar[sb], (q >> 1) & 1u)) {
                        if ((++spins & 255u) == 0u) {
                            const long long t = global_timer_ns();
                            if (t0 == 0) t0 = t;
                            else if (t - t0 > la.limit_ns) { atomicOr(&ctl->err, DEV_ERR_TIMEOUT); ok = 0; break; }
                        }
                    }
                    s_ok = ok;
                }
                __syncthreads();
                if (!s_ok) return;
                const unsigned char *sbase = stage + sb * kStageBytes;
                uint32_t *brow = bits + c * kChunkRows * kBitStride;
                const long long ychunk = chunk_row(tp, g, c);
#pragma unroll
                for (int i = 0; i < (kChunkRows * 64) / kThreads; ++i) {   // 32 rows x 64 groups of 16 cells
                    const int item = tid + i * kThreads;
                    const int rr = item >> 6, gidx = item & 63;
                    const int box = gidx >> 3, qq = gidx & 7;
                    uint32_t packed = 0u;
                    if (box_of(tp, g, ychunk, box).in)
                        packed = pack16(*(const uint4 *)(sbase + box * kMidBoxBytes + rr * kMidBoxW +
                                                         ((qq ^ (rr & 7)) << 4)));
                    ((unsigned short *)(brow + rr * kBitStride + 1 + (gidx >> 1)))[gidx & 1] = (unsigned short)packed;
                }
                if (tid < kChunkRows * 4) {                                // halo words 0 and 33
                    const int rr = tid >> 2, side = (tid >> 1) & 1, half = tid & 1;
                    uint32_t packed = 0u;
                    if (box_of(tp, g, ychunk, kMidBoxes + side).in)
                        packed = pack16(*(const uint4 *)(sbase + kMidBoxes * kMidBoxBytes + side * kHaloBoxBytes +
                                                         rr * kHaloBoxW + half * 16));
                    ((unsigned short *)(brow + rr * kBitStride + (side ? kWords - 1 : 0)))[half] =
                        (unsigned short)packed;
                }
                __syncthreads();                                           // staging buffer sb is free again
                const int nxt = ti * kChunks + c + 2;
                if (tid == 0 && nxt < nchunks)
                    issue_chunk(tp, srcbuf, tile_of(tp, (int)blockIdx.x + (nxt / kChunks) * (int)gridDim.x),
                                nxt % kChunks, stage + sb * kStageBytes, &mbar[sb]);
            }
            // ---- 2. evolve kp generations in registers ------------------------------
            uint32_t cur[kWords];
#pragma unroll
            for (int w = 0; w < kWords; ++w) cur[w] = bits[tid * kBitStride + w];
            const long long frame = g.frame0 + tid;
            const bool own_row = tid >= kHaloRows && tid < kHaloRows + kOwnRows && frame < tp.ny;
            const long long ocols = tp.nx - g.x0;
            const int own_words = ocols >= kOwnCols ? 32 : (int)(ocols / 32);
            // dead border: words [wlo, whi] of this row are inside the grid
            const long long yreal = g.real0 + tid;
            const bool row_in = WRAP || (yreal >= 0 && yreal < tp.ny);
            const int wlo = (WRAP || g.x0 > 0) ? 0 : 1;
            // word w holds columns x0 - 32 + 32w .. x0 + 32w - 1
            const long long wmax = (tp.nx - g.x0) / 32;
            const int whi = WRAP ? kWords - 1 : (int)(wmax < kWords - 1 ? wmax : kWords - 1);
            for (int j = 0; j < kp; ++j) {
                uint32_t *mine_x = xch + ((j & 1) * kWarps + warp) * 2 * kWords;
                if (lane == 0) {
#pragma unroll
                    for (int w = 0; w < kWords; ++w) mine_x[w] = cur[w];
                }
                if (lane == 31) {
#pragma unroll
                    for (int w = 0; w < kWords; ++w) mine_x[kWords + w] = cur[w];
                }
                __syncthreads();
                const uint32_t *upr = warp > 0 ? xch + (((j & 1) * kWarps + warp - 1) * 2 + 1) * kWords : zrow;
                const uint32_t *dnr = warp < kWarps - 1 ? xch + (((j & 1) * kWarps + warp + 1) * 2) * kWords : zrow;
                uint32_t Um = 0u, Cm = 0u, Dm = 0u;
                uint32_t Cc = cur[0];
                uint32_t Uc = __shfl_up_sync(0xffffffffu, Cc, 1), Dc = __shfl_down_sync(0xffffffffu, Cc, 1);
                if (lane == 0) Uc = upr[0];
                if (lane == 31) Dc = dnr[0];
                uint32_t changed = 0u, cnt = 0u;
#pragma unroll
                for (int w = 0; w < kWords; ++w) {
                    uint32_t Un = 0u, Cn = 0u, Dn = 0u;
                    if (w + 1 < kWords) {
                        Cn = cur[w + 1];
                        Un = __shfl_up_sync(0xffffffffu, Cn, 1);
                        Dn = __shfl_down_sync(0xffffffffu, Cn, 1);
                        if (lane == 0) Un = upr[w + 1];
                        if (lane == 31) Dn = dnr[w + 1];
                    }
                    uint32_t nw = life_word(Um, Uc, Un, Cm, Cc, Cn, Dm, Dc, Dn);
                    if (!WRAP && !(row_in && w >= wlo && w <= whi)) nw = 0u;
                    if (w >= 1 && w <= 32 && own_row && w <= own_words) {
                        changed |= nw ^ Cc;
                        cnt += (uint32_t)__popc(nw);
                    }
                    cur[w] = nw;
                    Um = Uc; Uc = Un; Cm = Cc; Cc = Cn; Dm = Dc; Dc = Dn;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                    changed |= __shfl_xor_sync(0xffffffffu, changed, o);
                }
                if (lane == 0) {
                    if (cnt) atomicAdd(&s_cnt[j], (unsigned long long)cnt);
                    if (changed) atomicOr(&s_ch[j], 1u);
                }
            }
            // ---- 3. store the owned region ----------------------------------------
            __syncthreads();
#pragma unroll
            for (int w = 1; w <= 32; ++w) bits[tid * kBitStride + w] = cur[w];
            __syncthreads();
            for (int i = 0; i < (kOwnRows * 64) / kThreads; ++i) {        // 224 rows x 64 groups
                const int item = tid + i * kThreads;
                const int rr = kHaloRows + (item >> 6), gidx = item & 63;
                const long long col = g.x0 + 16ll * gidx;
                if (col >= tp.nx || g.frame0 + rr >= tp.ny) continue;
                long long y = g.real0 + rr;
                if (tp.wrap) y = wrap_mod(y, tp.ny);
                const uint32_t word = bits[rr * kBitStride + 1 + (gidx >> 1)];
                *(uint4 *)(dst + y * tp.nx + col) = unpack16((gidx & 1) ? (word >> 16) : (word & 0xFFFFu));
            }
        }
        // ---- publish this CTA's per-generation reduces, then the grid barrier -------
        __syncthreads();
        if (tid < kp) {
            Slot *s = &ctl->sub[p % kSlots][tid];
            if (s_cnt[tid]) atomicAdd(&s->cnt, s_cnt[tid]);
            if (s_ch[tid]) atomicOr(&s->changed, 1u);
            s_cnt[tid] = 0ull;
            s_ch[tid] = 0u;
        }
        fence_proxy_async_global();
        if (!grid_barrier(ctl, (unsigned long long)(p + 1) * (unsigned long long)la.nblocks, la.limit_ns)) return;
        if (tid == 0) {
            if (blockIdx.x == 0)
                for (int j = 0; j < kMaxK; ++j) zero_slot(&ctl->sub[(p + 2) % kSlots][j]);
            int jstop = -1;
            Slot sj = {0ull, 0ull, 0ull, 0u, 0u};
            for (int j = 0; j < kp; ++j) {
                sj = read_slot(&ctl->sub[p % kSlots][j]);
                if (!sj.changed) { jstop = j; break; }
            }
            const long long itn = jstop >= 0 ? it + jstop + 1 : it + kp;
            const int conv = jstop >= 0;
            s_stop = conv || itn >= la.max_iters;
            s_it = itn;
            s_conv = conv;
            s_val = (double)sj.cnt;
            s_count = sj.cnt;
            if (s_stop && blockIdx.x == 0) {
                ctl->iters = itn;
                ctl->value = (double)sj.cnt;
                ctl->count = sj.cnt;
                ctl->changed = !conv;
                ctl->converged = conv;
            }
        }
        __syncthreads();
        it = s_it;
        if (s_stop) {
            if ((p & 1) == 0) grid_copy(la.b, la.a, (size_t)tp.nx * (size_t)tp.ny);
            return;
        }
    }
}


PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2D uint8 tensor map over an nx x ny row-major grid with the given box.
bool make_map(CUtensorMap *m, void *base, long long nx, long long ny, uint32_t box_w, uint32_t box_h,
              CUtensorMapSwizzle swz)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)nx};
    cuuint32_t box[2] = {box_w, box_h};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool life_tb_supported(const Problem &p)
{
    if (p.nx % 32 != 0 || p.nx < 32 || p.ny < 1) return false;
    if (p.wrap && (p.nx % kMidBoxW != 0 || p.ny % kChunkRows != 0)) return false;
    if (p.nx >= (1ll << 31) || p.ny >= (1ll << 31)) return false;
    return encode_fn() != nullptr;
}

int life_tb_default_k(const Problem &) { return 16; }

cudaError_t life_tb_persistent(const Problem &p, LoopArgs la, cudaStream_t st)
{
    if (!life_tb_supported(p)) return cudaErrorNotSupported;
    TbParams tp;
    memset(&tp, 0, sizeof(tp));
    void *bufs[2] = {la.a, la.b};
    for (int i = 0; i < 2; ++i) {
        if (!make_map(&tp.mid[i], bufs[i], p.nx, p.ny, kMidBoxW, kChunkRows, CU_TENSOR_MAP_SWIZZLE_128B) ||
            !make_map(&tp.halo[i], bufs[i], p.nx, p.ny, kHaloBoxW, kChunkRows, CU_TENSOR_MAP_SWIZZLE_NONE))
            return cudaErrorInvalidValue;
    }
    tp.nx = p.nx;
    tp.ny = p.ny;
    tp.wrap = p.wrap;
    tp.K = p.k > 0 ? (p.k > kHaloRows ? kHaloRows : p.k) : life_tb_default_k(p);
    tp.tiles_x = (int)((p.nx + kOwnCols - 1) / kOwnCols);
    tp.tiles_y = (int)((p.ny + kOwnRows - 1) / kOwnRows);
    auto kern = tp.wrap ? life_tb_kernel<true> : life_tb_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    return launch_cooperative(kern, kThreads, kSmemBytes, 2, la, &tp, st);
}

}  // namespace slr
