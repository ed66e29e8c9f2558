// life.cu -- Game of Life (B3/S23 over the 8 Moore neighbours, the elemental
// function of Fig. 1) fused with its two reduces (live count, any cell
// changed) and looped on the device (Sec. 3.1, -d and -s variants).
//
// Fast path (row length a multiple of 16 bytes): one warp owns a 512-column
// segment of a band of rows; each lane holds 16 cells of a row as four 32-bit
// words and walks down the band.  The 8-neighbour count is done four cells at a
// time inside 32-bit words (byte lanes never exceed 9, so no carries cross
// bytes): horizontal 3-sums with funnel shifts, the left/right edge bytes from
// the neighbouring lanes by shuffle, a sliding window of three horizontal sums
// for the vertical direction.  Every cell is read once from HBM per sweep (the
// band's two halo rows come from L2) and written once: 2 bytes per cell.
//
// Generic path (any width): one thread per cell, neighbours by index.
#include "slr_internal.cuh"

namespace slr {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kLifeThreads = 512;

// Next state of four cells packed one per byte.  S is the byte-wise sum of the
// 3x3 block INCLUDING the cell itself (0..9), self the current cells (0/1).
// Alive next  <=>  S == 3  or  (self and S == 4)   (B3/S23 with the centre
// counted in S).  Byte equality via the zero-byte test: for bytes < 0x80,
// (x + 0x7F) has bit 7 set iff x != 0, with no carry into the next byte.
__device__ __forceinline__ uint32_t life_rule4(uint32_t S, uint32_t self)
{
    const uint32_t nz3 = (S ^ 0x03030303u) + 0x7F7F7F7Fu;
    const uint32_t nz4 = (S ^ 0x04040404u) + 0x7F7F7F7Fu;
    const uint32_t alive7 = (~nz3 & 0x80808080u) | (~nz4 & (self << 7));
    return alive7 >> 7;
}

struct LifeFast {
    long long nx, ny;
    int wrap;

    __device__ __forceinline__ size_t state_bytes() const { return (size_t)nx * (size_t)ny; }

    // 16 cells of row r starting at column c0 (zeros for a dead border row).
    __device__ __forceinline__ uint4 row16(const unsigned char *src, long long r, long long c0, bool active) const
    {
        if (!active) return make_uint4(0u, 0u, 0u, 0u);
        if (r < 0 || r >= ny) {
            if (!wrap) return make_uint4(0u, 0u, 0u, 0u);
            r = r < 0 ? r + ny : r - ny;
        }
        return __ldcg((const uint4 *)(src + r * nx + c0));
    }

    // One cell (row r in [-1, ny], column c in [-1, nx]) as 0/1.
    __device__ __forceinline__ uint32_t cell(const unsigned char *src, long long r, long long c) const
    {
        if (r < 0 || r >= ny || c < 0 || c >= nx) {
            if (!wrap) return 0u;
            r = r < 0 ? r + ny : (r >= ny ? r - ny : r);
            c = c < 0 ? c + nx : (c >= nx ? c - nx : c);
        }
        return (uint32_t)__ldcg(src + r * nx + c);
    }

    // Byte-wise horizontal 3-sums of a 16-cell chunk.  Every lane of the warp
    // must call this (shuffles); v of inactive lanes is zero.
    __device__ __forceinline__ void hsum(const unsigned char *src, long long r, long long c0, int lane,
                                         bool active, bool right_in_warp, const uint4 &v, uint32_t h[4]) const
    {
        uint32_t prevw = __shfl_up_sync(kFull, v.w, 1);    // top byte = column c0 - 1
        uint32_t nextw = __shfl_down_sync(kFull, v.x, 1);  // low byte = column c0 + 16
        if (active) {
            if (lane == 0) prevw = cell(src, r, c0 - 1) << 24;
            if (!right_in_warp) nextw = cell(src, r, c0 + 16);
        }
        h[0] = __funnelshift_l(prevw, v.x, 8) + v.x + __funnelshift_r(v.x, v.y, 8);
        h[1] = __funnelshift_l(v.x, v.y, 8) + v.y + __funnelshift_r(v.y, v.z, 8);
        h[2] = __funnelshift_l(v.y, v.z, 8) + v.z + __funnelshift_r(v.z, v.w, 8);
        h[3] = __funnelshift_l(v.z, v.w, 8) + v.w + __funnelshift_r(v.w, nextw, 8);
    }

    template <bool REDUCE>
    __device__ __forceinline__ void sweep(const void *src_v, void *dst_v, Slot *slot) const
    {
        const unsigned char *src = (const unsigned char *)src_v;
        unsigned char *dst = (unsigned char *)dst_v;
        const int lane = threadIdx.x & 31;
        const long long wpb = blockDim.x >> 5;
        const long long warps = (long long)gridDim.x * wpb;
        const long long gw = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
        // units: (512-column segment, balanced band of rows)
        const long long C = (nx + 511) / 512;
        long long P = warps / C;
        if (P < 1) P = 1;
        const long long U = C * P;
        uint32_t changed = 0u;
        unsigned long long cnt = 0ull;
        for (long long u = gw; u < U; u += warps) {
            const long long seg = u % C, part = u / C;
            const long long r0 = part * ny / P, r1 = (part + 1) * ny / P;
            if (r0 >= r1) continue;
            const long long c0 = seg * 512 + (long long)lane * 16;
            const bool active = c0 < nx;
            const bool rin = lane < 31 && c0 + 16 < nx;
            uint4 vc = row16(src, r0, c0, active);
            uint32_t hp[4], hc[4];
            {
                const uint4 vp = row16(src, r0 - 1, c0, active);
                hsum(src, r0 - 1, c0, lane, active, rin, vp, hp);
                hsum(src, r0, c0, lane, active, rin, vc, hc);
            }
            for (long long r = r0; r < r1; r += 4) {
                uint4 nv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    nv[q] = (r + 1 + q <= r1) ? row16(src, r + 1 + q, c0, active) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (r + q < r1) {
                        uint32_t hn[4];
                        hsum(src, r + 1 + q, c0, lane, active, rin, nv[q], hn);
                        uint4 o;
                        o.x = life_rule4(hp[0] + hc[0] + hn[0], vc.x);
                        o.y = life_rule4(hp[1] + hc[1] + hn[1], vc.y);
                        o.z = life_rule4(hp[2] + hc[2] + hn[2], vc.z);
                        o.w = life_rule4(hp[3] + hc[3] + hn[3], vc.w);
                        if (active) {
                            *(uint4 *)(dst + (r + q) * nx + c0) = o;
                            if (REDUCE) {
                                changed |= (o.x ^ vc.x) | (o.y ^ vc.y) | (o.z ^ vc.z) | (o.w ^ vc.w);
                                cnt += (unsigned long long)(__popc(o.x) + __popc(o.y) + __popc(o.z) + __popc(o.w));
                            }
                        }
#pragma unroll
                        for (int t = 0; t < 4; ++t) { hp[t] = hc[t]; hc[t] = hn[t]; }
                        vc = nv[q];
                    }
                }
            }
        }
        if (REDUCE) block_to_slot(slot, 0ull, 0ull, cnt, changed ? 1u : 0u);
    }
};

struct LifeGeneric {
    long long nx, ny;
    int wrap;

    __device__ __forceinline__ size_t state_bytes() const { return (size_t)nx * (size_t)ny; }

    template <bool REDUCE>
    __device__ __forceinline__ void sweep(const void *src_v, void *dst_v, Slot *slot) const
    {
        const unsigned char *src = (const unsigned char *)src_v;
        unsigned char *dst = (unsigned char *)dst_v;
        uint32_t changed = 0u;
        unsigned long long cnt = 0ull;
        for (long long i = blockIdx.x; i < ny; i += gridDim.x) {
            for (long long j = threadIdx.x; j < nx; j += blockDim.x) {
                int n = 0;
                for (int di = -1; di <= 1; ++di)
                    for (int dj = -1; dj <= 1; ++dj) {
                        if (di == 0 && dj == 0) continue;
                        long long y = i + di, x = j + dj;
                        if (y < 0 || y >= ny || x < 0 || x >= nx) {
                            if (!wrap) continue;
                            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
                            x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
                        }
                        n += __ldcg(src + y * nx + x) != 0;
                    }
                const int self = __ldcg(src + i * nx + j) != 0;
                const int next = (n == 3) || (self && n == 2);
                dst[i * nx + j] = (unsigned char)next;
                if (REDUCE) { changed |= (uint32_t)(next != self); cnt += (unsigned long long)next; }
            }
        }
        if (REDUCE) block_to_slot(slot, 0ull, 0ull, cnt, changed);
    }
};

template <class Op>
__global__ void __launch_bounds__(kLifeThreads, 1) life_persistent_kernel(Op op, LoopArgs la)
{
    persistent_loop_body(op, la);
}

template <class Op>
__global__ void __launch_bounds__(kLifeThreads, 1) life_sweep_kernel(Op op, const void *src, void *dst)
{
    op.template sweep<false>(src, dst, nullptr);
}

// Any non-zero byte becomes 1 (16 bytes per thread and step where aligned).
__global__ void life_normalize_kernel(unsigned char *u, size_t n)
{
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nthr = (size_t)gridDim.x * blockDim.x;
    const size_t n16 = ((uintptr_t)u & 15u) ? 0 : n / 16;
    uint4 *u4 = (uint4 *)u;
    for (size_t i = tid; i < n16; i += nthr) {
        uint4 v = u4[i];
        uint32_t *w = &v.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t x = w[k];
            x |= x >> 4;
            x |= x >> 2;
            x |= x >> 1;
            w[k] = x & 0x01010101u;
        }
        u4[i] = v;
    }
    for (size_t i = n16 * 16 + tid; i < n; i += nthr) u[i] = u[i] != 0;
}

bool fast_ok(const Problem &p) { return p.nx % 16 == 0; }

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

cudaError_t life_persistent(const Problem &p, LoopArgs la, cudaStream_t st)
{
    if (fast_ok(p)) {
        LifeFast op{p.nx, p.ny, p.wrap};
        return launch_cooperative(life_persistent_kernel<LifeFast>, kLifeThreads, 0, 1, la, &op, st);
    }
    LifeGeneric op{p.nx, p.ny, p.wrap};
    return launch_cooperative(life_persistent_kernel<LifeGeneric>, kLifeThreads, 0, 1, la, &op, st);
}

cudaError_t life_sweep(const Problem &p, const void *src, void *dst, cudaStream_t st)
{
    const int grid = sm_count();
    if (fast_ok(p)) {
        LifeFast op{p.nx, p.ny, p.wrap};
        life_sweep_kernel<LifeFast><<<grid, kLifeThreads, 0, st>>>(op, src, dst);
    } else {
        LifeGeneric op{p.nx, p.ny, p.wrap};
        life_sweep_kernel<LifeGeneric><<<grid, kLifeThreads, 0, st>>>(op, src, dst);
    }
    return cudaGetLastError();
}

cudaError_t life_normalize(const Problem &p, void *u, cudaStream_t st)
{
    life_normalize_kernel<<<sm_count() * 4, 256, 0, st>>>((unsigned char *)u, p.state_bytes);
    return cudaGetLastError();
}

}  // namespace slr
