// restore.cu -- restoration phase of the two-phase denoiser (Sec. 4.3): a
// 2D stencil that replaces every noisy pixel by the minimiser of an
// edge-preserving function of its neighbourhood, iterated until the average
// absolute change over the noisy pixels falls below a threshold.
//
// Update (binary32, Jacobi: old values on both sides), for masked pixels only,
// neighbours in row-major order (dy = -1..1, dx = -1..1, centre skipped,
// out-of-range neighbours left out):
//     t = u - u_j;  w_j = 1 / sqrt(alpha + t*t);  num += w_j*u_j;  den += w_j
//     u' = num / den
// Unmasked pixels are copied.  Reduce: every |u' - u| of a masked pixel is
// truncated to a multiple of 2^-24 and summed as a 64-bit integer (exact,
// order-free); the mean is sum * 2^-24 / #masked.
//
// EXACT math: IEEE-rounded sqrt and divisions, no contraction (bit-identical
// to a sequential evaluation).  FAST math: the weight is the hardware
// reciprocal square root and products fuse into FMAs.
//
// Two sweep implementations: RestoreTma (rows a multiple of 16 bytes) streams
// 32 x 64 tiles through a ring of shared-memory stages, each tile arriving as
// two TMA boxes (state with a 1-pixel halo, mask); every warp lists the noisy
// pixels of its four rows with ballots, so the weight arithmetic runs on full
// warps, and the last warp done with a stage refills it.  RestoreOp is the
// plain per-pixel form for other widths and for the host-driven loop.  EXACT
// weights come from crmath.cuh (Markstein-corrected estimates, equal to the
// IEEE square root and reciprocal).
#include <string.h>

#include "crmath.cuh"
#include "restore_math.cuh"
#include "slr_internal.cuh"
#include "tma.cuh"

namespace slr {
namespace {

constexpr int kRThreads = 1024;

template <bool FAST>
struct RestoreOp {
    long long nx, ny;
    float alpha;
    const unsigned char *mask;

    __device__ __forceinline__ size_t state_bytes() const { return (size_t)nx * ny * sizeof(float); }
    __device__ __forceinline__ void prologue() const {}

    template <bool REDUCE>
    __device__ __forceinline__ void sweep(const void *src_v, void *dst_v, Slot *slot) const
    {
        const float *u = (const float *)src_v;
        float *v = (float *)dst_v;
        const long long chunks = (nx + blockDim.x - 1) / blockDim.x;
        const long long units = ny * chunks;
        unsigned long long sum = 0ull, cnt = 0ull;
        for (long long un = blockIdx.x; un < units; un += gridDim.x) {
            const long long i = un / chunks;
            const long long j = (un - i * chunks) * blockDim.x + threadIdx.x;
            if (j >= nx) continue;
            const long long c = i * nx + j;
            const float uc = __ldcg(u + c);
            if (!__ldg(mask + c)) { v[c] = uc; continue; }
            float num = 0.0f, den = 0.0f;
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
#pragma unroll
                for (int dj = -1; dj <= 1; ++dj) {
                    if (di == 0 && dj == 0) continue;
                    const long long y = i + di, x = j + dj;
                    if (y < 0 || y >= ny || x < 0 || x >= nx) continue;
                    const float uj = __ldcg(u + y * nx + x);
                    if (FAST) {
                        const float t = uc - uj;
                        const float w = rsqrtf(fmaf(t, t, alpha));
                        num = fmaf(w, uj, num);
                        den += w;
                    } else {
                        const float t = __fsub_rn(uc, uj);
                        const float w = inv_sqrt_rn2(__fadd_rn(alpha, __fmul_rn(t, t)));
                        num = __fadd_rn(num, __fmul_rn(w, uj));
                        den = __fadd_rn(den, w);
                    }
                }
            }
            const float nv = den > 0.0f ? __fdiv_rn(num, den) : uc;
            v[c] = nv;
            if (REDUCE) {
                sum += fixed_2m24(__fsub_rn(nv, uc));
                cnt += 1ull;
            }
        }
        if (REDUCE) block_to_slot(slot, 0ull, sum, cnt, sum != 0ull);
    }
};


// ---- TMA-tiled sweep -----------------------------------------------------------
constexpr int kTH = 32, kTW = 64;                 // tile of pixels
constexpr int kUBoxW = kTW + 8;                   // floats from x0 - 4 (16-byte aligned start)
constexpr int kMBoxW = kTW + 32;                  // mask bytes from x0 - 16
constexpr int kBoxH = kTH + 2;                    // rows y0 - 1 .. y0 + 32
// every TMA destination in shared memory must be 128-byte aligned
constexpr int kUBytes = (kUBoxW * kBoxH * 4 + 127) / 128 * 128;   // 9792 -> 9856
constexpr int kMBytes = (kMBoxW * kBoxH + 127) / 128 * 128;       // 3264 -> 3328
constexpr int kStage = kUBytes + kMBytes;                         // 13184
constexpr uint32_t kTxBytes = kUBoxW * kBoxH * 4 + kMBoxW * kBoxH; // bytes the two boxes deliver
constexpr int kTThreads = 256;                    // 8 warps x 4 tile rows
constexpr int kNS = 3;                            // stages in the ring
constexpr size_t kTSmem = 128 + (size_t)kNS * kStage + kNS * 8 + kNS * 4 + 16;   // stages, mbarriers, counts, counter
static_assert(kStage % 128 == 0 && kUBytes % 128 == 0, "TMA destinations must be 128-byte aligned");

// Each warp owns four rows of every tile: it copies their clean pixels,
// lists their noisy ones in its own shared-memory list and computes them, so
// warps never wait for one another inside a sweep.  Tiles stream through a
// ring of kNS stages; the last warp to finish with a stage refills it with the
// tile kNS further on, so a fast warp can run up to kNS - 1 tiles ahead and the
// tile-to-tile differences in noisy pixels per warp even out.
template <bool FAST>
struct RestoreTma {
    CUtensorMap umap[2];      // state maps over buffer A and buffer B
    CUtensorMap mmap;         // mask map
    const void *base[2];      // A and B, to pick the map of a sweep's source
    int *err;                 // control-block error word
    long long nx, ny;
    float alpha;
    int tiles_x, tiles_y;

    __device__ __forceinline__ size_t state_bytes() const { return (size_t)nx * ny * sizeof(float); }

    // dynamic shared memory: [stages][mbarriers][warps done per stage][tile counter]
    __device__ __forceinline__ unsigned char *stages() const
    {
        extern __shared__ unsigned char smem_dyn[];
        return align_up(smem_dyn, 128);
    }
    __device__ __forceinline__ uint64_t *bars() const { return (uint64_t *)(stages() + kNS * kStage); }
    __device__ __forceinline__ unsigned *done() const { return (unsigned *)(bars() + kNS); }
    // tiles consumed by this CTA so far: tile q uses stage q % kNS, phase (q / kNS) & 1
    __device__ __forceinline__ unsigned *counter() const { return done() + kNS; }

    __device__ __forceinline__ void prologue() const
    {
        if (threadIdx.x == 0) {
            for (int i = 0; i < kNS; ++i) {
                tma::mbar_init(&bars()[i], 1);
                done()[i] = 0u;
            }
            tma::mbar_init_fence();
            *counter() = 0u;
        }
        __syncthreads();
    }

    __device__ __forceinline__ void issue(int tile, int mi, int sb) const
    {
        const int tx = tile % tiles_x, ty = tile / tiles_x;
        const int x0 = tx * kTW, y0 = ty * kTH;
        unsigned char *st = stages() + sb * kStage;
        tma::mbar_expect_tx(&bars()[sb], kTxBytes);
        tma::load_2d(st, &umap[mi], x0 - 4, y0 - 1, &bars()[sb]);
        tma::load_2d(st + kUBytes, &mmap, x0 - 16, y0 - 1, &bars()[sb]);
    }

    template <bool REDUCE>
    __device__ __forceinline__ void sweep(const void *src_v, void *dst_v, Slot *slot) const
    {
        __shared__ unsigned short s_list[kTThreads / 32][4 * kTW];   // each warp's noisy pixels of a tile
        __shared__ int s_stop;
        float *dst = (float *)dst_v;
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        const unsigned lt_mask = (1u << lane) - 1u;
        const int mi = src_v == base[0] ? 0 : 1;
        const int ntiles = tiles_x * tiles_y;
        const int mine = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
        const unsigned q0 = *counter();
        if (tid == 0) {
            s_stop = ld_relaxed_u32((const unsigned *)err) != 0u;   // a wait ran out earlier
            if (!s_stop) {
                tma::fence_proxy_async_global();   // the previous sweep's stores, published by the grid barrier
                for (int i = 0; i < kNS && i < mine; ++i)
                    issue((int)blockIdx.x + i * (int)gridDim.x, mi, (int)((q0 + (unsigned)i) % kNS));
            }
        }
        __syncthreads();                                        // counter read, first tiles issued
        const int nxi = (int)nx, nyi = (int)ny;                 // extents are below 2^31 on this path
        unsigned short *list = s_list[warp];
        unsigned long long sum = 0ull, cnt = 0ull;
        for (int i = 0; i < mine && !s_stop; ++i) {
            const unsigned qn = q0 + (unsigned)i;
            const int sb = (int)(qn % kNS);
            const int tile = (int)blockIdx.x + i * (int)gridDim.x;
            const int x0 = (tile % tiles_x) * kTW, y0 = (tile / tiles_x) * kTH;
            const float *U = (const float *)(stages() + sb * kStage);   // [34][72]: row y0-1+r, column x0-4+c
            const unsigned char *M = stages() + sb * kStage + kUBytes;  // [34][96]: row y0-1+r, column x0-16+c
            const bool got = tma::bounded_wait(&bars()[sb], (qn / kNS) & 1u, tma::kLoadWaitNs, err);
            if (!__all_sync(0xffffffffu, got)) break;
            // the warp's four rows: clean pixels copied, noisy ones listed
            int n = 0;
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int rr = warp * 4 + (h >> 1), cc = (h & 1) * 32 + lane;
                const int y = y0 + rr, x = x0 + cc;
                const bool valid = y < nyi && x < nxi;
                const bool noisy = valid && M[(rr + 1) * kMBoxW + cc + 16] != 0;
                if (valid && !noisy) dst[(size_t)y * (size_t)nxi + x] = U[(rr + 1) * kUBoxW + cc + 4];
                const unsigned m = __ballot_sync(0xffffffffu, noisy);
                if (noisy) list[n + __popc(m & lt_mask)] = (unsigned short)(rr << 6 | cc);
                n += __popc(m);
            }
            __syncwarp();
            for (int t = lane; t < n; t += 32) {
                const int e = list[t];
                const int rr = e >> 6, cc = e & 63;
                const int y = y0 + rr, x = x0 + cc;
                const float *C = U + (rr + 1) * kUBoxW + cc + 4;
                const float uc = *C;
                // every pixel off the grid's border has all 8 neighbours
                const float nv = y > 0 && y + 1 < nyi && x > 0 && x + 1 < nxi
                                     ? restore_interior<FAST>(C, kUBoxW, alpha)
                                     : restore_border<FAST>(C, kUBoxW, alpha, y > 0, y + 1 < nyi, x > 0, x + 1 < nxi);
                dst[(size_t)y * (size_t)nxi + x] = nv;
                if (REDUCE) sum += fixed_2m24(__fsub_rn(nv, uc));
            }
            if (REDUCE && lane == 0) cnt += (unsigned long long)n;
            // done with the stage (and with the list): the last warp out refills it
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                const unsigned before = atomicAdd(&done()[sb], 1u);
                if (before == kTThreads / 32 - 1) {
                    __threadfence_block();
                    done()[sb] = 0u;
                    if (i + kNS < mine) issue(tile + kNS * (int)gridDim.x, mi, sb);
                }
            }
        }
        __syncthreads();                                       // every tile consumed, no copy in flight
        if (tid == 0) *counter() = q0 + (unsigned)mine;
        tma::fence_proxy_async_global();                       // this sweep's stores before the next TMA reads
        if (REDUCE) block_to_slot(slot, 0ull, sum, cnt, sum != 0ull);
    }
};

template <class Op>
__global__ void __launch_bounds__(kTThreads, 4) restore_tma_kernel(const __grid_constant__ Op op, LoopArgs la)
{
    op.prologue();
    persistent_loop_body(op, la);
}

template <class Op>
__global__ void __launch_bounds__(kRThreads, 1) restore_persistent_kernel(Op op, LoopArgs la)
{
    persistent_loop_body(op, la);
}

template <class Op>
__global__ void __launch_bounds__(kRThreads, 1) restore_sweep_kernel(Op op, const void *src, void *dst)
{
    op.template sweep<false>(src, dst, nullptr);
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}


template <bool FAST>
cudaError_t launch_tma(const Problem &p, LoopArgs la, cudaStream_t st)
{
    RestoreTma<FAST> op;
    memset(&op, 0, sizeof(op));
    if (!tma::make_map_2d(&op.umap[0], la.a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p.nx, p.ny, kUBoxW, kBoxH) ||
        !tma::make_map_2d(&op.umap[1], la.b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p.nx, p.ny, kUBoxW, kBoxH) ||
        !tma::make_map_2d(&op.mmap, la.aux, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, p.nx, p.ny, kMBoxW, kBoxH))
        return cudaErrorInvalidValue;
    op.base[0] = la.a;
    op.base[1] = la.b;
    op.err = &la.ctl->err;
    op.nx = p.nx;
    op.ny = p.ny;
    op.alpha = p.alpha;
    op.tiles_x = (int)((p.nx + kTW - 1) / kTW);
    op.tiles_y = (int)((p.ny + kTH - 1) / kTH);
    auto kern = restore_tma_kernel<RestoreTma<FAST>>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTSmem);
    if (e != cudaSuccess) return e;
    return launch_cooperative(kern, kTThreads, kTSmem, 4, la, &op, st);
}

// The TMA path needs 16-byte row strides for the state (nx % 4) and the mask
// (nx % 16), and the tensor-map encoder of the driver.
bool tma_ok(const Problem &p) { return p.nx % 16 == 0 && p.nx < (1ll << 31) && p.ny < (1ll << 31) && tma::encode_fn(); }

}  // namespace

bool restore_tma_ok(const Problem &p) { return tma_ok(p); }

cudaError_t restore_persistent(const Problem &p, LoopArgs la, void *lists, cudaStream_t st)
{
    if (restore_tb_resolve_k(p, la.a, la.b, la.aux) > 1) return restore_tb_persistent(p, la, lists, st);
    if (p.tiling != SLR_TILING_NONE && tma_ok(p))
        return p.math == SLR_MATH_FAST ? launch_tma<true>(p, la, st) : launch_tma<false>(p, la, st);
    if (p.math == SLR_MATH_FAST) {
        RestoreOp<true> op{p.nx, p.ny, p.alpha, (const unsigned char *)la.aux};
        return launch_cooperative(restore_persistent_kernel<RestoreOp<true>>, kRThreads, 0, 1, la, &op, st);
    }
    RestoreOp<false> op{p.nx, p.ny, p.alpha, (const unsigned char *)la.aux};
    return launch_cooperative(restore_persistent_kernel<RestoreOp<false>>, kRThreads, 0, 1, la, &op, st);
}

cudaError_t restore_sweep(const Problem &p, const void *src, void *dst, const void *mask, cudaStream_t st)
{
    if (p.math == SLR_MATH_FAST) {
        RestoreOp<true> op{p.nx, p.ny, p.alpha, (const unsigned char *)mask};
        restore_sweep_kernel<RestoreOp<true>><<<sm_count(), kRThreads, 0, st>>>(op, src, dst);
    } else {
        RestoreOp<false> op{p.nx, p.ny, p.alpha, (const unsigned char *)mask};
        restore_sweep_kernel<RestoreOp<false>><<<sm_count(), kRThreads, 0, st>>>(op, src, dst);
    }
    return cudaGetLastError();
}

}  // namespace slr
