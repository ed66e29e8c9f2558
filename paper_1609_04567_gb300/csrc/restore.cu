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
#include "slr_internal.cuh"

namespace slr {
namespace {

constexpr int kRThreads = 1024;

template <bool FAST>
struct RestoreOp {
    long long nx, ny;
    float alpha;
    const unsigned char *mask;

    __device__ __forceinline__ size_t state_bytes() const { return (size_t)nx * ny * sizeof(float); }

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
                        const float w = __fdiv_rn(1.0f, __fsqrt_rn(__fadd_rn(alpha, __fmul_rn(t, t))));
                        num = __fadd_rn(num, __fmul_rn(w, uj));
                        den = __fadd_rn(den, w);
                    }
                }
            }
            const float nv = den > 0.0f ? __fdiv_rn(num, den) : uc;
            v[c] = nv;
            if (REDUCE) {
                sum += (unsigned long long)__double2ull_rz((double)fabsf(__fsub_rn(nv, uc)) * 16777216.0);
                cnt += 1ull;
            }
        }
        if (REDUCE) block_to_slot(slot, 0ull, sum, cnt, sum != 0ull);
    }
};

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

}  // namespace

cudaError_t restore_persistent(const Problem &p, LoopArgs la, cudaStream_t st)
{
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
