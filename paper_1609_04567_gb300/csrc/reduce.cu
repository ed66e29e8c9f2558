// reduce.cu -- the separate reduce kernel of the host-driven loop (the plain
// schema of Fig. 2: stencil launch, then reduce, then a host-side test).  It
// recomputes the per-item change between the old and the new state and
// reduces it with the operator of the stencil, into one slot.
#include "slr_internal.cuh"

namespace slr {
namespace {

__device__ __forceinline__ double ldv(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float ldv(const float *p) { return __ldcg(p); }
__device__ __forceinline__ float ldv(const __nv_bfloat16 *p)
{
    return __uint_as_float((uint32_t)__ldcg((const unsigned short *)p) << 16);
}
__device__ __forceinline__ float ldv(const __half *p)
{
    return __half2float(__ushort_as_half(__ldcg((const unsigned short *)p)));
}
__device__ __forceinline__ unsigned long long abs_bits(double d) { return (unsigned long long)__double_as_longlong(fabs(d)); }
__device__ __forceinline__ unsigned long long abs_bits(float d) { return (unsigned long long)__double_as_longlong((double)fabsf(d)); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }

template <class T>
__global__ void reduce_max_delta(const T *a, const T *b, size_t n, Slot *slot)
{
    unsigned long long mx = 0ull;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long bits = abs_bits(sub_rn(ldv(b + i), ldv(a + i)));
        mx = bits > mx ? bits : mx;
    }
    block_to_slot(slot, mx, 0ull, 0ull, mx != 0ull);
}

__global__ void reduce_masked_mean(const float *a, const float *b, const unsigned char *mask, size_t n, Slot *slot)
{
    unsigned long long sum = 0ull, cnt = 0ull;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (!mask[i]) continue;
        sum += fixed_2m24(__fsub_rn(__ldcg(b + i), __ldcg(a + i)));
        cnt += 1ull;
    }
    block_to_slot(slot, 0ull, sum, cnt, sum != 0ull);
}

__global__ void reduce_life(const unsigned char *a, const unsigned char *b, size_t n, Slot *slot)
{
    unsigned long long cnt = 0ull;
    unsigned int ch = 0u;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned char x = __ldcg(b + i);
        cnt += x != 0;
        ch |= (unsigned)(x != __ldcg(a + i));
    }
    block_to_slot(slot, 0ull, 0ull, cnt, ch);
}

}  // namespace

cudaError_t reduce_states(const Problem &p, const void *src, const void *dst, const void *aux, Slot *slot,
                          cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (sms > 0 ? sms : 1) * 4;
    const size_t n = p.state_bytes / p.elem_bytes;
    if (p.stencil == SLR_LIFE) {
        reduce_life<<<grid, 256, 0, st>>>((const unsigned char *)src, (const unsigned char *)dst, n, slot);
    } else if (p.stencil == SLR_RESTORE8) {
        reduce_masked_mean<<<grid, 256, 0, st>>>((const float *)src, (const float *)dst,
                                                 (const unsigned char *)aux, n, slot);
    } else {
        switch (p.storage) {
        case SLR_F64: reduce_max_delta<<<grid, 256, 0, st>>>((const double *)src, (const double *)dst, n, slot); break;
        case SLR_F32: reduce_max_delta<<<grid, 256, 0, st>>>((const float *)src, (const float *)dst, n, slot); break;
        case SLR_BF16:
            reduce_max_delta<<<grid, 256, 0, st>>>((const __nv_bfloat16 *)src, (const __nv_bfloat16 *)dst, n, slot);
            break;
        case SLR_F16: reduce_max_delta<<<grid, 256, 0, st>>>((const __half *)src, (const __half *)dst, n, slot); break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

}  // namespace slr
