// selfcheck.cu -- on-device checks of the correctly rounded arithmetic of
// crmath.cuh.  slr_check_exact_division: the Jacobi sweeps' division by the
// constant d against the IEEE division.  slr_check_exact_math: the weight
// arithmetic of the restoration's EXACT math; for every non-negative
// binary32 x (2^31 bit patterns: zero, subnormals, normals, infinity, NaNs)
// inv_sqrt_rn2(x) must equal CUDA's IEEE __frcp_rn(__fsqrt_rn(x)) bit for
// bit, and on its fast-route inputs sqrt_markstein and rcp_markstein must
// equal __fsqrt_rn and __frcp_rn.  The counters live in a file-scope device
// array, so the check allocates nothing.
#include "crmath.cuh"
#include "slr_internal.cuh"

namespace {

static __device__ unsigned long long g_check_counts[4];   // mismatches of 3 checks, inputs checked

__global__ void __launch_bounds__(256) check_kernel(unsigned long long n)
{
    unsigned long long bad[3] = {0ull, 0ull, 0ull}, seen = 0ull;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t b = (uint32_t)i;
        const float x = __uint_as_float(b);
        const float s = __fsqrt_rn(x);
        bad[0] += __float_as_uint(slr::inv_sqrt_rn2(x)) != __float_as_uint(__frcp_rn(s));
        if (b - slr::kInvSqrtLoBits < slr::kInvSqrtHiBits - slr::kInvSqrtLoBits) {
            bad[1] += __float_as_uint(slr::sqrt_markstein(x)) != __float_as_uint(s);
            bad[2] += __float_as_uint(slr::rcp_markstein(s)) != __float_as_uint(__frcp_rn(s));
        }
        seen += 1ull;
    }
    unsigned long long v[4] = {bad[0], bad[1], bad[2], seen};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        unsigned long long t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0 && t) atomicAdd(&g_check_counts[k], t);
    }
}

static __device__ unsigned long long g_div_counts[4];     // mismatches binary32, binary64; inputs of each

// a / d through div_const_rn against the IEEE division: every binary32
// numerator (n32 = 2^32), and n64 binary64 numerators spread over the
// exponent range by a counter-based hash (SplitMix64 finaliser)
__global__ void __launch_bounds__(256) div_check_kernel(float d32, float y32, double d64, double y64,
                                                        unsigned long long n32, unsigned long long n64)
{
    unsigned long long bad32 = 0ull, bad64 = 0ull, s32 = 0ull, s64 = 0ull;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) {   // the host's reciprocals are the IEEE ones
        bad32 += __float_as_uint(y32) != __float_as_uint(__frcp_rn(d32));
        bad64 += __double_as_longlong(y64) != __double_as_longlong(__drcp_rn(d64));
    }
    for (unsigned long long i = t0; i < n32; i += stride) {
        const float a = __uint_as_float((uint32_t)i);
        const float q = slr::div_const_rn(a, d32, y32), r = __fdiv_rn(a, d32);
        // NaN quotients agree as NaNs (their payload bits are not compared)
        bad32 += (__float_as_uint(q) != __float_as_uint(r)) && !(q != q && r != r);
        s32 += 1ull;
    }
    for (unsigned long long i = t0; i < n64; i += stride) {
        unsigned long long z = (i + 1ull) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        // sign and significand from the hash, exponent within +-600 of 1
        const unsigned long long e = 1023ull - 600ull + (z >> 52) % 1201ull;
        const double a = __longlong_as_double((long long)((z & 0x800FFFFFFFFFFFFFull) | (e << 52)));
        const double q = slr::div_const_rn(a, d64, y64), r = __ddiv_rn(a, d64);
        bad64 += __double_as_longlong(q) != __double_as_longlong(r);
        s64 += 1ull;
    }
    unsigned long long v[4] = {bad32, bad64, s32, s64};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        unsigned long long t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0 && t) atomicAdd(&g_div_counts[k], t);
    }
}

}  // namespace

extern "C" slr_status slr_check_exact_division(double d, uint64_t *mismatches, uint64_t *checked, void *stream)
{
    const float d32 = (float)d;
    if (!slr::div_const_ok(d32) || !slr::div_const_ok(d)) return SLR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    void *counts = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&counts, g_div_counts);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * 4, st);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        div_check_kernel<<<(sms > 0 ? sms : 1) * 8, 256, 0, st>>>(d32, slr::host_rcp_rn(d32), d, slr::host_rcp_rn(d),
                                                                  1ull << 32, 1ull << 26);
        e = cudaGetLastError();
    }
    unsigned long long h[4] = {0ull, 0ull, 0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, counts, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SLR_ERR_CUDA;
    if (mismatches) {
        mismatches[0] = h[0];
        mismatches[1] = h[1];
    }
    if (checked) {
        checked[0] = h[2];
        checked[1] = h[3];
    }
    return SLR_OK;
}

extern "C" slr_status slr_check_exact_math(uint64_t *mismatches, uint64_t *checked, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    void *counts = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&counts, g_check_counts);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * 4, st);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        check_kernel<<<(sms > 0 ? sms : 1) * 8, 256, 0, st>>>(1ull << 31);
        e = cudaGetLastError();
    }
    unsigned long long h[4] = {0ull, 0ull, 0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, counts, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SLR_ERR_CUDA;
    if (mismatches) {
        mismatches[0] = h[0];
        mismatches[1] = h[1];
        mismatches[2] = h[2];
    }
    if (checked) *checked = h[3];
    return SLR_OK;
}

// The Sobel magnitude's clamped integer square root: isqrt_clamp255(n) must
// equal min(255, floor(sqrt(n))) (from the IEEE binary64 square root and two
// integer steps) for every 0 <= n < 2^22, the range of Gx^2 + Gy^2.
namespace {
static __device__ unsigned long long g_isqrt_counts[2];

__global__ void __launch_bounds__(256) isqrt_check_kernel(int n)
{
    unsigned long long bad = 0ull, seen = 0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        long long r = (long long)__dsqrt_rn((double)i);
        while (r * r > i) --r;
        while ((r + 1) * (r + 1) <= i) ++r;
        bad += slr::isqrt_clamp255(i) != (int)(r < 255 ? r : 255);
        seen += 1ull;
    }
    atomicAdd(&g_isqrt_counts[0], bad);
    atomicAdd(&g_isqrt_counts[1], seen);
}
}  // namespace

extern "C" slr_status slr_check_exact_isqrt(uint64_t *mismatches, uint64_t *checked, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    void *counts = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&counts, g_isqrt_counts);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * 2, st);
    if (e == cudaSuccess) {
        isqrt_check_kernel<<<1024, 256, 0, st>>>(1 << 22);
        e = cudaGetLastError();
    }
    unsigned long long h[2] = {0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, counts, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SLR_ERR_CUDA;
    if (mismatches) *mismatches = h[0];
    if (checked) *checked = h[1];
    return SLR_OK;
}
