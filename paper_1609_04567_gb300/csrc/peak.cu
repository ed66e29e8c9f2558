// peak.cu -- measured throughput of the logic pipe: the denominator of the
// Game of Life roofline.  The bit-sliced Life update is three-input logic
// operations and funnel shifts, which issue to the integer logic pipe; this
// kernel keeps that pipe busy with independent three-input logic operations
// (eight chains per thread, each step reading the previous step's values,
// 64 warps per SM) and the call times it with CUDA events.
#include "slr_internal.cuh"

namespace {

static __device__ unsigned int g_logic_sink[1];

__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    // (a ^ b) | (~a & c): neither idempotent nor an involution in a
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x5E;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__global__ void __launch_bounds__(256) logic_rate_kernel(uint32_t seed, int iters)
{
    uint32_t x[8];
    const uint32_t y = seed ^ (threadIdx.x * 0x9E3779B9u) ^ blockIdx.x;
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = seed * (uint32_t)(2 * i + 1) + threadIdx.x;
    for (int n = 0; n < iters; ++n) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            uint32_t t[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) t[i] = lop3(x[i], x[(i + 1) & 7], y);
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = t[i];
        }
    }
    uint32_t acc = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= x[i];
    if (acc == seed) g_logic_sink[0] = acc;      // keeps the chains live
}

}  // namespace

extern "C" slr_status slr_measure_logic_rate(double *ops_per_s, double *ms, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return SLR_ERR_CUDA;
    const int blocks = sms * 8, threads = 256, iters = 2048;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return SLR_ERR_CUDA;
    }
    logic_rate_kernel<<<blocks, threads, 0, st>>>(12345u, iters / 8);      // warm-up
    cudaEventRecord(a, st);
    logic_rate_kernel<<<blocks, threads, 0, st>>>(67890u, iters);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess || t <= 0.0f) return SLR_ERR_CUDA;
    const double ops = (double)blocks * threads * (double)iters * 16.0 * 8.0;
    if (ops_per_s) *ops_per_s = ops / ((double)t * 1e-3);
    if (ms) *ms = (double)t;
    return SLR_OK;
}
