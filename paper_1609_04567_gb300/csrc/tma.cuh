// tma.cuh -- Tensor Memory Accelerator helpers shared by the tiled kernels:
// mbarrier set-up and bounded waits, 2D tiled bulk tensor loads into shared
// memory, proxy fences, and host-side tensor-map encoding.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "slr_internal.cuh"

namespace slr {
namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make initialised mbarriers visible to the async proxy (the TMA unit).
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

// Limit of every wait for a TMA load's mbarrier: a load completes in
// microseconds, so only a lost transfer can reach it.  It is fixed rather
// than the caller's grid-barrier limit, which may be short enough to expire
// during an ordinary load under contention and leave a CTA while its copy
// is still writing shared memory.
constexpr long long kLoadWaitNs = 2000000000ll;

// Wait for phase `parity` of `bar`, giving up after limit_ns of %globaltimer
// (sets DEV_ERR_TIMEOUT in *err and returns false).
__device__ __forceinline__ bool bounded_wait(uint64_t *bar, uint32_t parity, long long limit_ns, int *err)
{
    long long t0 = 0;
    unsigned spins = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++spins & 255u) == 0u) {
            const long long t = global_timer_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) { atomicOr(err, DEV_ERR_TIMEOUT); return false; }
        }
    }
    return true;
}

// One 2D box of `map` at element coordinates (x, y) into shared memory; the
// transfer completes on `bar`.  x * element size must be a multiple of 16.
__device__ __forceinline__ void load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// One 3D box of `map` at element coordinates (x, y, z); x * element size a
// multiple of 16.
__device__ __forceinline__ void load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Order this thread's generic-proxy global accesses with later async-proxy
// (TMA) accesses, across a grid barrier.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// ---- host ------------------------------------------------------------------
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// Row-major 2D map of nx x ny elements of `esize` bytes (row stride
// pitch_bytes, or nx * esize when 0; a multiple of 16), box box_w x box_h,
// zero fill out of range.
inline bool make_map_2d(CUtensorMap *m, const void *base, CUtensorMapDataType dt, size_t esize, long long nx,
                        long long ny, uint32_t box_w, uint32_t box_h,
                        CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_NONE, long long pitch_bytes = 0)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)(pitch_bytes > 0 ? pitch_bytes : nx * (long long)esize)};
    cuuint32_t box[2] = {box_w, box_h};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Row-major 3D map of nx x ny x nz elements (x fastest), box box_x x box_y x
// box_z, no swizzle, zero fill out of range.
inline bool make_map_3d(CUtensorMap *m, const void *base, CUtensorMapDataType dt, size_t esize, long long nx,
                        long long ny, long long nz, uint32_t box_x, uint32_t box_y, uint32_t box_z)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)(nx * (long long)esize), (cuuint64_t)(nx * ny * (long long)esize)};
    cuuint32_t box[3] = {box_x, box_y, box_z};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tma
}  // namespace slr
