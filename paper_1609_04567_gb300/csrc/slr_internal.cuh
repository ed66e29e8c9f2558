// slr_internal.cuh -- shared device machinery of libslr: the workspace control
// block, the bounded grid barrier, the reduce slots and the persistent loop
// skeleton that keeps the loop-of-stencil-reduce iteration (Sec. 3.1) on the
// device.  Kernels of every stencil include this header.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>

#include "slr.h"

// __longlong_as_double exists only in device code; this works on both sides.
__host__ __device__ __forceinline__ double __longlong_as_double_hd(unsigned long long b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double d;
    __builtin_memcpy(&d, &b, 8);
    return d;
#endif
}

namespace slr {

// Device error bits written into Ctl::err.
enum : int { DEV_ERR_TIMEOUT = 1 };

// One reduce slot: the combined value of every CTA for one sweep.  All fields
// combine with order-independent integer operations (max of non-negative
// binary64 bit patterns, 64-bit sums, or), so the result is reproducible
// whatever order the CTAs arrive in.
struct Slot {
    unsigned long long maxbits;   // max |delta| as binary64 bits (>= 0 orders like u64)
    unsigned long long sum;       // fixed-point sum of |delta| (units 2^-24)
    unsigned long long cnt;       // live cells / masked pixels
    unsigned int changed;         // or of per-item "changed"
    unsigned int pad;
};

constexpr int kSlots = 3;         // reduce slots cycled by sweep number (see loop)
constexpr int kMaxK = 32;         // most sweeps a temporal-blocked pass may fuse

// Control block at the start of the workspace.  Written by device and host.
struct Ctl {
    unsigned long long bar;       // grid barrier arrivals (zeroed before every launch)
    int err;                      // DEV_ERR_* bits
    int converged;                // 1 once the test has passed
    long long iters;              // total iterations run by the handle
    double value;                 // reduced value of the last iteration
    unsigned long long count;     // integer count of the last iteration
    int changed;                  // any item changed in the last iteration
    int pad;
    Slot slot[kSlots];
    Slot sub[kSlots][kMaxK];      // per-sub-step slots of temporal-blocked passes
    unsigned int next_tile[kSlots];   // tiles handed out in a pass (dynamically scheduled passes)
    unsigned int pad2;
};

constexpr size_t kCtlBytes = 4096;            // Ctl padded; state buffer B follows
static_assert(sizeof(Ctl) <= kCtlBytes, "control block too large");

// p advanced to the next multiple of `align` bytes (a power of two) by pointer
// arithmetic on p itself, so that a pointer into shared memory stays one: a
// round trip through an integer would leave the compiler a generic pointer
// and turn every access through it into a generic load or store.
template <class T>
__device__ __forceinline__ T *align_up(T *p, uintptr_t align)
{
    const uintptr_t off = (align - ((uintptr_t)p & (align - 1))) & (align - 1);
    return (T *)((unsigned char *)p + off);
}

__device__ __forceinline__ long long global_timer_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_int(const int *p)
{
    return *(const volatile int *)p;
}

// Grid-wide barrier for a co-resident (cooperative) grid.  Thread 0 of each
// CTA publishes the CTA's writes (bar.sync, then its arrival as a gpu-scope
// release, which covers the writes the CTA barrier ordered before it), and
// spins with acquire loads until `target` arrivals are counted.  The spin
// is bounded by `limit_ns` of %globaltimer: on expiry it sets DEV_ERR_TIMEOUT
// and every CTA returns false (and then leaves the kernel), so a missing CTA
// can never hang the GPU.
__device__ __forceinline__ bool grid_barrier(Ctl *ctl, unsigned long long target, long long limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        red_release_add(&ctl->bar, 1ull);
        const long long t0 = global_timer_ns();
        unsigned spins = 0;
        while (ld_acquire(&ctl->bar) < target) {
            if ((++spins & 15u) == 0u) {
                if (ld_volatile_int(&ctl->err)) { ok = 0; break; }
                if (global_timer_ns() - t0 > limit_ns) {
                    atomicOr(&ctl->err, DEV_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Block-wide reduction of one thread's contribution into a slot with one
// atomic per field per CTA.  blockDim.x must be a multiple of 32, <= 1024.
__device__ __forceinline__ void block_to_slot(Slot *slot, unsigned long long maxbits,
                                              unsigned long long sum, unsigned long long cnt,
                                              unsigned int changed)
{
    __shared__ unsigned long long s_max[32], s_sum[32], s_cnt[32];
    __shared__ unsigned int s_ch[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long m2 = __shfl_xor_sync(0xffffffffu, maxbits, o);
        maxbits = m2 > maxbits ? m2 : maxbits;
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        changed |= __shfl_xor_sync(0xffffffffu, changed, o);
    }
    if (lane == 0) { s_max[warp] = maxbits; s_sum[warp] = sum; s_cnt[warp] = cnt; s_ch[warp] = changed; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        maxbits = lane < nw ? s_max[lane] : 0ull;
        sum = lane < nw ? s_sum[lane] : 0ull;
        cnt = lane < nw ? s_cnt[lane] : 0ull;
        changed = lane < nw ? s_ch[lane] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long m2 = __shfl_xor_sync(0xffffffffu, maxbits, o);
            maxbits = m2 > maxbits ? m2 : maxbits;
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            changed |= __shfl_xor_sync(0xffffffffu, changed, o);
        }
        if (lane == 0) {
            if (maxbits) atomicMax(&slot->maxbits, maxbits);
            if (sum) atomicAdd(&slot->sum, sum);
            if (cnt) atomicAdd(&slot->cnt, cnt);
            if (changed) atomicOr(&slot->changed, 1u);
        }
    }
    __syncthreads();
}

// |delta| truncated to a multiple of 2^-24, as an integer: trunc(|d| * 2^24).
// Scaling by 2^24 is exact in binary32, so for |d| < 256 (the product below
// 2^32) a binary32 multiply and an unsigned 32-bit truncation give the
// integer.  From 256 up the product is an integer already: the significand
// shifted by the exponent (integer operations only, so no binary64 work is
// compiled into the sweeps).  Products of 2^64 and more (|d| >= 2^40, or NaN)
// saturate.
static __device__ __noinline__ unsigned long long fixed_2m24_large(float a)
{
    if (!(a < 1099511627776.0f)) return ~0ull;
    const uint32_t b = __float_as_uint(a);
    // a = m * 2^(E - 150) with m the 24-bit significand; a * 2^24 = m << (E - 126)
    const unsigned long long m = (b & 0x7FFFFFu) | 0x800000u;
    return m << ((int)(b >> 23) - 126);
}
__device__ __forceinline__ unsigned long long fixed_2m24(float d)
{
    const float a = fabsf(d);
    if (a < 256.0f) return (unsigned long long)__float2uint_rz(a * 16777216.0f);
    return fixed_2m24_large(a);
}

// fixed_2m24 without a branch, for hot loops: the product a * 2^24 is exact
// and below 2^64 for every a < 2^40, so one conversion to a 64-bit integer
// gives the same integer; larger values and NaN saturate as above.
__device__ __forceinline__ unsigned long long fixed_2m24_nb(float d)
{
    const float a = fabsf(d);
    return a < 1099511627776.0f ? __float2ull_rz(a * 16777216.0f) : ~0ull;
}

// What every stencil's loop needs to decide after a sweep.
struct Decision {
    double value;
    unsigned long long count;
    int changed;
    int converged;
};

// The convergence test c(/+:d, it) of each reduce operator (Sec. 3.1 -d/-s).
__host__ __device__ __forceinline__ Decision decide(int reduce, const Slot &s, double tol)
{
    Decision d;
    d.changed = s.changed != 0u;
    d.count = s.cnt;
    if (reduce == SLR_RED_MAX_ABS_DELTA) {
        d.value = __longlong_as_double_hd(s.maxbits);
        d.converged = d.value < tol;
    } else if (reduce == SLR_RED_MEAN_ABS_DELTA_MASKED) {
        d.value = s.cnt ? ((double)s.sum * 0x1p-24) / (double)s.cnt : 0.0;
        d.converged = d.value < tol;
    } else {
        d.value = (double)s.cnt;
        d.converged = !d.changed;
    }
    return d;
}

// Sweeps of the next pass of a temporal-blocked loop (at most K): where the
// last pass's reduced values (v0 after its first sweep, v1 after its last of
// kp), decaying geometrically, predict the first value below tol, so that a
// stop seldom falls inside a pass and costs a rerun of it; K when the values
// do not decay or the prediction lies K or more sweeps ahead.  Only the
// speed depends on it: a stop inside a pass still reruns that pass.  Every
// CTA computes it from the same values and gets the same pass length.
__device__ __forceinline__ int predict_pass(double v0, double v1, int kp, double tol, int K)
{
    if (kp < 2 || !(tol > 0.0) || !(v1 > 0.0) || !(v1 < v0) || !(v1 >= tol)) return K;
    const double lr = log(v1 / v0) / (double)(kp - 1);   // log of the per-sweep ratio, < 0
    const double need = log(tol / v1) / lr;              // sweeps past the pass's last one
    if (!(need < (double)(K - 1))) return K;
    const int n = (int)floor(need) + 1;
    return n < 1 ? 1 : n;
}

// Arguments of every loop launch.
struct LoopArgs {
    void *a;                 // state buffer A (the caller's u)
    void *b;                 // state buffer B (workspace)
    const void *aux;         // f or mask
    Ctl *ctl;
    long long max_iters;     // absolute cap on Ctl::iters
    long long limit_ns;      // barrier wait limit
    double tol;
    int reduce;
    int nblocks;             // grid size of the persistent launch; on entry to a launcher,
                             // the requested CTAs (0 = all that can be co-resident)
    int debug_flags;         // SLR_DEBUG_* (fault injection for tests)
};


__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ Slot read_slot(const Slot *s)
{
    Slot r;
    r.maxbits = ld_relaxed_u64(&s->maxbits);
    r.sum = ld_relaxed_u64(&s->sum);
    r.cnt = ld_relaxed_u64(&s->cnt);
    r.changed = ld_relaxed_u32(&s->changed);
    r.pad = 0;
    return r;
}

__device__ __forceinline__ void zero_slot(Slot *s)
{
    s->maxbits = 0ull; s->sum = 0ull; s->cnt = 0ull; s->changed = 0u;
}

// Grid-stride copy of `bytes` from src to dst (state write-back B -> A).
// Both pointers are at least 16-byte aligned.
__device__ __forceinline__ void grid_copy(const void *src, void *dst, size_t bytes)
{
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nthr = (size_t)gridDim.x * blockDim.x;
    const size_t n16 = bytes / 16;
    const uint4 *s4 = (const uint4 *)src;
    uint4 *d4 = (uint4 *)dst;
    for (size_t i = tid; i < n16; i += nthr) d4[i] = __ldcg(s4 + i);
    const unsigned char *s1 = (const unsigned char *)src;
    unsigned char *d1 = (unsigned char *)dst;
    for (size_t i = n16 * 16 + tid; i < bytes; i += nthr) d1[i] = __ldcg(s1 + i);
}

// The loop-of-stencil-reduce-d-s procedure of Sec. 3.1 as one cooperative
// launch.  Sweep n reads buffer (n even ? A : B) and writes the other; its
// reduce goes to slot n % 3.  After the grid barrier every CTA reads the slot,
// takes the same decision, and either stops or swaps buffers.  Slot n+2 is
// cleared by CTA 0 right after barrier n: every CTA has read it (after
// barrier n-1) before arriving at barrier n, and nobody adds to it before
// barrier n+1.  The host clears slots 0 and 1 and the barrier counter before
// the launch.  When the last sweep wrote B the grid copies B back to A, so the
// caller's u always holds the result.
template <class Op>
__device__ __forceinline__ void persistent_loop_body(const Op &op, const LoopArgs &la)
{
    __shared__ int s_stop;
    Ctl *ctl = la.ctl;
    const long long it0 = ctl->iters;
    if (ctl->converged || it0 >= la.max_iters || ctl->err) return;
    if ((la.debug_flags & SLR_DEBUG_SKIP_ARRIVAL) && blockIdx.x == gridDim.x - 1) return;
    for (long long n = 0;; ++n) {
        const void *src = (n & 1) ? la.b : la.a;
        void *dst = (n & 1) ? la.a : la.b;
        op.template sweep<true>(src, dst, &ctl->slot[n % kSlots]);
        if (!grid_barrier(ctl, (unsigned long long)(n + 1) * (unsigned long long)la.nblocks, la.limit_ns))
            return;
        if (threadIdx.x == 0) {
            if (blockIdx.x == 0) zero_slot(&ctl->slot[(n + 2) % kSlots]);
            const Slot s = read_slot(&ctl->slot[n % kSlots]);
            const Decision d = decide(la.reduce, s, la.tol);
            const long long it = it0 + n + 1;
            const int stop = d.converged || it >= la.max_iters;
            if (stop && blockIdx.x == 0) {
                ctl->iters = it;
                ctl->value = d.value;
                ctl->count = d.count;
                ctl->changed = d.changed;
                ctl->converged = d.converged;
            }
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) {
            if ((n & 1) == 0) grid_copy(la.b, la.a, op.state_bytes());
            return;
        }
    }
}

}  // namespace slr


namespace slr {

// Everything a kernel needs to know about one problem, resolved on the host
// from an slr_desc.
struct Problem {
    int stencil, storage, reduce, wrap, math, k;
    int tiling;                      // slr_tiling (RESTORE8)
    long long nx, ny, nz;
    double ghost, h2, d, tol;        // Jacobi constants in binary64: h2 = h*h, d = 2n + sigma*h2
    float ghostf, h2f, df, alpha;    // the same rounded to binary32
    size_t elem_bytes, state_bytes;
};

// Host-side launchers, one set per stencil family (life.cu, jacobi.cu,
// restore.cu).  `persistent` runs the whole loop in one cooperative launch;
// `sweep` is one unfused sweep (no reduce) for the host-driven loop.
cudaError_t life_persistent(const Problem &p, LoopArgs la, cudaStream_t st);
cudaError_t life_sweep(const Problem &p, const void *src, void *dst, cudaStream_t st);
cudaError_t life_normalize(const Problem &p, void *u, cudaStream_t st);
// Temporal-blocked Life: k generations per pass over a bit-packed copy of the
// grid kept in two workspace buffers (life_tb.cu).  Returns
// cudaErrorNotSupported when the grid does not fit its tiling rules.
bool life_tb_supported(const Problem &p);
int life_tb_default_k(const Problem &p, int nblocks);
// The k a temporal-blocked launch of p would run with `grid_request` CTAs
// requested (p.k when > 1, else the default for the grid).
int life_tb_resolve_k(const Problem &p, int grid_request);
size_t life_tb_bits_bytes(long long nx, long long ny);
cudaError_t life_tb_persistent(const Problem &p, LoopArgs la, void *bits0, void *bits1, cudaStream_t st);
cudaError_t jacobi_persistent(const Problem &p, LoopArgs la, cudaStream_t st);
// Whether a persistent Jacobi sweep over state buffers a, b with right-hand
// side f takes the TMA path (forced: as for SLR_TILING_TMA, any grid size).
bool jacobi_tma_ok(const Problem &p, const void *a, const void *b, const void *f, bool forced);
cudaError_t jacobi_sweep(const Problem &p, const void *src, void *dst, const void *f, cudaStream_t st);
// `lists`: the workspace area of restore_tb_list_bytes(nx, ny) bytes (256-byte aligned).
cudaError_t restore_persistent(const Problem &p, LoopArgs la, void *lists, cudaStream_t st);
// Temporal-blocked restoration (restore_tb.cu): k sweeps per pass over 64 x 64
// tiles with an 8-pixel halo.  Supported for any width (rows that do not start
// on 16-byte boundaries go through padded copies in `lists`' area) and, where
// a buffer is read in place, 16-byte aligned arrays; resolve_k gives 1 (the one-sweep
// kernels) for temporal_k 1, for a problem it does not accept, or for
// temporal_k 0 with an explicit tiling; kRestoreTbDefaultK for temporal_k 0
// with SLR_TILING_AUTO; else temporal_k capped at 8.
constexpr int kRestoreTbDefaultK = 8;
bool restore_tb_supported(const Problem &p, const void *a, const void *b, const void *mask);
int restore_tb_resolve_k(const Problem &p, const void *a, const void *b, const void *mask);
// Workspace bytes of the per-tile noisy-pixel records (0 for rows that are not
// whole 16-byte mask groups, where the temporal-blocked kernel does not run).
size_t restore_tb_list_bytes(long long nx, long long ny);
cudaError_t restore_tb_persistent(const Problem &p, LoopArgs la, void *lists, cudaStream_t st);
// Whether the TMA-tiled restoration sweep accepts p (nx % 16 == 0).
bool restore_tma_ok(const Problem &p);
cudaError_t restore_sweep(const Problem &p, const void *src, void *dst, const void *mask, cudaStream_t st);
// FP64 defect correction around FP32 Jacobi inner solves, 2D and 3D (dc.cu).
size_t dc_workspace_bytes(long long nx, long long ny, long long nz);
cudaError_t dc_persistent(const Problem &p, LoopArgs la, int inner, void *fp32_area, cudaStream_t st);
// The separate reduce kernel of the host-driven loop: delta between two
// states (and the mask), reduced into *slot.
cudaError_t reduce_states(const Problem &p, const void *src, const void *dst, const void *aux,
                          Slot *slot, cudaStream_t st);

// Descriptor checks and problem set-up (slr_api.cu), for other entry points.
std::string describe_invalid(const slr_desc *d, bool *unsupported);
Problem problem_of(const slr_desc *d);
// slr_create with (use_cache) or without the autotuner's cache.
slr_status create_handle(const slr_desc *d, void *u, const void *aux, void *workspace, size_t workspace_bytes,
                         void *stream, slr_handle *out, bool use_cache);
const slr_desc *handle_desc(slr_handle h);
// Fill the library-choice fields of *d from the autotuner's cache (tune.cu).
void tune_fill(slr_desc *d);

// CTAs of a persistent launch: the co-resident capacity (sms * per_sm), or
// the request when it is smaller and positive.
inline int grid_ctas(int sms, int per_sm, int request)
{
    const int cap = sms * per_sm;
    return request > 0 && request < cap ? request : cap;
}

// Cooperative launch of a persistent kernel with as many CTAs as can be
// co-resident (at most `max_per_sm` per SM), or la.nblocks if that is
// smaller and positive.  Sets la.nblocks to the grid launched.
template <class K>
cudaError_t launch_cooperative(K kernel, int threads, size_t smem, int max_per_sm, LoopArgs &la,
                               const void *op, cudaStream_t st)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    if (per_sm > max_per_sm) per_sm = max_per_sm;
    la.nblocks = grid_ctas(sms, per_sm, la.nblocks);
    void *args[] = {const_cast<void *>(op), (void *)&la};
    return cudaLaunchCooperativeKernel((const void *)kernel, dim3(la.nblocks), dim3(threads), args, smem, st);
}

}  // namespace slr
