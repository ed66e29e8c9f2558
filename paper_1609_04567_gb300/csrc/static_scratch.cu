// static_scratch.cu -- a Jacobi solve that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they want a
// solve: code that runs under a device-memory budget owned by another
// framework's allocator, real-time loops that forbid allocation after start-up,
// or host threads where cudaMalloc/cudaFree would synchronise the device and
// stall other streams.  slr_run_static serves them: the second state buffer
// and the loop's control block live in one file-scope device array, so the
// call needs nothing beyond the caller's own input and output buffers.
//
// The array is a single block shared by every call in the process (on each
// GPU that loads this library it stays resident until the process exits).  A
// call clears the control block before it starts, so the contents a previous
// call left behind do not matter; two calls whose GPU work overlaps (different
// streams, or different host threads on one device) use the same array and
// race.
#include <stdio.h>

#include <mutex>

#include "jacobi_tb.h"
#include "slr_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = slr::kCtlBytes + (size_t)SLR_STATIC_STATE_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

thread_local std::string g_static_error = "no error";

slr_status static_fail(slr_status s, const std::string &msg)
{
    g_static_error = msg;
    return s;
}

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address comes from the
// runtime, once per device, with that device current.  The address is kept
// for the life of the process: a cudaDeviceReset of that device unloads the
// module and leaves it stale, so this entry point must not be used after one.
slr_status scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(SLR_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(SLR_ERR_UNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return static_fail(SLR_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SLR_OK;
}

}  // namespace

extern "C" {

slr_status slr_run_static(const slr_desc *d, void *u, const void *f, int64_t max_iters, void *stream,
                          double *value, int64_t *iters, int32_t *converged)
{
    bool unsup = false;
    const std::string why = slr::describe_invalid(d, &unsup);
    if (!why.empty()) return static_fail(unsup ? SLR_ERR_UNSUPPORTED : SLR_ERR_INVALID_ARG, why);
    if ((d->stencil != SLR_J2D5 && d->stencil != SLR_J3D7) || d->defect_correction)
        return static_fail(SLR_ERR_UNSUPPORTED, "slr_run_static runs the Jacobi stencils (SLR_J2D5, SLR_J3D7) only");
    if (d->loop == SLR_LOOP_HOST)
        return static_fail(SLR_ERR_UNSUPPORTED, "slr_run_static runs the persistent device loop only (loop AUTO or PERSISTENT)");
    if (!u || ((uintptr_t)u & 15u)) return static_fail(SLR_ERR_INVALID_ARG, "u must be a 16-byte aligned device pointer");
    if (!f) return static_fail(SLR_ERR_INVALID_ARG, "f is required");
    if (max_iters < 0) return static_fail(SLR_ERR_INVALID_ARG, "max_iters must be >= 0");
    const slr::Problem p = slr::problem_of(d);
    if (p.state_bytes > (size_t)SLR_STATIC_STATE_BYTES) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "grid state is %zu bytes; slr_run_static holds at most %u bytes (SLR_STATIC_STATE_BYTES), "
                 "use slr_create with a caller workspace instead",
                 p.state_bytes, (unsigned)SLR_STATIC_STATE_BYTES);
        return static_fail(SLR_ERR_INVALID_ARG, buf);
    }
    void *scratch = nullptr;
    slr_status s = scratch_address(&scratch);
    if (s != SLR_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    slr::Ctl *ctl = (slr::Ctl *)scratch;
    // the array keeps the previous call's contents: the whole control block
    // (iteration count, flags, barrier counter, reduce slots) must start at zero
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(slr::Ctl), st);
    if (e != cudaSuccess) return static_fail(SLR_ERR_CUDA, std::string("clear control block: ") + cudaGetErrorString(e));
    slr::LoopArgs la;
    la.a = u;
    la.b = (unsigned char *)scratch + slr::kCtlBytes;
    la.aux = f;
    la.ctl = ctl;
    la.max_iters = max_iters;
    la.limit_ns = d->wait_limit_ns > 0 ? d->wait_limit_ns : 2000000000ll;
    la.tol = p.tol;
    la.reduce = p.reduce;
    la.nblocks = d->grid_ctas;
    la.debug_flags = 0;
    e = slr::jacobi_tb_resolve_k(p, la.a, la.b, la.aux) > 1 ? slr::jacobi_tb_persistent(p, la, st)
                                                             : slr::jacobi_persistent(p, la, st);
    if (e != cudaSuccess) return static_fail(SLR_ERR_CUDA, std::string("persistent loop launch: ") + cudaGetErrorString(e));
    slr::Ctl h;
    e = cudaMemcpyAsync(&h, ctl, sizeof(slr::Ctl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_fail(SLR_ERR_CUDA, std::string("read control block: ") + cudaGetErrorString(e));
    if (value) *value = h.value;
    if (iters) *iters = h.iters;
    if (converged) *converged = h.converged;
    if (h.err & slr::DEV_ERR_TIMEOUT) return static_fail(SLR_ERR_TIMEOUT, "a device-side grid barrier wait ran out its limit");
    return h.converged ? SLR_OK : SLR_NOT_CONVERGED;
}

const char *slr_static_last_error(void) { return g_static_error.c_str(); }

}  // extern "C"
