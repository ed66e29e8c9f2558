// slr_api.cu -- the C ABI of include/slr.h: descriptor validation, workspace
// layout, handle state and the two loop drivers (persistent device loop and
// the plain host-driven loop of Fig. 2).
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "jacobi_tb.h"
#include "slr_internal.cuh"

using slr::Ctl;
using slr::Problem;
using slr::Slot;

struct slr_ctx {
    slr_desc desc;
    Problem prob;
    void *u;
    const void *aux;
    unsigned char *ws;
    size_t ws_bytes;
    cudaStream_t stream;
    Ctl host_ctl;          // host copy used by the host-driven loop and by reads
    std::string err;
};

namespace {

thread_local std::string g_create_error = "no error";

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int elem_bytes_of(int dtype)
{
    switch (dtype) {
    case SLR_U8: return 1;
    case SLR_BF16:
    case SLR_F16: return 2;
    case SLR_F32: return 4;
    case SLR_F64: return 8;
    default: return 0;
    }
}

int reduce_of(int stencil)
{
    switch (stencil) {
    case SLR_J2D5:
    case SLR_J3D7: return SLR_RED_MAX_ABS_DELTA;
    case SLR_LIFE: return SLR_RED_LIVE_COUNT;
    case SLR_RESTORE8: return SLR_RED_MEAN_ABS_DELTA_MASKED;
    default: return -1;
    }
}

// Returns an empty string when the descriptor is valid, else the reason.
// *unsupported is set for well-formed but unimplemented combinations.
std::string check_desc(const slr_desc *d, bool *unsupported)
{
    *unsupported = false;
    if (!d) return "descriptor is NULL";
    if (d->stencil < SLR_J2D5 || d->stencil > SLR_RESTORE8) return "unknown stencil";
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return "extents must be >= 1";
    if (d->nx > (1ll << 31) - 4096 || d->ny > (1ll << 31) - 4096 || d->nz > (1ll << 31) - 4096)
        return "extent too large (each must be below 2^31 - 4096)";
    if (d->stencil != SLR_J3D7 && d->nz != 1) return "2D stencil needs nz == 1";
    if (d->boundary != SLR_DIRICHLET && d->boundary != SLR_WRAP) return "unknown boundary";
    if (d->reduce != reduce_of(d->stencil)) return "reduce operator does not match the stencil";
    if (d->loop < SLR_LOOP_AUTO || d->loop > SLR_LOOP_PERSISTENT) return "unknown loop mode";
    if (d->math != SLR_MATH_EXACT && d->math != SLR_MATH_FAST) return "unknown math mode";
    if (d->temporal_k < 0 || d->temporal_k > slr::kMaxK) return "temporal_k out of range";
    if (d->grid_ctas < 0) return "grid_ctas must be >= 0";
    if (d->tiling < SLR_TILING_AUTO || d->tiling > SLR_TILING_TMA) return "unknown tiling";
    switch (d->stencil) {
    case SLR_J2D5:
    case SLR_J3D7:
        if (d->storage != SLR_F64 && d->storage != SLR_F32 && d->storage != SLR_BF16 && d->storage != SLR_F16)
            return "Jacobi storage must be F64, F32, BF16 or F16";
        if (!(d->h == d->h) || !(d->sigma == d->sigma)) return "sigma/h is NaN";
        break;
    case SLR_LIFE:
        if (d->storage != SLR_U8) return "Life storage must be U8";
        break;
    case SLR_RESTORE8:
        if (d->storage != SLR_F32) return "restoration storage must be F32";
        if (d->boundary != SLR_DIRICHLET) {
            *unsupported = true;
            return "restoration leaves out-of-range neighbours out; only DIRICHLET is accepted";
        }
        if (!(d->alpha > 0.0f)) return "alpha must be > 0";
        break;
    }
    if (d->defect_correction) {
        if ((d->stencil != SLR_J2D5 && d->stencil != SLR_J3D7) || d->storage != SLR_F64 ||
            d->boundary != SLR_DIRICHLET || d->ghost != 0.0 || d->loop == SLR_LOOP_HOST) {
            *unsupported = true;
            return "defect correction runs SLR_J2D5 or SLR_J3D7 in F64 with ghost 0 on the persistent loop";
        }
        if (d->inner_sweeps < 0) return "inner_sweeps must be >= 0";
    }
    const double cells = (double)d->nx * (double)d->ny * (double)d->nz;
    if (cells * elem_bytes_of(d->storage) > 4.0e11) return "grid larger than device memory";
    return std::string();
}

Problem make_problem(const slr_desc *d)
{
    Problem p;
    memset(&p, 0, sizeof(p));
    p.stencil = d->stencil;
    p.storage = d->storage;
    p.reduce = d->reduce;
    p.wrap = d->boundary == SLR_WRAP;
    p.math = d->math;
    p.k = d->temporal_k;
    p.tiling = d->tiling;
    p.nx = d->nx; p.ny = d->ny; p.nz = d->nz;
    p.ghost = d->ghost;
    p.tol = d->tol;
    // mesh width and Jacobi constants: h2 = h*h, d = 2n + sigma*h2 in binary64,
    // rounded once for the binary32 paths
    const double h = d->h > 0.0 ? d->h : 1.0 / (double)(d->nx + 1);
    p.h2 = h * h;
    p.d = (d->stencil == SLR_J3D7 ? 6.0 : 4.0) + d->sigma * p.h2;
    p.ghostf = (float)d->ghost;
    p.h2f = (float)p.h2;
    p.df = (float)p.d;
    p.alpha = d->alpha;
    p.elem_bytes = (size_t)elem_bytes_of(d->storage);
    p.state_bytes = (size_t)d->nx * (size_t)d->ny * (size_t)d->nz * p.elem_bytes;
    return p;
}

slr_status fail(slr_handle h, slr_status s, const std::string &msg)
{
    if (h) h->err = msg; else g_create_error = msg;
    return s;
}

slr_status cuda_fail(slr_handle h, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, SLR_ERR_CUDA, m);
}

Ctl *dev_ctl(slr_handle h) { return (Ctl *)h->ws; }
void *dev_b(slr_handle h) { return h->ws + slr::kCtlBytes; }
// Life only: the two bit-packed buffers of the temporal-blocked path
void *dev_bits(slr_handle h, int i)
{
    const size_t b = round_up(slr::life_tb_bits_bytes(h->prob.nx, h->prob.ny), 256);
    return h->ws + slr::kCtlBytes + round_up(h->prob.state_bytes, 256) + (size_t)i * b;
}

slr_status run_persistent(slr_handle h, int64_t max_iters)
{
    Ctl *ctl = dev_ctl(h);
    cudaError_t e = cudaMemsetAsync(&ctl->bar, 0, sizeof(ctl->bar), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&ctl->slot[0], 0, 2 * sizeof(Slot), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&ctl->sub[0][0], 0, 2 * sizeof(ctl->sub[0]), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&ctl->next_tile[0], 0, 2 * sizeof(ctl->next_tile[0]), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reset loop state");
    slr::LoopArgs la;
    la.a = h->u;
    la.b = dev_b(h);
    la.aux = h->aux;
    la.ctl = ctl;
    la.max_iters = max_iters;
    la.limit_ns = h->desc.wait_limit_ns > 0 ? h->desc.wait_limit_ns : 2000000000ll;
    la.tol = h->prob.tol;
    la.reduce = h->prob.reduce;
    la.nblocks = h->desc.grid_ctas;
    la.debug_flags = h->desc.debug_flags;
    switch (h->prob.stencil) {
    case SLR_LIFE:
        e = h->prob.k != 1 && slr::life_tb_supported(h->prob)
                ? slr::life_tb_persistent(h->prob, la, dev_bits(h, 0), dev_bits(h, 1), h->stream)
                : slr::life_persistent(h->prob, la, h->stream);
        break;
    case SLR_J2D5:
    case SLR_J3D7:
        e = h->desc.defect_correction
                ? slr::dc_persistent(h->prob, la, h->desc.inner_sweeps,
                                     h->ws + slr::kCtlBytes + round_up(h->prob.state_bytes, 256), h->stream)
                : slr::jacobi_tb_resolve_k(h->prob, la.a, la.b, la.aux) > 1
                      ? slr::jacobi_tb_persistent(h->prob, la, h->stream)
                      : slr::jacobi_persistent(h->prob, la, h->stream);
        break;
    case SLR_RESTORE8:
        e = slr::restore_persistent(h->prob, la, h->ws + slr::kCtlBytes + round_up(h->prob.state_bytes, 256),
                                    h->stream);
        break;
    default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "persistent loop launch");
    return SLR_OK;
}

slr_status read_ctl(slr_handle h)
{
    cudaError_t e = cudaMemcpyAsync(&h->host_ctl, dev_ctl(h), sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "read control block");
    return SLR_OK;
}

// The plain schema of Fig. 2: per iteration one sweep launch, one reduce
// launch, a device-to-host copy of the reduced value and the test on the host.
slr_status run_host(slr_handle h, int64_t max_iters)
{
    slr_status s = read_ctl(h);
    if (s != SLR_OK) return s;
    Ctl &c = h->host_ctl;
    if (c.converged || c.iters >= max_iters) return SLR_OK;
    Ctl *ctl = dev_ctl(h);
    void *a = h->u, *b = dev_b(h);
    long long n = 0;
    for (;; ++n) {
        const void *src = (n & 1) ? b : a;
        void *dst = (n & 1) ? a : b;
        cudaError_t e;
        switch (h->prob.stencil) {
        case SLR_LIFE: e = slr::life_sweep(h->prob, src, dst, h->stream); break;
        case SLR_RESTORE8: e = slr::restore_sweep(h->prob, src, dst, h->aux, h->stream); break;
        default: e = slr::jacobi_sweep(h->prob, src, dst, h->aux, h->stream); break;
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(&ctl->slot[0], 0, sizeof(Slot), h->stream);
        if (e == cudaSuccess) e = slr::reduce_states(h->prob, src, dst, h->aux, &ctl->slot[0], h->stream);
        Slot hs;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, &ctl->slot[0], sizeof(Slot), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "host-driven iteration");
        const slr::Decision d = slr::decide(h->prob.reduce, hs, h->prob.tol);
        c.iters += 1;
        c.value = d.value;
        c.count = d.count;
        c.changed = d.changed;
        c.converged = d.converged;
        if (d.converged || c.iters >= max_iters) break;
    }
    cudaError_t e = cudaSuccess;
    if ((n & 1) == 0) e = cudaMemcpyAsync(a, b, h->prob.state_bytes, cudaMemcpyDeviceToDevice, h->stream);
    // publish the loop state where slr_reduce_value reads it
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&ctl->iters, &c.iters, offsetof(Ctl, slot) - offsetof(Ctl, iters),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl->converged, &c.converged, sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "host-driven loop write-back");
    return SLR_OK;
}

}  // namespace

namespace slr {
// Validation and problem set-up shared with entry points in other files.
std::string describe_invalid(const slr_desc *d, bool *unsupported) { return check_desc(d, unsupported); }
// Entry points without a handle report through slr_last_error(NULL).
void set_handleless_error(const std::string &msg) { g_create_error = msg; }
Problem problem_of(const slr_desc *d) { return make_problem(d); }

// slr_create without the autotuner's cache: the descriptor's library-choice
// fields keep the built-in defaults.  The tuner creates its trial handles
// with it.
slr_status create_handle(const slr_desc *d, void *u, const void *aux, void *workspace, size_t workspace_bytes,
                         void *stream, slr_handle *out, bool use_cache)
{
    if (!out) return fail(nullptr, SLR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    bool unsup = false;
    std::string why = check_desc(d, &unsup);
    if (!why.empty()) return fail(nullptr, unsup ? SLR_ERR_UNSUPPORTED : SLR_ERR_INVALID_ARG, why);
    if (!u || ((uintptr_t)u & 15u)) return fail(nullptr, SLR_ERR_INVALID_ARG, "u must be a 16-byte aligned device pointer");
    if (d->stencil != SLR_LIFE && !aux) return fail(nullptr, SLR_ERR_INVALID_ARG, "aux (f or mask) is required");
    if (!workspace || ((uintptr_t)workspace & 255u))
        return fail(nullptr, SLR_ERR_INVALID_ARG, "workspace must be a 256-byte aligned device pointer");
    const size_t need = slr_workspace_size(d);
    if (workspace_bytes < need) {
        char buf[128];
        snprintf(buf, sizeof buf, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
        return fail(nullptr, SLR_ERR_WORKSPACE, buf);
    }
    slr_ctx *h = new (std::nothrow) slr_ctx();
    if (!h) return fail(nullptr, SLR_ERR_INVALID_ARG, "host allocation failed");
    h->desc = *d;
    if (use_cache) tune_fill(&h->desc);
    if (h->desc.loop == SLR_LOOP_AUTO) h->desc.loop = SLR_LOOP_PERSISTENT;
    h->prob = make_problem(&h->desc);
    h->u = u;
    h->aux = aux;
    h->ws = (unsigned char *)workspace;
    h->ws_bytes = workspace_bytes;
    h->stream = (cudaStream_t)stream;
    memset(&h->host_ctl, 0, sizeof(Ctl));
    h->err = "no error";
    cudaError_t e = cudaMemsetAsync(h->ws, 0, sizeof(Ctl), h->stream);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "workspace reset");
        delete h;
        return SLR_ERR_CUDA;
    }
    *out = h;
    return SLR_OK;
}

// The descriptor a handle runs (library-choice fields resolved).
const slr_desc *handle_desc(slr_handle h) { return &h->desc; }
}  // namespace slr

extern "C" {

void slr_desc_init(slr_desc *d, int32_t stencil, int64_t nx, int64_t ny, int64_t nz)
{
    if (!d) return;
    memset(d, 0, sizeof(*d));
    d->stencil = stencil;
    d->nx = nx; d->ny = ny; d->nz = nz;
    d->reduce = reduce_of(stencil);
    d->boundary = stencil == SLR_LIFE ? SLR_WRAP : SLR_DIRICHLET;
    d->storage = stencil == SLR_LIFE ? SLR_U8 : (stencil == SLR_RESTORE8 ? SLR_F32 : SLR_F64);
    d->ghost = 0.0;
    d->tol = stencil == SLR_RESTORE8 ? 1e-3 : 1e-6;
    d->sigma = 1.0;
    d->h = 0.0;
    d->alpha = 100.0f;
    d->loop = SLR_LOOP_AUTO;
    d->math = SLR_MATH_EXACT;
    d->temporal_k = 0;
    d->wait_limit_ns = 0;
}

size_t slr_workspace_size(const slr_desc *d)
{
    bool unsup = false;
    if (!check_desc(d, &unsup).empty()) return 0;
    const Problem p = make_problem(d);
    size_t bytes = slr::kCtlBytes + round_up(p.state_bytes, 256);
    if (p.stencil == SLR_LIFE) bytes += 2 * round_up(slr::life_tb_bits_bytes(p.nx, p.ny), 256);
    if (d->defect_correction) bytes += slr::dc_workspace_bytes(p.nx, p.ny, p.nz);
    if (p.stencil == SLR_RESTORE8) bytes += slr::restore_tb_list_bytes(p.nx, p.ny);
    return bytes;
}

slr_status slr_create(const slr_desc *d, void *u, const void *aux, void *workspace, size_t workspace_bytes,
                      void *stream, slr_handle *out)
{
    return slr::create_handle(d, u, aux, workspace, workspace_bytes, stream, out, true);
}

slr_status slr_run_until(slr_handle h, int64_t max_iters)
{
    if (!h) return fail(nullptr, SLR_ERR_INVALID_ARG, "handle is NULL");
    if (max_iters < 0) return fail(h, SLR_ERR_INVALID_ARG, "max_iters must be >= 0");
    // Life reads any non-zero byte as alive; the temporal-blocked path folds
    // that into its pack phase, the other paths normalise the cells first
    const bool life_tb = h->prob.stencil == SLR_LIFE && h->desc.loop != SLR_LOOP_HOST && h->prob.k != 1 &&
                         slr::life_tb_supported(h->prob);
    if (h->prob.stencil == SLR_LIFE && !life_tb) {
        cudaError_t e = slr::life_normalize(h->prob, h->u, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "normalize cells");
    }
    if (h->desc.loop == SLR_LOOP_HOST) return run_host(h, max_iters);
    return run_persistent(h, max_iters);
}

slr_status slr_reduce_value(slr_handle h, double *value, int64_t *iters, int32_t *converged, uint64_t *count)
{
    if (!h) return fail(nullptr, SLR_ERR_INVALID_ARG, "handle is NULL");
    slr_status s = read_ctl(h);
    if (s != SLR_OK) return s;
    const Ctl &c = h->host_ctl;
    if (value) *value = c.value;
    if (iters) *iters = c.iters;
    if (converged) *converged = c.converged;
    if (count) *count = c.count;
    if (c.err & slr::DEV_ERR_TIMEOUT) return fail(h, SLR_ERR_TIMEOUT, "a device-side grid barrier wait ran out its limit");
    return c.converged ? SLR_OK : SLR_NOT_CONVERGED;
}

slr_status slr_destroy(slr_handle h)
{
    delete h;
    return SLR_OK;
}

const char *slr_last_error(slr_handle h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

const char *slr_version(void)
{
    return "slr 0.1 (sm_103a)";
}

}  // extern "C"
