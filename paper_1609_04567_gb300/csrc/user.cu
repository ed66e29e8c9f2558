// user.cu -- loop-of-stencil-reduce over elemental functions the caller writes.
//
// The pattern of Sec. 3.2 (Fig. 1) takes its stencil and reduce functions from
// the user as source code that the runtime compiles for the device.  Here the
// caller's CUDA C++ defines
//
//   __device__ slr_t  slr_update(const slr_nbr &u, slr_t aux, long long i, long long j, const double *p);
//   __device__ double slr_delta(slr_t new_value, slr_t old_value);
//
// (slr_t = float or double, the state's type; u(di, dj) reads the neighbour at
// offset (di, dj) under the boundary rule; aux is the item's right-hand side
// or 0; p holds up to 8 constants), and the library wraps them in a sweep
// kernel and a fold kernel compiled at run time by NVRTC for sm_103a, without
// floating-point contraction, so every operation the user writes rounds as
// written.  One iteration: the sweep writes u' = slr_update(...) for every item
// into the other state buffer and reduces slr_delta(u', u) per CTA (max or sum,
// in a fixed order), the CTAs' partials are folded in a fixed order, and the
// test (value < tol) decides.  By default the whole loop is one cooperative
// launch with a bounded grid barrier per iteration; the host-driven form (a
// sweep launch, a fold launch and a host read per iteration, the schema of
// Fig. 2) partitions the items the same way and gives the same values.  Compiled programs are cached per
// (source, state type) for the life of the process.
#include <nvrtc.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>

#include "slr_internal.cuh"

struct slr_user_handle_s {
    slr_user_desc d;
    void *u;
    const void *aux;
    unsigned char *b;        // second state buffer
    double *partials;        // one per CTA of the sweep
    double *value;           // the fold's result
    cudaStream_t stream;
    cudaKernel_t sweep, fold, loop;
    int nblocks;
    int cur;                 // buffer holding the current state (0: u, 1: b)
    long long iters;
    double last;
    int converged;
    std::string err;
};

namespace {

constexpr int kUserThreads = 256;
constexpr int kUserMaxBlocks = 1024;
thread_local std::string g_user_error = "no error";

// The generated program around the user's functions.
const char *kPrelude = R"(
struct slr_nbr {
    const slr_t *u;
    long long nx, ny, i, j;
    int wrap;
    slr_t ghost;
    __device__ slr_t operator()(int di, int dj) const
    {
        long long y = i + di, x = j + dj;
        if (wrap) {
            y = ((y % ny) + ny) % ny;
            x = ((x % nx) + nx) % nx;
        } else if (y < 0 || y >= ny || x < 0 || x >= nx) {
            return ghost;
        }
        return u[y * nx + x];
    }
};
)";

const char *kKernels = R"(
// max: identity -inf, a NaN delta is skipped; sum: identity 0
__device__ double slr_combine(double a, double b, int sum) { return sum ? a + b : (b > a ? b : a); }

__device__ double slr_block_reduce(double acc, int sum)
{
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = slr_combine(red[threadIdx.x], red[threadIdx.x + s], sum);
        __syncthreads();
    }
    return red[0];
}

extern "C" __global__ void __launch_bounds__(256) slr_user_sweep(const slr_t *u, slr_t *v, const slr_t *aux,
    long long nx, long long ny, int wrap, slr_t ghost, int sum, const double *p0, double *partials)
{
    double p[8];
    for (int k = 0; k < 8; ++k) p[k] = p0[k];
    double acc = sum ? 0.0 : __longlong_as_double(0xfff0000000000000ll);
    const long long n = nx * ny;
    for (long long c = (long long)blockIdx.x * 256 + threadIdx.x; c < n; c += (long long)gridDim.x * 256) {
        const long long i = c / nx, j = c - i * nx;
        slr_nbr nb;
        nb.u = u; nb.nx = nx; nb.ny = ny; nb.i = i; nb.j = j; nb.wrap = wrap; nb.ghost = ghost;
        const slr_t nv = slr_update(nb, aux ? aux[c] : (slr_t)0, i, j, p);
        acc = slr_combine(acc, slr_delta(nv, u[c]), sum);
        v[c] = nv;
    }
    const double r = slr_block_reduce(acc, sum);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

extern "C" __global__ void __launch_bounds__(256) slr_user_fold(const double *partials, int nb, int sum,
                                                                double *out)
{
    double acc = sum ? 0.0 : __longlong_as_double(0xfff0000000000000ll);
    for (int k = threadIdx.x; k < nb; k += 256) acc = slr_combine(acc, partials[k], sum);
    const double r = slr_block_reduce(acc, sum);
    if (threadIdx.x == 0) out[0] = r;
}

struct slr_user_ctl {
    unsigned long long bar;    // grid barrier arrivals (zeroed before every launch)
    long long iters;
    double value;
    int converged;
    int err;
};

// The whole loop in one cooperative launch (at most one CTA per SM): the same
// sweep and per-CTA partials as slr_user_sweep, a bounded grid barrier, then
// every CTA folds the partials in the same fixed order (the same value as
// slr_user_fold) and applies the test, so all CTAs stop together.
extern "C" __global__ void __launch_bounds__(256) slr_user_loop(slr_t *ua, slr_t *ub, const slr_t *aux,
    long long nx, long long ny, int wrap, slr_t ghost, int sum, const double *p0, double *partials,
    slr_user_ctl *ctl, long long max_iters, double tol, long long limit_ns)
{
    __shared__ int s_ok;
    double p[8];
    for (int k = 0; k < 8; ++k) p[k] = p0[k];
    const long long it0 = ctl->iters;
    if (ctl->converged || it0 >= max_iters || ctl->err) return;
    const long long n = nx * ny;
    const double ident = sum ? 0.0 : __longlong_as_double(0xfff0000000000000ll);
    long long k = 0;
    for (;; ++k) {
        const slr_t *src = (k & 1) ? ub : ua;
        slr_t *dst = (k & 1) ? ua : ub;
        double acc = ident;
        for (long long c = (long long)blockIdx.x * 256 + threadIdx.x; c < n; c += (long long)gridDim.x * 256) {
            const long long i = c / nx, j = c - i * nx;
            slr_nbr nb;
            nb.u = src; nb.nx = nx; nb.ny = ny; nb.i = i; nb.j = j; nb.wrap = wrap; nb.ghost = ghost;
            const slr_t nv = slr_update(nb, aux ? aux[c] : (slr_t)0, i, j, p);
            acc = slr_combine(acc, slr_delta(nv, src[c]), sum);
            dst[c] = nv;
        }
        double *part = partials + (k & 1) * 1024;      // alternate: read while the next sweep writes
        const double r = slr_block_reduce(acc, sum);
        if (threadIdx.x == 0) part[blockIdx.x] = r;
        // bounded grid barrier
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            __threadfence();
            asm volatile("red.release.gpu.global.add.u64 [%0], 1;" :: "l"(&ctl->bar) : "memory");
            const unsigned long long target = (unsigned long long)(k + 1) * gridDim.x;
            long long t0;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            for (unsigned spins = 0;; ++spins) {
                unsigned long long v;
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(&ctl->bar) : "memory");
                if (v >= target) break;
                if ((spins & 15u) == 15u) {
                    long long t;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                    if (*(volatile int *)&ctl->err || t - t0 > limit_ns) {
                        atomicOr(&ctl->err, 1);
                        ok = 0;
                        break;
                    }
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        double acc2 = ident;
        for (int t = threadIdx.x; t < (int)gridDim.x; t += 256) acc2 = slr_combine(acc2, __ldcg(part + t), sum);
        const double v = slr_block_reduce(acc2, sum);
        const long long it = it0 + k + 1;
        const int conv = v < tol;
        if (conv || it >= max_iters) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                ctl->iters = it;
                ctl->value = v;
                ctl->converged = conv;
            }
            break;
        }
        __syncthreads();                                // red[] is free before the next sweep reduces
    }
    // the caller's buffer receives the state (every CTA's writes are behind the last barrier)
    if ((k & 1) == 0)
        for (long long c = (long long)blockIdx.x * 256 + threadIdx.x; c < n; c += (long long)gridDim.x * 256)
            ua[c] = __ldcg(ub + c);
}
)";

struct Compiled {
    cudaLibrary_t lib;
    cudaKernel_t sweep, fold, loop;
};

std::mutex g_mu;
std::map<std::pair<int, std::string>, Compiled> g_cache;

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

size_t elem_of(int dtype) { return dtype == SLR_F32 ? 4 : (dtype == SLR_F64 ? 8 : 0); }

// CTAs of both loops (the same partition of the items, so the same partial
// sums): at most one per SM, so the cooperative launch is always co-resident
int blocks_of(const slr_user_desc *d)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        sms = 1;
    }
    const long long cells = d->nx * d->ny;
    long long b = (cells + kUserThreads - 1) / kUserThreads;
    if (b > sms) b = sms;
    return (int)(b < kUserMaxBlocks ? b : kUserMaxBlocks);
}

std::string check(const slr_user_desc *d)
{
    if (!d) return "descriptor is NULL";
    if (d->dtype != SLR_F32 && d->dtype != SLR_F64) return "dtype must be SLR_F32 or SLR_F64";
    if (d->nx < 1 || d->ny < 1 || d->nx > (1ll << 40) / d->ny) return "nx, ny must be >= 1 (and nx * ny < 2^40)";
    if (d->boundary != SLR_DIRICHLET && d->boundary != SLR_WRAP) return "boundary must be SLR_DIRICHLET or SLR_WRAP";
    if (d->reduce != SLR_USER_MAX && d->reduce != SLR_USER_SUM) return "reduce must be SLR_USER_MAX or SLR_USER_SUM";
    if (d->loop != SLR_LOOP_AUTO && d->loop != SLR_LOOP_HOST && d->loop != SLR_LOOP_PERSISTENT)
        return "loop must be a slr_loop value";
    return "";
}

slr_status fail(slr_user_handle h, slr_status s, const std::string &msg)
{
    if (h) h->err = msg; else g_user_error = msg;
    return s;
}

// Compile (or find) the program for (dtype, source).
slr_status compile(int dtype, const char *source, Compiled *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    const auto key = std::make_pair(dtype, std::string(source));
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *out = it->second;
        return SLR_OK;
    }
    std::string prog = std::string("typedef ") + (dtype == SLR_F32 ? "float" : "double") + " slr_t;\n" + kPrelude +
                       "#line 1 \"user\"\n" + source + "\n#line 1 \"slr_kernels\"\n" + kKernels;
    nvrtcProgram p;
    if (nvrtcCreateProgram(&p, prog.c_str(), "slr_user.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return fail(nullptr, SLR_ERR_CUDA, "slr_user_create: nvrtcCreateProgram failed");
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "--fmad=false", "-default-device"};
    const nvrtcResult cr = nvrtcCompileProgram(p, 4, opts);
    if (cr != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(p, &n);
        std::string log(n, '\0');
        if (n) nvrtcGetProgramLog(p, &log[0]);
        nvrtcDestroyProgram(&p);
        return fail(nullptr, SLR_ERR_INVALID_ARG, std::string("slr_user_create: the source does not compile:\n") + log);
    }
    size_t n = 0;
    nvrtcGetCUBINSize(p, &n);
    std::string cubin(n, '\0');
    nvrtcGetCUBIN(p, &cubin[0]);
    nvrtcDestroyProgram(&p);
    Compiled c;
    cudaError_t e = cudaLibraryLoadData(&c.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&c.sweep, c.lib, "slr_user_sweep");
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&c.fold, c.lib, "slr_user_fold");
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&c.loop, c.lib, "slr_user_loop");
    if (e != cudaSuccess)
        return fail(nullptr, SLR_ERR_CUDA, std::string("slr_user_create: load: ") + cudaGetErrorString(e));
    g_cache[key] = c;
    *out = c;
    return SLR_OK;
}

}  // namespace

extern "C" {

size_t slr_user_workspace_size(const slr_user_desc *d)
{
    if (!check(d).empty()) return 0;
    return round256((size_t)(d->nx * d->ny) * elem_of(d->dtype)) + round256(2 * kUserMaxBlocks * 8 + 18 * 8) + 256;
}

slr_status slr_user_create(const slr_user_desc *d, const char *source, void *u, const void *aux, void *workspace,
                           size_t workspace_bytes, void *stream, slr_user_handle *out)
{
    if (!out) return fail(nullptr, SLR_ERR_INVALID_ARG, "slr_user_create: out is NULL");
    *out = nullptr;
    const std::string why = check(d);
    if (!why.empty()) return fail(nullptr, SLR_ERR_INVALID_ARG, "slr_user_create: " + why);
    if (!source) return fail(nullptr, SLR_ERR_INVALID_ARG, "slr_user_create: source is NULL");
    if (!u || (uintptr_t)u % elem_of(d->dtype) != 0 || (aux && (uintptr_t)aux % elem_of(d->dtype) != 0))
        return fail(nullptr, SLR_ERR_INVALID_ARG, "slr_user_create: u (and aux) must be aligned device pointers");
    if (!workspace || (uintptr_t)workspace % 256 != 0)
        return fail(nullptr, SLR_ERR_INVALID_ARG, "slr_user_create: workspace must be 256-byte aligned");
    if (workspace_bytes < slr_user_workspace_size(d))
        return fail(nullptr, SLR_ERR_WORKSPACE, "slr_user_create: workspace smaller than slr_user_workspace_size()");
    Compiled c;
    const slr_status s = compile(d->dtype, source, &c);
    if (s != SLR_OK) return s;
    slr_user_handle h = new (std::nothrow) slr_user_handle_s();
    if (!h) return fail(nullptr, SLR_ERR_CUDA, "slr_user_create: out of host memory");
    h->d = *d;
    h->u = u;
    h->aux = aux;
    h->b = (unsigned char *)workspace;
    h->partials = (double *)(h->b + round256((size_t)(d->nx * d->ny) * elem_of(d->dtype)));
    h->value = h->partials + 2 * kUserMaxBlocks;      // value, 8 constants, the device loop's control
    h->loop = c.loop;
    h->stream = (cudaStream_t)stream;
    h->sweep = c.sweep;
    h->fold = c.fold;
    h->nblocks = blocks_of(d);
    h->cur = 0;
    h->iters = 0;
    h->last = 0.0;
    h->converged = 0;
    cudaError_t e = cudaMemcpyAsync(h->value + 1, d->params, sizeof d->params, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->value + 9, 0, 32, h->stream);     // device loop control
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, SLR_ERR_CUDA, std::string("slr_user_create: ") + cudaGetErrorString(e));
    }
    *out = h;
    return SLR_OK;
}

namespace {
// the device loop: one cooperative launch, then one read of its control block
slr_status run_device(slr_user_handle h, int64_t max_iters)
{
    if (h->converged || h->iters >= max_iters) return h->converged ? SLR_OK : SLR_NOT_CONVERGED;
    struct Ctl {
        unsigned long long bar;
        long long iters;
        double value;
        int converged, err;
    };
    Ctl *ctl = (Ctl *)(h->value + 9);
    void *ua = h->u, *ub = h->b;
    const void *aux = h->aux;
    long long nx = h->d.nx, ny = h->d.ny, mi = max_iters;
    long long limit = 2000000000ll;
    const int sum = h->d.reduce == SLR_USER_SUM, wrap = h->d.boundary == SLR_WRAP;
    const float gf = (float)h->d.ghost;
    const double gd = h->d.ghost, tol = h->d.tol;
    const double *params = h->value + 1;
    void *args[] = {&ua, &ub, (void *)&aux, &nx, &ny, (void *)&wrap,
                    h->d.dtype == SLR_F32 ? (void *)&gf : (void *)&gd, (void *)&sum, (void *)&params,
                    &h->partials, &ctl, &mi, (void *)&tol, &limit};
    cudaError_t e = cudaMemsetAsync(&ctl->bar, 0, sizeof ctl->bar, h->stream);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void *)h->loop, dim3(h->nblocks), dim3(kUserThreads), args, 0,
                                        h->stream);
    Ctl host;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, ctl, sizeof host, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, SLR_ERR_CUDA, std::string("slr_user_run_until: ") + cudaGetErrorString(e));
    if (host.err) return fail(h, SLR_ERR_TIMEOUT, "slr_user_run_until: a grid barrier wait ran out its limit");
    h->iters = host.iters;
    h->last = host.value;
    h->converged = host.converged;
    return h->converged ? SLR_OK : SLR_NOT_CONVERGED;
}
}  // namespace

slr_status slr_user_run_until(slr_user_handle h, int64_t max_iters)
{
    if (!h) return fail(nullptr, SLR_ERR_INVALID_ARG, "slr_user_run_until: handle is NULL");
    if (h->d.loop != SLR_LOOP_HOST) return run_device(h, max_iters);
    const size_t bytes = (size_t)(h->d.nx * h->d.ny) * elem_of(h->d.dtype);
    const int sum = h->d.reduce == SLR_USER_SUM;
    const int wrap = h->d.boundary == SLR_WRAP;
    const float gf = (float)h->d.ghost;
    const double gd = h->d.ghost;
    long long nx = h->d.nx, ny = h->d.ny;
    const double *params = h->value + 1;
    while (!h->converged && h->iters < max_iters) {
        void *src = h->cur == 0 ? h->u : (void *)h->b;
        void *dst = h->cur == 0 ? (void *)h->b : h->u;
        const void *aux = h->aux;
        void *args[] = {&src, &dst, (void *)&aux, &nx, &ny, (void *)&wrap,
                        h->d.dtype == SLR_F32 ? (void *)&gf : (void *)&gd, (void *)&sum, (void *)&params,
                        &h->partials};
        cudaError_t e = cudaLaunchKernel((const void *)h->sweep, dim3(h->nblocks), dim3(kUserThreads), args, 0,
                                         h->stream);
        int nb = h->nblocks;
        void *fargs[] = {&h->partials, &nb, (void *)&sum, &h->value};
        if (e == cudaSuccess) e = cudaLaunchKernel((const void *)h->fold, dim3(1), dim3(kUserThreads), fargs, 0, h->stream);
        double v = 0.0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&v, h->value, sizeof v, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return fail(h, SLR_ERR_CUDA, std::string("slr_user_run_until: ") + cudaGetErrorString(e));
        h->cur ^= 1;
        h->iters += 1;
        h->last = v;
        h->converged = v < h->d.tol;
    }
    if (h->cur == 1) {
        // the caller's buffer receives the state
        cudaError_t e = cudaMemcpyAsync(h->u, h->b, bytes, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return fail(h, SLR_ERR_CUDA, std::string("slr_user_run_until: ") + cudaGetErrorString(e));
        h->cur = 0;
    }
    return h->converged ? SLR_OK : SLR_NOT_CONVERGED;
}

slr_status slr_user_reduce_value(slr_user_handle h, double *value, int64_t *iters, int32_t *converged)
{
    if (!h) return fail(nullptr, SLR_ERR_INVALID_ARG, "slr_user_reduce_value: handle is NULL");
    if (value) *value = h->last;
    if (iters) *iters = h->iters;
    if (converged) *converged = h->converged;
    return h->converged ? SLR_OK : SLR_NOT_CONVERGED;
}

slr_status slr_user_destroy(slr_user_handle h)
{
    delete h;
    return SLR_OK;
}

const char *slr_user_last_error(slr_user_handle h) { return h ? h->err.c_str() : g_user_error.c_str(); }

}  // extern "C"
