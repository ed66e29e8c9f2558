// tune.cu -- the autotuner.  The paper picks its work-group layout with fixed
// heuristics (Sec. 3.3); here the launch choices that leave results unchanged
// (loop driver, sweeps per HBM pass of Life, the 2D Jacobi and the
// restoration, the one-sweep kernels' tiling and the persistent grid size) are
// timed on the caller's own data and the
// fastest is kept in a process-wide cache that slr_create consults.
//
// Search: stage 1 times loop x temporal_k x tiling with all co-resident CTAs
// (the library default first), stage 2 times grid sizes for the stage-1
// winner.  Each candidate runs from a fresh copy of u in the caller's scratch,
// once untimed and twice timed with CUDA events on the caller's stream; its
// score is the shorter time per iteration.  A candidate must beat the best so
// far by more than 1% to replace it.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "jacobi_tb.h"
#include "slr_internal.cuh"

namespace {

struct Key {
    int dev, sms, stencil, storage, boundary, math, dc, bucket;
    long long nx, ny, nz;
    bool operator<(const Key &o) const
    {
        return std::tie(dev, sms, stencil, storage, boundary, math, dc, bucket, nx, ny, nz) <
               std::tie(o.dev, o.sms, o.stencil, o.storage, o.boundary, o.math, o.dc, o.bucket, o.nx, o.ny, o.nz);
    }
};

std::mutex g_mu;
std::map<Key, slr_tune_result> g_cache;
thread_local std::string g_tune_error = "no error";

long long floor_log2(long long v)
{
    long long b = 0;
    while (v > 1) { v >>= 1; ++b; }
    return b;
}

bool make_key(const slr_desc *d, bool bucket, Key *k)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    k->dev = dev;
    k->sms = sms;
    k->stencil = d->stencil;
    k->storage = d->storage;
    k->boundary = d->boundary;
    k->math = d->math;
    k->dc = d->defect_correction != 0;
    k->bucket = bucket;
    k->nx = bucket ? floor_log2(d->nx) : d->nx;
    k->ny = bucket ? floor_log2(d->ny) : d->ny;
    k->nz = bucket ? floor_log2(d->nz) : d->nz;
    return true;
}

// Cached choice for d: exact key, else the bucket key.  Caller holds g_mu.
bool lookup_locked(const slr_desc *d, slr_tune_result *out)
{
    if (g_cache.empty()) return false;
    Key k;
    for (int bucket = 0; bucket < 2; ++bucket) {
        if (!make_key(d, bucket != 0, &k)) return false;
        auto it = g_cache.find(k);
        if (it != g_cache.end()) {
            *out = it->second;
            return true;
        }
    }
    return false;
}

slr_status tune_fail(slr_status s, const std::string &msg)
{
    g_tune_error = msg;
    return s;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

struct Timer {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Timer()
    {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

struct Bench {
    const void *u;
    const void *aux;
    unsigned char *state;      // copy of u the trials run on
    unsigned char *ws;         // trial workspace
    size_t state_bytes, ws_bytes;
    cudaStream_t st;
    int64_t iters;
    Timer t;
    int trials = 0;
};

// Score of one candidate (ms per iteration), or an error status.
slr_status score(Bench &b, const slr_desc &d, double *ms_per_iter)
{
    double best = INFINITY;
    for (int rep = 0; rep < 3; ++rep) {
        cudaError_t e = cudaMemcpyAsync(b.state, b.u, b.state_bytes, cudaMemcpyDeviceToDevice, b.st);
        if (e != cudaSuccess) return tune_fail(SLR_ERR_CUDA, std::string("trial copy: ") + cudaGetErrorString(e));
        slr_handle h = nullptr;
        slr_status s = slr::create_handle(&d, b.state, b.aux, b.ws, b.ws_bytes, b.st, &h, false);
        if (s != SLR_OK) return tune_fail(s, std::string("trial create: ") + slr_last_error(nullptr));
        e = cudaEventRecord(b.t.e0, b.st);
        if (e == cudaSuccess) s = slr_run_until(h, b.iters);
        if (e == cudaSuccess && s >= 0) e = cudaEventRecord(b.t.e1, b.st);
        int64_t it = 0;
        if (e == cudaSuccess && s >= 0) s = slr_reduce_value(h, nullptr, &it, nullptr, nullptr);
        float ms = 0.0f;
        if (e == cudaSuccess && s >= 0) e = cudaEventElapsedTime(&ms, b.t.e0, b.t.e1);
        if (s < 0) {
            std::string m = std::string("trial run: ") + slr_last_error(h);
            slr_destroy(h);
            return tune_fail(s, m);
        }
        slr_destroy(h);
        if (e != cudaSuccess) return tune_fail(SLR_ERR_CUDA, std::string("trial timing: ") + cudaGetErrorString(e));
        if (rep > 0 && it > 0) best = fmin(best, (double)ms / (double)it);
    }
    b.trials += 1;
    *ms_per_iter = best;
    return SLR_OK;
}

}  // namespace

namespace slr {
void tune_fill(slr_desc *d)
{
    std::lock_guard<std::mutex> lk(g_mu);
    slr_tune_result r;
    if (!lookup_locked(d, &r)) return;
    if (d->loop == SLR_LOOP_AUTO) d->loop = r.loop;
    const bool blocked = d->stencil == SLR_LIFE || d->stencil == SLR_RESTORE8 ||
                         (d->stencil == SLR_J2D5 && !d->defect_correction);
    if (d->temporal_k == 0 && blocked) d->temporal_k = r.temporal_k;
    if (d->tiling == SLR_TILING_AUTO && d->stencil != SLR_LIFE) d->tiling = r.tiling;
    // the grid size was timed with the kernel of the cached choice only
    const bool same_kernel = d->loop == r.loop && (!blocked || d->temporal_k == r.temporal_k) &&
                             (d->stencil == SLR_LIFE || d->tiling == r.tiling);
    if (d->grid_ctas == 0 && same_kernel) d->grid_ctas = r.grid_ctas;
}
}  // namespace slr

extern "C" {

size_t slr_tune_scratch_size(const slr_desc *d)
{
    const size_t ws = slr_workspace_size(d);
    if (ws == 0) return 0;
    return round256(slr::problem_of(d).state_bytes) + ws;
}

slr_status slr_tune(const slr_desc *d, const void *u, const void *aux, void *scratch, size_t scratch_bytes,
                    void *stream, int64_t trial_iters, slr_tune_result *out)
{
    bool unsup = false;
    std::string why = slr::describe_invalid(d, &unsup);
    if (!why.empty()) return tune_fail(unsup ? SLR_ERR_UNSUPPORTED : SLR_ERR_INVALID_ARG, why);
    if (!u || ((uintptr_t)u & 15u)) return tune_fail(SLR_ERR_INVALID_ARG, "u must be a 16-byte aligned device pointer");
    if (d->stencil != SLR_LIFE && !aux) return tune_fail(SLR_ERR_INVALID_ARG, "aux (f or mask) is required");
    if (!scratch || ((uintptr_t)scratch & 255u))
        return tune_fail(SLR_ERR_INVALID_ARG, "scratch must be a 256-byte aligned device pointer");
    const size_t need = slr_tune_scratch_size(d);
    if (scratch_bytes < need) {
        char buf[128];
        snprintf(buf, sizeof buf, "scratch too small: %zu < %zu bytes", scratch_bytes, need);
        return tune_fail(SLR_ERR_WORKSPACE, buf);
    }
    const slr::Problem p = slr::problem_of(d);
    Bench b;
    b.u = u;
    b.aux = aux;
    b.state = (unsigned char *)scratch;
    b.state_bytes = p.state_bytes;
    b.ws = (unsigned char *)scratch + round256(p.state_bytes);
    b.ws_bytes = scratch_bytes - round256(p.state_bytes);
    b.st = (cudaStream_t)stream;
    b.iters = trial_iters > 0 ? trial_iters : (d->defect_correction ? 4 : 64);
    int sms = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaEventCreate(&b.t.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&b.t.e1);
    if (e != cudaSuccess) return tune_fail(SLR_ERR_CUDA, std::string("tuner set-up: ") + cudaGetErrorString(e));

    // The library default: explicit fields as given, the rest at built-in
    // defaults; the convergence test is disabled so every trial runs the
    // same number of sweeps (Life still stops at a still state).
    slr_desc base = *d;
    base.tol = -1.0;
    if (base.loop == SLR_LOOP_AUTO) base.loop = SLR_LOOP_PERSISTENT;
    const bool persistent = base.loop == SLR_LOOP_PERSISTENT;
    const bool life_tb = d->stencil == SLR_LIFE && slr::life_tb_supported(p);
    const bool jacobi = (d->stencil == SLR_J2D5 || d->stencil == SLR_J3D7) && !d->defect_correction;
    // the trial buffers stand in for the caller's (same alignment: 256 bytes)
    const void *ta = b.state, *tb = b.ws + slr::kCtlBytes;
    const bool tma = (d->stencil == SLR_RESTORE8 && slr::restore_tma_ok(p)) ||
                     (jacobi && slr::jacobi_tma_ok(p, ta, tb, aux, true));

    const bool jacobi_tb = jacobi && slr::jacobi_tb_supported(p, ta, tb, aux);
    const bool restore_tb = d->stencil == SLR_RESTORE8 && slr::restore_tb_supported(p, ta, tb, aux);

    // What the default resolves to, so that equal configurations are timed once.
    auto resolved_k = [&](const slr_desc &c) {
        if (c.loop == SLR_LOOP_HOST) return 1;
        if (life_tb) return slr::life_tb_resolve_k(slr::problem_of(&c), c.grid_ctas);
        if (jacobi_tb) return slr::jacobi_tb_resolve_k(slr::problem_of(&c), ta, tb, aux);
        if (restore_tb) return slr::restore_tb_resolve_k(slr::problem_of(&c), ta, tb, aux);
        return 1;
    };
    auto resolved_tiling = [&](const slr_desc &c) {
        if (c.loop != SLR_LOOP_PERSISTENT || !tma || c.tiling == SLR_TILING_NONE) return (int)SLR_TILING_NONE;
        if (jacobi && c.tiling == SLR_TILING_AUTO)   // the size rule of the library default
            return slr::jacobi_tma_ok(slr::problem_of(&c), ta, tb, aux, false) ? (int)SLR_TILING_TMA
                                                                                 : (int)SLR_TILING_NONE;
        return (int)SLR_TILING_TMA;
    };

    std::vector<slr_desc> stage1;
    stage1.push_back(base);
    if (persistent && d->stencil == SLR_LIFE && d->temporal_k == 0) {
        const int def_k = resolved_k(base);
        static const int ks[] = {1, 2, 4, 6, 8, 10, 12, 14, 16, 20, 24, 32};
        for (int k : ks) {
            if (k == def_k || (k > 1 && !life_tb)) continue;
            slr_desc c = base;
            c.temporal_k = k;
            stage1.push_back(c);
        }
    }
    if (persistent && jacobi_tb && d->temporal_k == 0) {
        // sweeps per pass of the Jacobi: one (the one-sweep kernels), 4, 8 in
        // 2D; one, 2, 4 in 3D
        const int def_k = resolved_k(base);
        static const int ks2[] = {1, 4, 8}, ks3[] = {1, 2, 4};
        for (int k : (d->stencil == SLR_J3D7 ? ks3 : ks2)) {
            if (k == def_k) continue;
            slr_desc c = base;
            c.temporal_k = k;
            stage1.push_back(c);
        }
    }
    if (persistent && restore_tb && d->temporal_k == 0) {
        // sweeps per pass of the restoration: one (the one-sweep kernels), 2, 4, 8
        const int def_k = resolved_k(base);
        static const int ks[] = {1, 2, 4, 8};
        for (int k : ks) {
            if (k == def_k) continue;
            slr_desc c = base;
            c.temporal_k = k;
            stage1.push_back(c);
        }
    }
    if (persistent && (d->stencil == SLR_RESTORE8 || jacobi) && d->tiling == SLR_TILING_AUTO && tma) {
        // the other staging than the default's
        slr_desc c = base;
        c.tiling = resolved_tiling(base) == SLR_TILING_TMA ? SLR_TILING_NONE : SLR_TILING_TMA;
        stage1.push_back(c);
    }
    if (d->loop == SLR_LOOP_AUTO && !d->defect_correction) {
        slr_desc c = base;
        c.loop = SLR_LOOP_HOST;
        stage1.push_back(c);
    }

    double def_ms = 0.0, best_ms = INFINITY;
    slr_desc best = base;
    for (size_t i = 0; i < stage1.size(); ++i) {
        double ms = 0.0;
        slr_status s = score(b, stage1[i], &ms);
        if (s != SLR_OK) return s;
        if (i == 0) def_ms = ms;
        if (ms < 0.99 * best_ms) {
            best_ms = ms;
            best = stage1[i];
        }
    }
    if (best.loop == SLR_LOOP_PERSISTENT && d->grid_ctas == 0) {
        // fix the stage-1 choice of k before shrinking the grid (the default
        // k depends on the grid size)
        if ((d->stencil == SLR_LIFE || jacobi_tb || restore_tb) && best.temporal_k == 0)
            best.temporal_k = resolved_k(best);
        const int grids[] = {2 * sms, sms, sms / 2, sms / 4, sms / 8, sms / 16};
        int last = -1;
        for (int g : grids) {
            if (g < 1 || g == last) continue;
            last = g;
            slr_desc c = best;
            c.grid_ctas = g;
            double ms = 0.0;
            slr_status s = score(b, c, &ms);
            if (s != SLR_OK) return s;
            if (ms < 0.99 * best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    }

    slr_tune_result r;
    memset(&r, 0, sizeof(r));
    r.loop = best.loop;
    r.temporal_k = d->stencil == SLR_LIFE || d->stencil == SLR_RESTORE8 || (jacobi && d->stencil == SLR_J2D5)
                       ? resolved_k(best)
                       : 0;
    r.tiling = d->stencil == SLR_RESTORE8 || jacobi ? resolved_tiling(best) : SLR_TILING_AUTO;
    r.grid_ctas = best.loop == SLR_LOOP_PERSISTENT ? best.grid_ctas : 0;
    r.trials = b.trials;
    r.ms_per_iter = best_ms;
    r.default_ms_per_iter = def_ms;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        Key k;
        if (make_key(d, false, &k)) g_cache[k] = r;
        if (make_key(d, true, &k)) g_cache[k] = r;
    }
    if (out) *out = r;
    return SLR_OK;
}

int32_t slr_tune_lookup(const slr_desc *d, slr_tune_result *out)
{
    if (!d) return 0;
    std::lock_guard<std::mutex> lk(g_mu);
    slr_tune_result r;
    if (!lookup_locked(d, &r)) return 0;
    if (out) *out = r;
    return 1;
}

void slr_tune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache.clear();
}

const char *slr_tune_last_error(void) { return g_tune_error.c_str(); }

}  // extern "C"
