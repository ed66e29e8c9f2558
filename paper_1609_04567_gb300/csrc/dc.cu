// dc.cu -- FP64 defect correction around FP32 Jacobi inner solves (2D
// 5-point and 3D 7-point Helmholtz, Dirichlet ghost 0), as one persistent
// launch.
//
// The loop of Sec. 3.1 whose elemental step is one correction: with
// A u = ((2n + sigma h^2) u - sum of neighbours) / h^2 and r = f - A u,
//     e = 0;  inner_sweeps binary32 Jacobi sweeps  e' = (h2 r32 + sum of e's neighbours) / d
//     u' = u + (double) e;   r' = f - A u'  (binary64);   rho = max |h2 r' / d|
// neighbours summed ((N + S) + W) + E in 2D, x-, x+, y-, y+, z-, z+ in 3D.
// until rho < tol or the cap.  FP64 arithmetic is used only for the update,
// the defect and its reduce; the inner solves run in binary32.
//
// Buffers: u (caller, binary64) and one binary64 workspace buffer ping-pong
// across corrections; r32 and two e buffers are binary32.  The correction pass
// reads u_old and e and writes u_new, so the neighbours of u_new are formed as
// u_old + e on the fly (the same binary64 operation as updating first), with
// no barrier between the update and the defect.  Every operation is IEEE
// rounded in the oracle's order (no contraction), so results are bit-exact.
#include "slr_internal.cuh"

namespace slr {
namespace {

constexpr int kDThreads = 1024;

__device__ __forceinline__ double add_rn(double x, double y) { return __dadd_rn(x, y); }
__device__ __forceinline__ float add_rn(float x, float y) { return __fadd_rn(x, y); }

struct DcArgs {
    double *u;          // caller state (A)
    double *ub;         // workspace state (B)
    const double *f;
    float *r32;
    float *e[2];
    long long nx, ny, nz;
    double h2, d;
    float h2f, df;
    int inner;
};

// Grid-stride over cells by (plane, row, 1024-column chunk) units.
template <class F>
__device__ __forceinline__ void for_cells(long long nx, long long ny, long long nz, F fn)
{
    const long long chunks = (nx + blockDim.x - 1) / blockDim.x;
    const long long units = nz * ny * chunks;
    for (long long un = blockIdx.x; un < units; un += gridDim.x) {
        const long long row = un / chunks;
        const long long j = (un - row * chunks) * blockDim.x + threadIdx.x;
        if (j < nx) fn(row / ny, row % ny, j);
    }
}

__device__ __forceinline__ bool outside(const DcArgs &a, long long k, long long i, long long j)
{
    return k < 0 || k >= a.nz || i < 0 || i >= a.ny || j < 0 || j >= a.nx;
}

__device__ __forceinline__ long long cell(const DcArgs &a, long long k, long long i, long long j)
{
    return (k * a.ny + i) * a.nx + j;
}

// the sum of the neighbours of (k, i, j) read through `val`, in the oracle's order
template <int DIM, class T, class V>
__device__ __forceinline__ T nbr_sum(long long k, long long i, long long j, V val)
{
    if (DIM == 2)
        return add_rn(add_rn(add_rn(val(k, i - 1, j), val(k, i + 1, j)), val(k, i, j - 1)), val(k, i, j + 1));
    return add_rn(add_rn(add_rn(add_rn(add_rn(val(k, i, j - 1), val(k, i, j + 1)), val(k, i - 1, j)), val(k, i + 1, j)),
                         val(k - 1, i, j)),
                  val(k + 1, i, j));
}

// r = f - A v with v read through `val` (ghost 0); returns r (binary64)
template <int DIM, class V>
__device__ __forceinline__ double defect_at(const DcArgs &a, long long k, long long i, long long j, V val)
{
    const double s = nbr_sum<DIM, double>(k, i, j, val);
    const double au = __ddiv_rn(__dsub_rn(__dmul_rn(a.d, val(k, i, j)), s), a.h2);
    return __dsub_rn(__ldg(a.f + cell(a, k, i, j)), au);
}

template <int DIM>
__global__ void __launch_bounds__(kDThreads, 1) dc_kernel(DcArgs a, LoopArgs la)
{
    __shared__ int s_stop;
    Ctl *ctl = la.ctl;
    const long long it0 = ctl->iters;
    if (ctl->converged || it0 >= la.max_iters || ctl->err) return;
    if ((la.debug_flags & SLR_DEBUG_SKIP_ARRIVAL) && blockIdx.x == gridDim.x - 1) return;
    unsigned long long bar = 0;
    // initial defect of the caller's state
    for_cells(a.nx, a.ny, a.nz, [&](long long k, long long i, long long j) {
        const double r = defect_at<DIM>(a, k, i, j, [&](long long z, long long y, long long x) {
            return outside(a, z, y, x) ? 0.0 : __ldcg(a.u + cell(a, z, y, x));
        });
        a.r32[cell(a, k, i, j)] = (float)r;
    });
    bar += la.nblocks;
    if (!grid_barrier(ctl, bar, la.limit_ns)) return;
    for (long long n = 0;; ++n) {
        const double *uo = (n & 1) ? a.ub : a.u;
        double *un = (n & 1) ? a.u : a.ub;
        // inner binary32 Jacobi sweeps from e = 0
        for (int m = 0; m < a.inner; ++m) {
            const float *es = a.e[m & 1];
            float *ed = a.e[(m + 1) & 1];
            const bool zero = m == 0;
            for_cells(a.nx, a.ny, a.nz, [&](long long k, long long i, long long j) {
                float sn = 0.0f;
                if (!zero)
                    sn = nbr_sum<DIM, float>(k, i, j, [&](long long z, long long y, long long x) {
                        return outside(a, z, y, x) ? 0.0f : __ldcg(es + cell(a, z, y, x));
                    });
                const long long c = cell(a, k, i, j);
                const float t = __fmul_rn(a.h2f, __ldcg(a.r32 + c));
                ed[c] = __fdiv_rn(__fadd_rn(t, sn), a.df);
            });
            bar += la.nblocks;
            if (!grid_barrier(ctl, bar, la.limit_ns)) return;
        }
        // correction and new defect in one pass
        const float *e = a.e[a.inner & 1];
        unsigned long long mx = 0ull;
        for_cells(a.nx, a.ny, a.nz, [&](long long k, long long i, long long j) {
            const long long c = cell(a, k, i, j);
            const double unew = __dadd_rn(__ldcg(uo + c), (double)__ldcg(e + c));
            un[c] = unew;
            // u_old + e at each neighbour, the ghost 0 outside the grid
            const double r = defect_at<DIM>(a, k, i, j, [&](long long z, long long y, long long x) {
                if (outside(a, z, y, x)) return 0.0;
                const long long q = cell(a, z, y, x);
                return __dadd_rn(__ldcg(uo + q), (double)__ldcg(e + q));
            });
            a.r32[c] = (float)r;
            const unsigned long long b =
                (unsigned long long)__double_as_longlong(fabs(__ddiv_rn(__dmul_rn(a.h2, r), a.d)));
            mx = b > mx ? b : mx;
        });
        block_to_slot(&ctl->slot[n % kSlots], mx, 0ull, 0ull, 1u);
        bar += la.nblocks;
        if (!grid_barrier(ctl, bar, la.limit_ns)) return;
        if (threadIdx.x == 0) {
            if (blockIdx.x == 0) zero_slot(&ctl->slot[(n + 2) % kSlots]);
            const Slot s = read_slot(&ctl->slot[n % kSlots]);
            const Decision dcs = decide(SLR_RED_MAX_ABS_DELTA, s, la.tol);
            const long long it = it0 + n + 1;
            s_stop = dcs.converged || it >= la.max_iters;
            if (s_stop && blockIdx.x == 0) {
                ctl->iters = it;
                ctl->value = dcs.value;
                ctl->count = 0;
                ctl->changed = 1;
                ctl->converged = dcs.converged;
            }
        }
        __syncthreads();
        if (s_stop) {
            if ((n & 1) == 0) grid_copy(a.ub, a.u, (size_t)a.nx * (size_t)a.ny * (size_t)a.nz * sizeof(double));
            return;
        }
    }
}

}  // namespace

size_t dc_workspace_bytes(long long nx, long long ny, long long nz)
{
    const size_t cells = (size_t)nx * (size_t)ny * (size_t)nz;
    return 3 * ((cells * 4 + 255) / 256 * 256);   // r32, e[0], e[1] (the FP64 buffer is the usual state buffer)
}

cudaError_t dc_persistent(const Problem &p, LoopArgs la, int inner, void *fp32_area, cudaStream_t st)
{
    DcArgs a;
    a.u = (double *)la.a;
    a.ub = (double *)la.b;
    a.f = (const double *)la.aux;
    const size_t cells = (size_t)p.nx * (size_t)p.ny * (size_t)p.nz;
    const size_t blk = (cells * 4 + 255) / 256 * 256;
    a.r32 = (float *)fp32_area;
    a.e[0] = (float *)((unsigned char *)fp32_area + blk);
    a.e[1] = (float *)((unsigned char *)fp32_area + 2 * blk);
    a.nx = p.nx;
    a.ny = p.ny;
    a.nz = p.nz;
    a.h2 = p.h2;
    a.d = p.d;
    a.h2f = p.h2f;
    a.df = p.df;
    a.inner = inner > 0 ? inner : 50;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *kern = p.stencil == SLR_J3D7 ? (const void *)dc_kernel<3> : (const void *)dc_kernel<2>;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    la.nblocks = grid_ctas(sms, 1, la.nblocks);
    void *args[] = {&a, &la};
    return cudaLaunchCooperativeKernel(kern, dim3(la.nblocks), dim3(kDThreads), args, 0, st);
}

}  // namespace slr
