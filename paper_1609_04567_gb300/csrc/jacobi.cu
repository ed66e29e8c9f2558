// jacobi.cu -- Helmholtz Jacobi sweeps (the Sec. 4.1 solver: each point of
// the read-only right-hand side f combined with the neighbourhood of the
// current solution) in 2D (5-point) and 3D (7-point), fused with the
// max |u' - u| reduce and looped on the device (Sec. 3.1, -d and -s variants).
//
//   2D: u' = (h2 f + ((u_N + u_S) + u_W) + u_E) / (4 + sigma h2)
//   3D: u' = (h2 f + ((((u_x- + u_x+) + u_y-) + u_y+) + u_z-) + u_z+) / (6 + sigma h2)
//
// Storage: binary64 (binary64 arithmetic), binary32, bfloat16 or binary16
// (binary32 arithmetic; the new value is rounded to nearest even into the
// storage type and the change is taken between stored values).  Every
// operation is an explicitly rounded IEEE operation (no contraction into
// fused multiply-adds), in the order above, so results are bit-identical to a
// sequential evaluation of the same formula.
#include "slr_internal.cuh"

namespace slr {
namespace {

constexpr int kJThreads = 1024;

// ---- storage types --------------------------------------------------------
template <class T> struct Store;
template <> struct Store<double> {
    using C = double;
    __device__ __forceinline__ static C ld(const double *p) { return __ldcg(p); }
    __device__ __forceinline__ static C ldf(const double *p) { return __ldg(p); }
    __device__ __forceinline__ static double st(C v) { return v; }
    __device__ __forceinline__ static C back(double s) { return s; }
};
template <> struct Store<float> {
    using C = float;
    __device__ __forceinline__ static C ld(const float *p) { return __ldcg(p); }
    __device__ __forceinline__ static C ldf(const float *p) { return __ldg(p); }
    __device__ __forceinline__ static float st(C v) { return v; }
    __device__ __forceinline__ static C back(float s) { return s; }
};
template <> struct Store<__nv_bfloat16> {
    using C = float;
    __device__ __forceinline__ static C ld(const __nv_bfloat16 *p)
    {
        return __uint_as_float((uint32_t)__ldcg((const unsigned short *)p) << 16);
    }
    __device__ __forceinline__ static C ldf(const __nv_bfloat16 *p)
    {
        return __uint_as_float((uint32_t)__ldg((const unsigned short *)p) << 16);
    }
    __device__ __forceinline__ static __nv_bfloat16 st(C v) { return __float2bfloat16_rn(v); }
    __device__ __forceinline__ static C back(__nv_bfloat16 s) { return __bfloat162float(s); }
};
template <> struct Store<__half> {
    using C = float;
    __device__ __forceinline__ static C ld(const __half *p)
    {
        const unsigned short b = __ldcg((const unsigned short *)p);
        return __half2float(__ushort_as_half(b));
    }
    __device__ __forceinline__ static C ldf(const __half *p)
    {
        const unsigned short b = __ldg((const unsigned short *)p);
        return __half2float(__ushort_as_half(b));
    }
    __device__ __forceinline__ static __half st(C v) { return __float2half_rn(v); }
    __device__ __forceinline__ static C back(__half s) { return __half2float(s); }
};

// ---- explicitly rounded arithmetic ---------------------------------------
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }

// Running max of |delta| as bit patterns: for non-negative IEEE values the
// unsigned order of the bits is the numeric order (and a NaN stays the max).
// binary32 deltas keep 32-bit patterns and are widened once, at the end.
__device__ __forceinline__ void max_bits(unsigned long long &m, double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(d));
    m = b > m ? b : m;
}
__device__ __forceinline__ void max_bits(unsigned int &m, float d)
{
    const unsigned int b = __float_as_uint(fabsf(d));
    m = b > m ? b : m;
}
__device__ __forceinline__ unsigned long long widen_bits(unsigned long long m) { return m; }
__device__ __forceinline__ unsigned long long widen_bits(unsigned int m)
{
    return (unsigned long long)__double_as_longlong((double)__uint_as_float(m));
}
template <class C> struct MaxBits { using type = unsigned long long; };
template <> struct MaxBits<float> { using type = unsigned int; };

template <class T, int DIM>
struct JacobiOp {
    using C = typename Store<T>::C;
    long long nx, ny, nz;
    int wrap;
    C ghost, h2, d;
    const T *f;

    __device__ __forceinline__ size_t state_bytes() const { return (size_t)nx * ny * nz * sizeof(T); }

    // value at (k, i, j) with the boundary rule
    __device__ __forceinline__ C at(const T *u, long long k, long long i, long long j) const
    {
        if (i < 0 || i >= ny || j < 0 || j >= nx || k < 0 || k >= nz) {
            if (!wrap) return ghost;
            i = i < 0 ? i + ny : (i >= ny ? i - ny : i);
            j = j < 0 ? j + nx : (j >= nx ? j - nx : j);
            k = k < 0 ? k + nz : (k >= nz ? k - nz : k);
        }
        return Store<T>::ld(u + (k * ny + i) * nx + j);
    }

    template <bool REDUCE>
    __device__ __forceinline__ void sweep(const void *src_v, void *dst_v, Slot *slot) const
    {
        const T *u = (const T *)src_v;
        T *v = (T *)dst_v;
        const long long chunks = (nx + blockDim.x - 1) / blockDim.x;
        const long long units = ny * nz * chunks;
        typename MaxBits<C>::type mx = 0;
        for (long long un = blockIdx.x; un < units; un += gridDim.x) {
            const long long row = un / chunks;
            const long long j = (un - row * chunks) * blockDim.x + threadIdx.x;
            if (j >= nx) continue;
            const long long k = row / ny, i = row - k * ny;
            const long long c = row * nx + j;
            const C uc = Store<T>::ld(u + c);
            C s;
            if (DIM == 2) {
                s = add_rn(add_rn(add_rn(at(u, k, i - 1, j), at(u, k, i + 1, j)), at(u, k, i, j - 1)),
                           at(u, k, i, j + 1));
            } else {
                s = add_rn(add_rn(add_rn(add_rn(add_rn(at(u, k, i, j - 1), at(u, k, i, j + 1)),
                                                at(u, k, i - 1, j)), at(u, k, i + 1, j)),
                                  at(u, k - 1, i, j)), at(u, k + 1, i, j));
            }
            const C t = mul_rn(h2, Store<T>::ldf(f + c));
            const T nv = Store<T>::st(div_rn(add_rn(t, s), d));
            v[c] = nv;
            if (REDUCE) max_bits(mx, sub_rn(Store<T>::back(nv), uc));
        }
        if (REDUCE) block_to_slot(slot, widen_bits(mx), 0ull, 0ull, mx != 0);
    }
};

template <class Op>
__global__ void __launch_bounds__(kJThreads, 1) jacobi_persistent_kernel(Op op, LoopArgs la)
{
    persistent_loop_body(op, la);
}

template <class Op>
__global__ void __launch_bounds__(kJThreads, 1) jacobi_sweep_kernel(Op op, const void *src, void *dst)
{
    op.template sweep<false>(src, dst, nullptr);
}

template <class T, int DIM>
JacobiOp<T, DIM> make_op(const Problem &p, const void *f)
{
    JacobiOp<T, DIM> op;
    op.nx = p.nx; op.ny = p.ny; op.nz = p.nz; op.wrap = p.wrap;
    if (sizeof(typename Store<T>::C) == 8) {
        op.ghost = (typename Store<T>::C)p.ghost; op.h2 = (typename Store<T>::C)p.h2; op.d = (typename Store<T>::C)p.d;
    } else {
        op.ghost = (typename Store<T>::C)p.ghostf; op.h2 = (typename Store<T>::C)p.h2f; op.d = (typename Store<T>::C)p.df;
    }
    op.f = (const T *)f;
    return op;
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <class T, int DIM>
cudaError_t run_persistent(const Problem &p, LoopArgs la, cudaStream_t st)
{
    auto op = make_op<T, DIM>(p, la.aux);
    return launch_cooperative(jacobi_persistent_kernel<JacobiOp<T, DIM>>, kJThreads, 0, 1, la, &op, st);
}

template <class T, int DIM>
cudaError_t run_sweep(const Problem &p, const void *src, void *dst, const void *f, cudaStream_t st)
{
    auto op = make_op<T, DIM>(p, f);
    jacobi_sweep_kernel<JacobiOp<T, DIM>><<<sm_count(), kJThreads, 0, st>>>(op, src, dst);
    return cudaGetLastError();
}

template <int DIM>
cudaError_t dispatch_persistent(const Problem &p, LoopArgs la, cudaStream_t st)
{
    switch (p.storage) {
    case SLR_F64: return run_persistent<double, DIM>(p, la, st);
    case SLR_F32: return run_persistent<float, DIM>(p, la, st);
    case SLR_BF16: return run_persistent<__nv_bfloat16, DIM>(p, la, st);
    case SLR_F16: return run_persistent<__half, DIM>(p, la, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int DIM>
cudaError_t dispatch_sweep(const Problem &p, const void *src, void *dst, const void *f, cudaStream_t st)
{
    switch (p.storage) {
    case SLR_F64: return run_sweep<double, DIM>(p, src, dst, f, st);
    case SLR_F32: return run_sweep<float, DIM>(p, src, dst, f, st);
    case SLR_BF16: return run_sweep<__nv_bfloat16, DIM>(p, src, dst, f, st);
    case SLR_F16: return run_sweep<__half, DIM>(p, src, dst, f, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t jacobi_persistent(const Problem &p, LoopArgs la, cudaStream_t st)
{
    return p.stencil == SLR_J3D7 ? dispatch_persistent<3>(p, la, st) : dispatch_persistent<2>(p, la, st);
}

cudaError_t jacobi_sweep(const Problem &p, const void *src, void *dst, const void *f, cudaStream_t st)
{
    return p.stencil == SLR_J3D7 ? dispatch_sweep<3>(p, src, dst, f, st) : dispatch_sweep<2>(p, src, dst, f, st);
}

}  // namespace slr
