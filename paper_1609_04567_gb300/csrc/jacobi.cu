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
// operation rounds as the IEEE operation in the order above (no contraction
// of a product into a sum), so results are bit-identical to a sequential
// evaluation of the same formula; the division by the constant d is formed
// from its correctly rounded reciprocal with two FMA corrections
// (crmath.cuh), which gives the IEEE quotient.
//
// Two sweep implementations, both one cooperative persistent launch per run:
// JacobiTma (Dirichlet ghost +0, rows of whole 16-byte groups, large grids)
// marches 256-cell columns with every step staged by TMA in a ring of
// shared-memory stages; JacobiStream (any boundary and width) marches row
// segments with the rows held in registers.
#include <string.h>

#include <cmath>
#include <type_traits>

#include "crmath.cuh"
#include "slr_internal.cuh"
#include "tma.cuh"

namespace slr {
namespace {

constexpr int kJThreads = 256;

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
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
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

// ---- streaming sweep ----------------------------------------------------------
// A warp owns a segment of 32*V consecutive cells of a row (V cells per lane,
// one 16-byte access when the row allows it) and marches along the slowest
// axis (y in 2D, z in 3D) over a run of rows or planes, keeping a window of
// rows of its segment in registers and loading the next few rows (and their
// f) together before computing them: each cell of u
// is loaded from memory about once per sweep in 2D (the 3D sweep also loads
// the rows y - 1 and y + 1 of the current plane, which the neighbouring warps
// have just brought into L2).  x-neighbours come from the adjacent lanes by
// shuffles; the segment's two outer neighbours, and those beyond the grid,
// by single loads with the boundary rule.
// V consecutive cells of a row in their storage format, packed in 32-bit
// words (4 words for a 16-byte group), widened to the compute type on use; a
// row past a Dirichlet edge is flagged instead (its cells read as the ghost).
template <class T, int V>
struct Packed {
    static constexpr int kWords = (V * (int)sizeof(T) + 3) / 4;
    uint32_t w[kWords];
    bool ghost;

    __device__ __forceinline__ void load(const T *p, bool readonly)
    {
        ghost = false;
        if constexpr (V * sizeof(T) == 16) {
            const uint4 r = readonly ? __ldg((const uint4 *)p) : __ldcg((const uint4 *)p);
            w[0] = r.x; w[1] = r.y; w[2] = r.z; w[3] = r.w;
        } else if constexpr (sizeof(T) == 8) {
            const unsigned long long r = readonly ? __ldg((const unsigned long long *)p)
                                                  : __ldcg((const unsigned long long *)p);
            w[0] = (uint32_t)r; w[1] = (uint32_t)(r >> 32);
        } else if constexpr (sizeof(T) == 4) {
            w[0] = readonly ? __ldg((const unsigned int *)p) : __ldcg((const unsigned int *)p);
        } else {
            w[0] = readonly ? __ldg((const unsigned short *)p) : __ldcg((const unsigned short *)p);
        }
    }

    // cell k widened (exact: every storage value is a compute-type value)
    __device__ __forceinline__ typename Store<T>::C raw(int k) const
    {
        if constexpr (sizeof(T) == 8) {
            return __hiloint2double((int)w[2 * k + 1], (int)w[2 * k]);
        } else if constexpr (sizeof(T) == 4) {
            return __uint_as_float(w[k]);
        } else {
            const uint32_t h = (k & 1) ? (w[k >> 1] >> 16) : (w[k >> 1] & 0xFFFFu);
            if constexpr (std::is_same<T, __nv_bfloat16>::value) return __uint_as_float(h << 16);
            else return __half2float(__ushort_as_half((unsigned short)h));
        }
    }

    __device__ __forceinline__ typename Store<T>::C at(int k, typename Store<T>::C g) const
    {
        return ghost ? g : raw(k);
    }
};

// storage bits of one value, in the low bits of a 32-bit word (2-byte types)
__device__ __forceinline__ uint32_t bits16(__nv_bfloat16 h) { return (uint32_t)__bfloat16_as_ushort(h); }
__device__ __forceinline__ uint32_t bits16(__half h) { return (uint32_t)__half_as_ushort(h); }

// two computed values rounded to the storage type by one paired conversion, in
// one 32-bit word (the first in the low half), and the stored values widened back
template <class T> struct Pair2;
template <> struct Pair2<__nv_bfloat16> {
    __device__ __forceinline__ static uint32_t pack(float a, float b)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *(const uint32_t *)&h;
    }
    __device__ __forceinline__ static float2 widen(uint32_t w)
    {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
    }
};
template <> struct Pair2<__half> {
    __device__ __forceinline__ static uint32_t pack(float a, float b)
    {
        const __half2 h = __floats2half2_rn(a, b);
        return *(const uint32_t *)&h;
    }
    __device__ __forceinline__ static float2 widen(uint32_t w)
    {
        return __half22float2(*(const __half2 *)&w);
    }
};

// ---- streaming sweep ----------------------------------------------------------
// A warp owns a segment of 32*V consecutive cells of a row (V cells per lane,
// one 16-byte access when the row allows it) and marches along the slowest
// axis (y in 2D, z in 3D) over a run of rows or planes, keeping a window of
// rows of its segment in registers and loading the next few rows (and their
// f) together before computing them: each cell of u
// is loaded from memory about once per sweep in 2D (the 3D sweep also loads
// the rows y - 1 and y + 1 of the current plane, which the neighbouring warps
// have just brought into L2).  x-neighbours come from the adjacent lanes by
// shuffles; the segment's two outer neighbours, and those beyond the grid,
// by single loads with the boundary rule.
template <class T, int DIM, int V>
struct JacobiStream {
    using C = typename Store<T>::C;
    using Row = Packed<T, V>;
    static constexpr int kSeg = 32 * V;   // cells per warp segment
    int nx, ny, nz;                       // extents, each below 2^31 - 4096
    int nseg;                             // segments per row
    int run;                              // rows (2D) or planes (3D) one warp marches per unit
    int wrap;
    C ghost, h2, d;
    C yd;                                 // RN(1 / d)
    int dconst;                           // d in the range of div_const_rn
    const T *f;

    __device__ __forceinline__ size_t state_bytes() const { return (size_t)nx * ny * nz * sizeof(T); }
    __device__ __forceinline__ void prologue() const {}

    __device__ __forceinline__ C divide(C a) const { return dconst ? div_const_rn(a, d, yd) : div_ieee(a, d); }

    __device__ __forceinline__ size_t off(int y, int z, int x) const { return ((size_t)z * ny + y) * nx + x; }

    // the segment of row (y, z) starting at x, or a ghost row past a Dirichlet edge
    __device__ __forceinline__ void row(const T *u, int y, int z, int x, bool ok, Row &r) const
    {
        if (y < 0 || y >= ny || z < 0 || z >= nz) {
            if (!wrap) {
                r.ghost = true;
                return;
            }
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
        }
        if (ok) r.load(u + off(y, z, x), false);
        else r.ghost = true;
    }

    // cell (y, z, x) of an in-range row, x possibly -1 or nx
    __device__ __forceinline__ C cell(const T *u, int y, int z, int x) const
    {
        if (x < 0 || x >= nx) {
            if (!wrap) return ghost;
            x = x < 0 ? x + nx : x - nx;
        }
        return Store<T>::ld(u + off(y, z, x));
    }

    // new values of the lane's V cells of row (y, z): c = this row, a/b = the
    // rows before/after along the march (y in 2D, z in 3D), n/s = the rows
    // y - 1 / y + 1 of the same plane (3D)
    template <bool REDUCE>
    __device__ __forceinline__ void update(const T *u, T *v, int y, int z, int x, bool ok, int lane, const Row &a,
                                           const Row &c, const Row &b, const Row &fr, const Row &n, const Row &s,
                                           typename MaxBits<C>::type &mx) const
    {
        C left = __shfl_up_sync(0xffffffffu, c.raw(V - 1), 1);
        C right = __shfl_down_sync(0xffffffffu, c.raw(0), 1);
        if (!ok) return;                                   // past the end of the row
        if (lane == 0) left = cell(u, y, z, x - 1);
        if (lane == 31 || x + V >= nx) right = cell(u, y, z, x + V);   // x + V <= nx here
        uint32_t ow[Row::kWords];                          // the new values, packed like a Row
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const C w = k > 0 ? c.raw(k - 1) : left, e = k < V - 1 ? c.raw(k + 1) : right;
            C sum;
            if (DIM == 2) sum = add_rn(add_rn(add_rn(a.at(k, ghost), b.at(k, ghost)), w), e);
            else sum = add_rn(add_rn(add_rn(add_rn(add_rn(w, e), n.at(k, ghost)), s.at(k, ghost)), a.at(k, ghost)),
                              b.at(k, ghost));
            const T o = Store<T>::st(divide(add_rn(mul_rn(h2, fr.raw(k)), sum)));
            if (REDUCE) max_bits(mx, sub_rn(Store<T>::back(o), c.raw(k)));
            if constexpr (sizeof(T) == 8) {
                ow[2 * k] = (uint32_t)__double2loint((double)o);
                ow[2 * k + 1] = (uint32_t)__double2hiint((double)o);
            } else if constexpr (sizeof(T) == 4) {
                ow[k] = __float_as_uint((float)o);
            } else {
                if (k & 1) ow[k >> 1] |= bits16(o) << 16;
                else ow[k >> 1] = bits16(o);
            }
        }
        T *dst = v + off(y, z, x);
        if constexpr (V * sizeof(T) == 16) *(uint4 *)dst = make_uint4(ow[0], ow[1], ow[2], ow[3]);
        else if constexpr (sizeof(T) == 8) *(unsigned long long *)dst = (unsigned long long)ow[1] << 32 | ow[0];
        else if constexpr (sizeof(T) == 4) *(unsigned int *)dst = ow[0];
        else *(unsigned short *)dst = (unsigned short)ow[0];
    }

    template <bool REDUCE>
    __device__ __forceinline__ void sweep(const void *src_v, void *dst_v, Slot *slot) const
    {
        constexpr int P = DIM == 2 ? 4 : 2;                    // rows computed per batch of loads
        const T *u = (const T *)src_v;
        T *v = (T *)dst_v;
        const int lane = threadIdx.x & 31;
        const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
        const int mlen = DIM == 2 ? ny : nz;                   // extent of the march axis
        const int runs = (mlen + run - 1) / run;
        const long long units = (long long)runs * (DIM == 2 ? 1 : ny) * nseg;
        typename MaxBits<C>::type mx = 0;
        // consecutive units (neighbouring segments, then rows) go to the same
        // warp slot of consecutive CTAs, which run at the same time
        for (long long un = (long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; un < units; un += nw) {
            const int seg = (int)(un % nseg);
            const long long rest = un / nseg;
            const int y3 = DIM == 2 ? 0 : (int)(rest % ny);
            const int m0 = (int)(DIM == 2 ? rest : rest / ny) * run;
            const int m1 = m0 + run < mlen ? m0 + run : mlen;
            const int x = seg * kSeg + lane * V;
            const bool ok = x < nx;
            // window w[0..P+1] = rows m-1 .. m+P along the march; w[0], w[1]
            // carry over from the previous batch
            Row w[P + 2], fq[P], nq[P], sq[P];
            if (DIM == 2) {
                row(u, m0 - 1, 0, x, ok, w[0]);
                row(u, m0, 0, x, ok, w[1]);
            } else {
                row(u, y3, m0 - 1, x, ok, w[0]);
                row(u, y3, m0, x, ok, w[1]);
            }
            for (int m = m0; m < m1; m += P) {
                // every load of the batch first, so their latencies overlap
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    w[j + 2].ghost = fq[j].ghost = nq[j].ghost = sq[j].ghost = true;
                    if (m + 1 + j <= m1) {
                        if (DIM == 2) row(u, m + 1 + j, 0, x, ok, w[j + 2]);
                        else row(u, y3, m + 1 + j, x, ok, w[j + 2]);
                    }
                    if (m + j < m1 && ok) {
                        fq[j].load(f + off(DIM == 2 ? m + j : y3, DIM == 2 ? 0 : m + j, x), true);
                        if (DIM == 3) {
                            row(u, y3 - 1, m + j, x, ok, nq[j]);
                            row(u, y3 + 1, m + j, x, ok, sq[j]);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < P; ++j) {
                    if (m + j < m1) {
                        if (DIM == 2) update<REDUCE>(u, v, m + j, 0, x, ok, lane, w[j], w[j + 1], w[j + 2], fq[j], nq[j], sq[j], mx);
                        else update<REDUCE>(u, v, y3, m + j, x, ok, lane, w[j], w[j + 1], w[j + 2], fq[j], nq[j], sq[j], mx);
                    }
                }
                w[0] = w[P];
                w[1] = w[P + 1];
            }
        }
        if (REDUCE) block_to_slot(slot, widen_bits(mx), 0ull, 0ull, mx != 0);
    }
};

// ---- TMA tiles (Dirichlet boundary with ghost 0, large grids) -----------------
// A CTA owns a column of the grid 256 cells wide (3D: and kTY rows high) and
// marches along the slowest axis: in 3D one z-plane of its tile per step
// (the tile's kTY rows plus the rows above and below), in 2D a block of kTY
// rows per step.  Every step arrives in a ring of kNS shared-memory stages as
// TMA boxes: the tile, a 16-byte column on each side of it (the x-neighbours
// of the tile's edge cells) and the tile of f; the tensor maps fill
// everything outside the grid with zeros, which is the ghost.  The CTA
// computes step j from the stages of steps j - 1, j and j + 1 while the next
// step's boxes are in flight; one CTA barrier per step frees the oldest
// stage, which thread 0 refills.  (column, step) pairs are dealt out to the
// CTAs in contiguous ranges of equal length, so every CTA does the same work
// in a sweep.
template <class T, int DIM>
struct JacobiTma {
    using C = typename Store<T>::C;
    using Row = Packed<T, 16 / sizeof(T)>;
    static constexpr int V = 16 / (int)sizeof(T);
    static constexpr int kTX = 256;                                  // tile width (cells)
    static constexpr int kG = kTX / V;                               // 16-byte groups per tile row
    static constexpr int kTY = 32 / (int)sizeof(T);                  // tile rows (a tile row is kTX cells)
    static constexpr int kHalo = DIM == 3 ? 1 : 0;                   // y-halo rows above and below (3D)
    static constexpr int kRowBytes = kTX * (int)sizeof(T);
    static constexpr int kMainBytes = (kTY + 2 * kHalo) * kRowBytes;
    static constexpr int kSideBytes = (kTY * 16 + 127) / 128 * 128;
    static constexpr int kFBytes = kTY * kRowBytes;
    static constexpr int kStage = kMainBytes + 2 * kSideBytes + kFBytes;
    static constexpr int kNS = 4;                                    // stages (a power of 2)
    static constexpr int kPer = kTY * kG / kJThreads;                // 16-byte groups per thread per step
    static constexpr size_t kSmem = 128 + (size_t)kNS * kStage + kNS * 8 + 16;
    static_assert(kStage % 128 == 0 && kMainBytes % 128 == 0 && kFBytes % 128 == 0, "TMA destinations");
    static_assert(kPer * kJThreads == kTY * kG, "threads tile the step");

    CUtensorMap umap[2], smap[2], fmap;      // tile and side-column maps over A and B, f map
    const void *base[2];
    int *err;
    long long limit_ns;
    int nx, ny, nz;
    int tiles_x, tiles_y;                    // tiles across the plane (2D: tiles_y = 1)
    C h2, d, yd;
    int dconst;

    __device__ __forceinline__ size_t state_bytes() const { return (size_t)nx * ny * nz * sizeof(T); }
    __device__ __forceinline__ C divide(C a) const { return dconst ? div_const_rn(a, d, yd) : div_ieee(a, d); }

    __device__ __forceinline__ unsigned char *stages() const
    {
        extern __shared__ unsigned char smem_dyn[];
        return align_up(smem_dyn, 128);
    }
    __device__ __forceinline__ const T *main_of(int s) const { return (const T *)(stages() + s * kStage); }
    __device__ __forceinline__ const T *side_of(int s, int i) const
    {
        return (const T *)(stages() + s * kStage + kMainBytes + i * kSideBytes);   // 0: left, 1: right
    }
    __device__ __forceinline__ const T *f_of(int s) const
    {
        return (const T *)(stages() + s * kStage + kMainBytes + 2 * kSideBytes);
    }
    __device__ __forceinline__ uint64_t *bar(int s) const { return (uint64_t *)(stages() + kNS * kStage) + s; }
    __device__ __forceinline__ unsigned *counter() const { return (unsigned *)(bar(kNS)); }

    __device__ __forceinline__ void prologue() const
    {
        if (threadIdx.x == 0) {
            for (int s = 0; s < kNS; ++s) tma::mbar_init(bar(s), 1);
            *counter() = 0u;
            tma::mbar_init_fence();
        }
        __syncthreads();
    }

    // thread 0: boxes of step j of column col into stage sl; f only for the
    // steps the CTA computes.  A box entirely outside the grid is not issued
    // (its cells are ghosts, and the compute side knows which ones).
    __device__ __forceinline__ void issue(int mi, int sl, int col, int j, bool with_f) const
    {
        unsigned char *st = stages() + sl * kStage;
        const int tx = col % tiles_x, ty = col / tiles_x;
        const int x0 = tx * kTX;
        const bool step_in = DIM == 3 ? (j >= 0 && j < nz) : (j >= 0 && j * kTY < ny);
        const bool left_in = step_in && x0 > 0, right_in = step_in && x0 + kTX < nx;
        const uint32_t bytes = (step_in ? (uint32_t)kMainBytes : 0u) + (left_in ? kTY * 16u : 0u) +
                               (right_in ? kTY * 16u : 0u) + (with_f ? (uint32_t)kFBytes : 0u);
        tma::mbar_expect_tx(bar(sl), bytes);
        const int y0 = DIM == 3 ? ty * kTY : j * kTY;
        if (DIM == 3) {
            if (step_in) tma::load_3d(st, &umap[mi], x0, y0 - 1, j, bar(sl));
            if (left_in) tma::load_3d(st + kMainBytes, &smap[mi], x0 - V, y0, j, bar(sl));
            if (right_in) tma::load_3d(st + kMainBytes + kSideBytes, &smap[mi], x0 + kTX, y0, j, bar(sl));
            if (with_f) tma::load_3d(st + kMainBytes + 2 * kSideBytes, &fmap, x0, y0, j, bar(sl));
        } else {
            if (step_in) tma::load_2d(st, &umap[mi], x0, y0, bar(sl));
            if (left_in) tma::load_2d(st + kMainBytes, &smap[mi], x0 - V, y0, bar(sl));
            if (right_in) tma::load_2d(st + kMainBytes + kSideBytes, &smap[mi], x0 + kTX, y0, bar(sl));
            if (with_f) tma::load_2d(st + kMainBytes + 2 * kSideBytes, &fmap, x0, y0, bar(sl));
        }
    }

    __device__ __forceinline__ Row lds(const T *p) const
    {
        const uint4 q = *(const uint4 *)p;
        Row r;
        r.w[0] = q.x; r.w[1] = q.y; r.w[2] = q.z; r.w[3] = q.w;
        r.ghost = false;
        return r;
    }

    // all threads: rows [r0, r0 + n) of stage s's tile set to +0
    __device__ __forceinline__ void zero_rows(int s, int r0, int n) const
    {
        uint4 *p = (uint4 *)(stages() + s * kStage + r0 * kRowBytes);
        for (int i = threadIdx.x; i < n * kRowBytes / 16; i += kJThreads) p[i] = make_uint4(0u, 0u, 0u, 0u);
    }

    template <bool REDUCE>
    __device__ __forceinline__ void sweep(const void *src_v, void *dst_v, Slot *slot) const
    {
        __shared__ int s_stop;
        __shared__ T s_ghost;                                      // the ghost value 0, for the end lanes
        T *v = (T *)dst_v;
        const int tid = threadIdx.x;
        const int mi = src_v == base[0] ? 0 : 1;
        const int ncols = tiles_x * tiles_y;
        const int mlen = DIM == 3 ? nz : (ny + kTY - 1) / kTY;       // steps per column
        typename MaxBits<C>::type mx = 0;
        float mxf = 0.0f;                                          // binary32 compute: max |delta|
        unsigned q = *counter();
        if (tid == 0) {
            s_stop = ld_relaxed_u32((const unsigned *)err) != 0u;   // a wait ran out earlier
            s_ghost = Store<T>::st(C(0));
            tma::fence_proxy_async_global();   // the previous sweep's stores before this sweep's copies
        }
        __syncthreads();
        const long long total = (long long)ncols * mlen;
        long long L = s_stop ? 0 : (long long)blockIdx.x * total / gridDim.x;
        const long long Lend = s_stop ? 0 : ((long long)blockIdx.x + 1) * total / gridDim.x;
        bool alive = true;
        while (L < Lend && alive) {
            const int col = (int)(L / mlen);
            const int ja = (int)(L - (long long)col * mlen);
            const int jb = (long long)mlen - ja < Lend - L ? mlen : ja + (int)(Lend - L);
            const int R = jb - ja + 2;                               // steps ja - 1 .. jb
            const int tx = col % tiles_x, ty = col / tiles_x;
            const int x0 = tx * kTX, y0 = ty * kTY;
            if (tid == 0)
                for (int i = 0; i < R && i < kNS; ++i)
                    issue(mi, (int)((q + (unsigned)i) & (kNS - 1)), col, ja - 1 + i, i >= 1 && i <= jb - ja);
            int waited = -1;
            for (int j = ja; j < jb; ++j) {
                const int ic = j - ja + 1;
                bool got = true;
                while (waited < ic + 1) {
                    ++waited;
                    const unsigned qi = q + (unsigned)waited;
                    got = got && tma::bounded_wait(bar((int)(qi & (kNS - 1))), (qi / kNS) & 1u, tma::kLoadWaitNs, err);
                }
                const int sa = (int)((q + (unsigned)(ic - 1)) & (kNS - 1)), sc = (int)((q + (unsigned)ic) & (kNS - 1)),
                          sb = (int)((q + (unsigned)(ic + 1)) & (kNS - 1));
                // steps -1 and mlen lie outside the grid and were not loaded:
                // the rows of them this step reads are set to the ghost 0
                if (j == 0 || j + 1 == mlen) {
                    if (j == 0) zero_rows(sa, DIM == 3 ? 1 : kTY - 1, DIM == 3 ? kTY : 1);
                    if (j + 1 == mlen) zero_rows(sb, DIM == 3 ? 1 : 0, DIM == 3 ? kTY : 1);
                    __syncthreads();
                }
                const T *Mc = main_of(sc), *Ma = main_of(sa), *Mb = main_of(sb), *F = f_of(sc);
                // the side columns, or the ghost where the tile touches the grid's edge
                const T *SL = x0 > 0 ? side_of(sc, 0) + V - 1 : &s_ghost;
                const T *SR = x0 + kTX < nx ? side_of(sc, 1) : &s_ghost;
                const int sstep_l = x0 > 0 ? V : 0, sstep_r = x0 + kTX < nx ? V : 0;
#pragma unroll
                for (int p = 0; p < kPer; ++p) {
                    const int g = tid + p * kJThreads;
                    const int r = g / kG, c = g % kG;          // a warp covers 32 consecutive groups of one row
                    const int x = x0 + c * V;
                    const int y = DIM == 3 ? y0 + r : j * kTY + r;
                    const T *ctr = Mc + (r + kHalo) * kTX + c * V;
                    const Row cv = lds(ctr);
                    // x-neighbours of the lane's first and last cell from the adjacent lanes;
                    // the warp's two end lanes read them from the tile or the side columns
                    const int lane = tid & 31;
                    C left = __shfl_up_sync(0xffffffffu, cv.raw(V - 1), 1);
                    C right = __shfl_down_sync(0xffffffffu, cv.raw(0), 1);
                    if (!got || x >= nx || y >= ny) continue;
                    const T *lp = c > 0 ? ctr - 1 : SL + r * sstep_l;
                    const T *rp = c < kG - 1 ? ctr + V : SR + r * sstep_r;
                    if (lane == 0) left = Store<T>::back(*lp);
                    if (lane == 31) right = Store<T>::back(*rp);
                    const Row fr = lds(F + r * kTX + c * V);
                    Row nr, sr, ar, br;                              // y-1, y+1, march-1, march+1
                    if (DIM == 3) {
                        nr = lds(ctr - kTX);
                        sr = lds(ctr + kTX);
                        ar = lds(Ma + (r + 1) * kTX + c * V);
                        br = lds(Mb + (r + 1) * kTX + c * V);
                    } else {
                        ar = lds(r > 0 ? ctr - kTX : Ma + (kTY - 1) * kTX + c * V);
                        br = lds(r < kTY - 1 ? ctr + kTX : Mb + c * V);
                        nr.ghost = sr.ghost = true;
                    }
                    uint32_t ow[Row::kWords];
                    if constexpr (std::is_same<C, float>::value) {
                        // two cells per paired binary32 operation (same rounding per cell).
                        // The numerators of the group come first; one range test over all of
                        // them (|a| in [2^-40, 2^40)) then picks Markstein's corrected quotient
                        // for the whole group, or the per-cell path when any falls outside.
                        float q[V];
                        float amin = INFINITY, amax = 0.0f;       // |numerator| over the group
                        const float2 y2 = make_float2(yd, yd), nd2 = make_float2(-d, -d);
#pragma unroll
                        for (int k = 0; k < V; k += 2) {
                            const float2 w = make_float2(k > 0 ? cv.raw(k - 1) : left, cv.raw(k));
                            const float2 e = make_float2(cv.raw(k + 1), k + 2 < V ? cv.raw(k + 2) : right);
                            const float2 a2 = make_float2(ar.raw(k), ar.raw(k + 1));
                            const float2 b2 = make_float2(br.raw(k), br.raw(k + 1));
                            float2 sum;
                            if (DIM == 2) {
                                sum = __fadd2_rn(__fadd2_rn(__fadd2_rn(a2, b2), w), e);
                            } else {
                                const float2 n2 = make_float2(nr.raw(k), nr.raw(k + 1));
                                const float2 s2 = make_float2(sr.raw(k), sr.raw(k + 1));
                                sum = __fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(w, e), n2), s2), a2), b2);
                            }
                            // h^2 f with the scalar operation: a paired product feeding a paired
                            // sum may be contracted into one fused operation
                            const float2 t = make_float2(__fmul_rn(h2, fr.raw(k)), __fmul_rn(h2, fr.raw(k + 1)));
                            const float2 num = __fadd2_rn(t, sum);
                            // a NaN numerator passes the test and gives NaN either way
                            amin = min3f(amin, fabsf(num.x), fabsf(num.y));
                            amax = max3f(amax, fabsf(num.x), fabsf(num.y));
                            q[k] = num.x;
                            q[k + 1] = num.y;
                        }
                        if (dconst && amin >= 0x1p-40f && amax < 0x1p40f) {
#pragma unroll
                            for (int k = 0; k < V; k += 2) {
                                // Markstein's corrected quotient; fma(q, -d, a) is the residual a - q d
                                const float2 num = make_float2(q[k], q[k + 1]);
                                const float2 q0 = __fmul2_rn(num, y2);
                                const float2 q1 = __ffma2_rn(__ffma2_rn(q0, nd2, num), y2, q0);
                                const float2 qq = __ffma2_rn(__ffma2_rn(q1, nd2, num), y2, q1);
                                q[k] = qq.x;
                                q[k + 1] = qq.y;
                            }
                        } else {
                            // rare: a numerator outside the range of the corrected quotient
#pragma unroll
                            for (int k = 0; k < V; ++k) q[k] = divide(q[k]);
                        }
                        const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
                        for (int k = 0; k < V; k += 2) {
                            float2 o;                                // the stored values, widened
                            if constexpr (sizeof(T) == 4) {
                                ow[k] = __float_as_uint(q[k]);
                                ow[k + 1] = __float_as_uint(q[k + 1]);
                                o = make_float2(q[k], q[k + 1]);
                            } else {
                                ow[k >> 1] = Pair2<T>::pack(q[k], q[k + 1]);
                                o = Pair2<T>::widen(ow[k >> 1]);
                            }
                            if (REDUCE) {
                                // |old - new| (fma(new, -1, old) is the rounded difference);
                                // max as binary32 in one op, a NaN skipped as by the
                                // sequential test d > max
                                const float2 dl = __ffma2_rn(o, m1, make_float2(cv.raw(k), cv.raw(k + 1)));
                                mxf = max3f(mxf, fabsf(dl.x), fabsf(dl.y));
                            }
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < V; ++k) {
                            const C w = k > 0 ? cv.raw(k - 1) : left, e = k < V - 1 ? cv.raw(k + 1) : right;
                            C sum;
                            if (DIM == 2) sum = add_rn(add_rn(add_rn(ar.raw(k), br.raw(k)), w), e);
                            else sum = add_rn(add_rn(add_rn(add_rn(add_rn(w, e), nr.raw(k)), sr.raw(k)), ar.raw(k)),
                                              br.raw(k));
                            const T o = Store<T>::st(divide(add_rn(mul_rn(h2, fr.raw(k)), sum)));
                            if (REDUCE) max_bits(mx, sub_rn(Store<T>::back(o), cv.raw(k)));
                            ow[2 * k] = (uint32_t)__double2loint((double)o);
                            ow[2 * k + 1] = (uint32_t)__double2hiint((double)o);
                        }
                    }
                    const size_t off = DIM == 3 ? ((size_t)j * ny + y) * nx + x : (size_t)y * nx + x;
                    *(uint4 *)(v + off) = make_uint4(ow[0], ow[1], ow[2], ow[3]);
                }
                // the stage of step j - 1 is free once every thread is past this step
                if (__syncthreads_or(!got)) { alive = false; break; }
                if (tid == 0 && ic - 1 + kNS < R)
                    issue(mi, sa, col, j - 1 + kNS, ic - 1 + kNS <= jb - ja);
            }
            q += (unsigned)R;
            L += jb - ja;
        }
        __syncthreads();
        if (tid == 0) *counter() = q;
        tma::fence_proxy_async_global();                             // this sweep's stores before later copies
        if constexpr (std::is_same<C, float>::value) mx = __float_as_uint(mxf);   // non-negative: bits order as values
        if (REDUCE) block_to_slot(slot, widen_bits(mx), 0ull, 0ull, mx != 0);
    }
};

template <class Op>
__global__ void __launch_bounds__(kJThreads, 3) jacobi_persistent_kernel(const __grid_constant__ Op op, LoopArgs la)
{
    op.prologue();
    persistent_loop_body(op, la);
}

template <class Op>
__global__ void __launch_bounds__(kJThreads, 3) jacobi_sweep_kernel(const __grid_constant__ Op op, const void *src,
                                                                     void *dst)
{
    op.prologue();
    op.template sweep<false>(src, dst, nullptr);
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <class T, int DIM, int V>
JacobiStream<T, DIM, V> make_op(const Problem &p, const void *f)
{
    JacobiStream<T, DIM, V> op;
    op.nx = (int)p.nx; op.ny = (int)p.ny; op.nz = (int)p.nz; op.wrap = p.wrap;
    op.nseg = (int)((p.nx + JacobiStream<T, DIM, V>::kSeg - 1) / JacobiStream<T, DIM, V>::kSeg);
    // run length: up to 32, short enough that every warp of a full grid gets
    // about four units
    const long long across = (long long)op.nseg * (DIM == 2 ? 1 : p.ny);
    const long long mlen = DIM == 2 ? p.ny : p.nz;
    const long long warps = (long long)sm_count() * 3 * (kJThreads / 32);
    long long run = mlen * across / (4 * warps);
    op.run = (int)(run < 1 ? 1 : (run > 32 ? 32 : run));
    if (sizeof(typename Store<T>::C) == 8) {
        op.ghost = (typename Store<T>::C)p.ghost; op.h2 = (typename Store<T>::C)p.h2; op.d = (typename Store<T>::C)p.d;
    } else {
        op.ghost = (typename Store<T>::C)p.ghostf; op.h2 = (typename Store<T>::C)p.h2f; op.d = (typename Store<T>::C)p.df;
    }
    op.dconst = div_const_ok(op.d);
    op.yd = host_rcp_rn(op.d);
    op.f = (const T *)f;
    return op;
}

// 16-byte accesses need rows of whole 16-byte groups and 16-byte aligned arrays
// (grids too small to give every lane of a full grid V cells run one cell per
// lane instead, which spreads their arithmetic over more SMs)
template <class T>
bool vector_ok(const Problem &p, const void *a, const void *b, const void *f, bool any_size = false)
{
    constexpr int V = 16 / sizeof(T);
    const long long lanes = (long long)sm_count() * 3 * kJThreads;
    if (!any_size && p.nx * p.ny * p.nz / V < 2 * lanes) return false;
    return p.nx % V == 0 && ((uintptr_t)a % 16) == 0 && ((uintptr_t)b % 16) == 0 && ((uintptr_t)f % 16) == 0;
}

template <class T> CUtensorMapDataType tma_type();
template <> CUtensorMapDataType tma_type<double>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT64; }
template <> CUtensorMapDataType tma_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> CUtensorMapDataType tma_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
template <> CUtensorMapDataType tma_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

// The TMA path: Dirichlet boundary with ghost +0 (the tensor maps' fill),
// rows of whole 16-byte groups, large grids.  Returns cudaErrorNotSupported
// when the problem does not qualify.
template <class T, int DIM>
cudaError_t run_tma(const Problem &p, LoopArgs la, cudaStream_t st)
{
    using Op = JacobiTma<T, DIM>;
    // SLR_TILING_TMA asks for the TMA path whatever the grid's size
    if (p.wrap || p.ghost != 0.0 || std::signbit(p.ghost) ||
        !vector_ok<T>(p, la.a, la.b, la.aux, p.tiling == SLR_TILING_TMA) || !tma::encode_fn())
        return cudaErrorNotSupported;
    Op op;
    memset(&op, 0, sizeof(op));
    const CUtensorMapDataType dt = tma_type<T>();
    const size_t es = sizeof(T);
    bool ok = true;
    for (int i = 0; i < 2; ++i) {
        const void *b = i == 0 ? la.a : la.b;
        if (DIM == 3) {
            ok = ok && tma::make_map_3d(&op.umap[i], b, dt, es, p.nx, p.ny, p.nz, Op::kTX, Op::kTY + 2, 1) &&
                 tma::make_map_3d(&op.smap[i], b, dt, es, p.nx, p.ny, p.nz, Op::V, Op::kTY, 1);
        } else {
            ok = ok && tma::make_map_2d(&op.umap[i], b, dt, es, p.nx, p.ny, Op::kTX, Op::kTY) &&
                 tma::make_map_2d(&op.smap[i], b, dt, es, p.nx, p.ny, Op::V, Op::kTY);
        }
    }
    ok = ok && (DIM == 3 ? tma::make_map_3d(&op.fmap, la.aux, dt, es, p.nx, p.ny, p.nz, Op::kTX, Op::kTY, 1)
                         : tma::make_map_2d(&op.fmap, la.aux, dt, es, p.nx, p.ny, Op::kTX, Op::kTY));
    if (!ok) return cudaErrorNotSupported;
    const auto sop = make_op<T, DIM, Op::V>(p, la.aux);
    op.base[0] = la.a;
    op.base[1] = la.b;
    op.err = &la.ctl->err;
    op.limit_ns = la.limit_ns;
    op.nx = (int)p.nx; op.ny = (int)p.ny; op.nz = (int)p.nz;
    op.tiles_x = (int)((p.nx + Op::kTX - 1) / Op::kTX);
    op.tiles_y = DIM == 3 ? (int)((p.ny + Op::kTY - 1) / Op::kTY) : 1;
    op.h2 = sop.h2; op.d = sop.d; op.yd = sop.yd; op.dconst = sop.dconst;
    auto kern = jacobi_persistent_kernel<Op>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Op::kSmem);
    if (e != cudaSuccess) return e;
    return launch_cooperative(kern, kJThreads, Op::kSmem, 3, la, &op, st);
}

template <class T, int DIM>
cudaError_t run_persistent(const Problem &p, LoopArgs la, cudaStream_t st)
{
    constexpr int V = 16 / sizeof(T);
    if (p.tiling != SLR_TILING_NONE) {
        const cudaError_t e = run_tma<T, DIM>(p, la, st);
        if (e != cudaErrorNotSupported) return e;
    }
    if (vector_ok<T>(p, la.a, la.b, la.aux)) {
        auto op = make_op<T, DIM, V>(p, la.aux);
        return launch_cooperative(jacobi_persistent_kernel<JacobiStream<T, DIM, V>>, kJThreads, 0, 3, la, &op, st);
    }
    auto op = make_op<T, DIM, 1>(p, la.aux);
    return launch_cooperative(jacobi_persistent_kernel<JacobiStream<T, DIM, 1>>, kJThreads, 0, 3, la, &op, st);
}

template <class T, int DIM>
cudaError_t run_sweep(const Problem &p, const void *src, void *dst, const void *f, cudaStream_t st)
{
    constexpr int V = 16 / sizeof(T);
    if (vector_ok<T>(p, src, dst, f)) {
        auto op = make_op<T, DIM, V>(p, f);
        jacobi_sweep_kernel<JacobiStream<T, DIM, V>><<<sm_count() * 3, kJThreads, 0, st>>>(op, src, dst);
    } else {
        auto op = make_op<T, DIM, 1>(p, f);
        jacobi_sweep_kernel<JacobiStream<T, DIM, 1>><<<sm_count() * 3, kJThreads, 0, st>>>(op, src, dst);
    }
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

bool jacobi_tma_ok(const Problem &p, const void *a, const void *b, const void *f, bool forced)
{
    if (p.wrap || p.ghost != 0.0 || std::signbit(p.ghost) || !tma::encode_fn()) return false;
    switch (p.storage) {
    case SLR_F64: return vector_ok<double>(p, a, b, f, forced);
    case SLR_F32: return vector_ok<float>(p, a, b, f, forced);
    case SLR_BF16: return vector_ok<__nv_bfloat16>(p, a, b, f, forced);
    case SLR_F16: return vector_ok<__half>(p, a, b, f, forced);
    default: return false;
    }
}

cudaError_t jacobi_persistent(const Problem &p, LoopArgs la, cudaStream_t st)
{
    return p.stencil == SLR_J3D7 ? dispatch_persistent<3>(p, la, st) : dispatch_persistent<2>(p, la, st);
}

cudaError_t jacobi_sweep(const Problem &p, const void *src, void *dst, const void *f, cudaStream_t st)
{
    return p.stencil == SLR_J3D7 ? dispatch_sweep<3>(p, src, dst, f, st) : dispatch_sweep<2>(p, src, dst, f, st);
}

}  // namespace slr
