// restore_math.cuh -- the restoration update of one noisy pixel (Sec. 4.3) from
// its neighbours in a row-major array (shared memory), shared by the tiled
// one-sweep kernel (restore.cu) and the temporal-blocked one (restore_tb.cu).
//
//     t = u - u_j;  w_j = 1 / sqrt(alpha + t*t);  num += w_j*u_j;  den += w_j
//     u' = num / den
// over the in-range neighbours in row-major order (dy = -1..1, dx = -1..1,
// centre skipped).  EXACT: every operation rounds as the sequential binary32
// evaluation does (the weight from Markstein-corrected estimates, equal to
// __frcp_rn(__fsqrt_rn(x)); two neighbours per paired instruction for
// interior pixels, the sums still in row-major order).  FAST: the hardware
// reciprocal square root and fused multiply-adds.
#pragma once

#include "crmath.cuh"

namespace slr {

// one neighbour's term of the weighted mean
template <bool FAST>
__device__ __forceinline__ void restore_accumulate(float uc, float uj, float alpha, float &num, float &den)
{
    if (FAST) {
        const float w = rsqrtf(fmaf(uc - uj, uc - uj, alpha));
        num = fmaf(w, uj, num);
        den += w;
    } else {
        const float tt = __fsub_rn(uc, uj);
        const float w = inv_sqrt_rn2(__fadd_rn(alpha, __fmul_rn(tt, tt)));
        num = __fadd_rn(num, __fmul_rn(w, uj));
        den = __fadd_rn(den, w);
    }
}

template <bool FAST>
__device__ __forceinline__ float restore_quotient(float num, float den, float uc)
{
    return den > 0.0f ? (FAST ? __fdividef(num, den) : __fdiv_rn(num, den)) : uc;
}

// New value of a pixel all of whose 8 neighbours lie in the grid; C points at
// the pixel in an array of row pitch P.
template <bool FAST>
__device__ __forceinline__ float restore_interior(const float *C, int P, float alpha)
{
    const float uc = *C;
    float num = 0.0f, den = 0.0f;
    if (FAST) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (k != 4) restore_accumulate<true>(uc, C[(k / 3 - 1) * P + k % 3 - 1], alpha, num, den);
    } else {
        // neighbours in pairs (row-major order kept for the sums)
        float2 nd = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            const int k0 = k < 4 ? k : k + 1, k1 = k + 1 < 4 ? k + 1 : k + 2;
            const float u0 = C[(k0 / 3 - 1) * P + k0 % 3 - 1];
            const float u1 = C[(k1 / 3 - 1) * P + k1 % 3 - 1];
            const float2 w = weights_rn2(uc, u0, u1, alpha);
            nd = __fadd2_rn(nd, make_float2(__fmul_rn(w.x, u0), w.x));
            nd = __fadd2_rn(nd, make_float2(__fmul_rn(w.y, u1), w.y));
        }
        num = nd.x;
        den = nd.y;
    }
    return restore_quotient<FAST>(num, den, uc);
}

// EXACT new value of a pixel all of whose 8 neighbours lie in the grid, for
// states known to stay in range: alpha in [2^-100, 2^124) and every |u| below
// 2^61, so that every t = u - u_j has |t| < 2^62 and every x = alpha + t*t lies
// in [2^-100, 2^126), the weights' fast route, with no check per weight.  The
// same operations in the same order as restore_interior<false>.
__device__ __forceinline__ float restore_interior_in_range(const float *C, int P, float alpha)
{
    const float uc = *C;
    float2 nd = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        const int k0 = k < 4 ? k : k + 1, k1 = k + 1 < 4 ? k + 1 : k + 2;
        const float u0 = C[(k0 / 3 - 1) * P + k0 % 3 - 1];
        const float u1 = C[(k1 / 3 - 1) * P + k1 % 3 - 1];
        const float2 w = weights_rn2_in_range(uc, u0, u1, alpha);
        nd = __fadd2_rn(nd, make_float2(__fmul_rn(w.x, u0), w.x));
        nd = __fadd2_rn(nd, make_float2(__fmul_rn(w.y, u1), w.y));
    }
    return restore_quotient<false>(nd.x, nd.y, uc);
}

// Whether alpha lets restore_interior_in_range run (states below 2^61 in magnitude).
__host__ __device__ __forceinline__ bool restore_alpha_in_range(float alpha)
{
    return alpha >= 0x1p-100f && alpha < 0x1p124f;
}

// New value of a pixel on the grid's border: the neighbours outside the grid
// (up: the row above exists, and so on) are left out of both sums.
template <bool FAST>
__device__ __forceinline__ float restore_border(const float *C, int P, float alpha, bool up, bool down, bool left,
                                                bool right)
{
    const float uc = *C;
    float num = 0.0f, den = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int di = k / 3 - 1, dj = k % 3 - 1;
        if (k == 4 || (di < 0 && !up) || (di > 0 && !down) || (dj < 0 && !left) || (dj > 0 && !right)) continue;
        restore_accumulate<FAST>(uc, C[di * P + dj], alpha, num, den);
    }
    return restore_quotient<FAST>(num, den, uc);
}

}  // namespace slr
