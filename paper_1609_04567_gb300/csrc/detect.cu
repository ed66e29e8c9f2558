// detect.cu -- adaptive median noise detection: the detection phase of the
// two-phase restoration of Sec. 4.3, which feeds RESTORE8 its noisy-pixel mask.
//
// The paper names a traditional adaptive median filter without defining it;
// this is the textbook filter.  For the pixel z, square windows of side
// 3, 5, ..., wmax centred on it and clipped to the image give zmin, zmax and
// zmed, the lower median (element floor((n - 1) / 2) of the n window values
// in ascending order).  The first window with zmin < zmed < zmax decides: the
// filter outputs z when zmin < z < zmax, else zmed; when no window qualifies
// it outputs zmed of the largest window.  A pixel is noisy (mask 1) where the
// output differs from z.
//
// One thread per pixel of a 32 x 8 block; the block's pixels and a halo of
// wmax / 2 on every side are staged in shared memory.  A window's median is
// found bit by bit from the most significant: the m-th smallest value is the
// largest v with at most m values below it (8 counting passes over the
// window, the first one also taking the minimum and maximum).  Integer only:
// the mask equals the oracle's bit for bit.  The same pass can write the
// frame as the restoration's binary32 state; a second kernel turns a
// restored state back into a uint8 frame (round to nearest even, clamped).
#include <string>

#include "crmath.cuh"
#include "slr_internal.cuh"

namespace slr {

void set_handleless_error(const std::string &msg);   // slr_api.cu: slr_last_error(NULL)

namespace {

constexpr int kDX = 32, kDY = 8;                 // pixels per block
constexpr int kMaxW = 15;                        // largest window side accepted
constexpr int kMaxR = kMaxW / 2;
constexpr int kTileX = kDX + 2 * kMaxR, kTileY = kDY + 2 * kMaxR;

__global__ void __launch_bounds__(kDX * kDY) amf_detect_kernel(const unsigned char *img, unsigned char *mask,
                                                               float *state, int nx, int ny, int wmax)
{
    __shared__ unsigned char tile[kTileY][kTileX];
    const int R = wmax / 2;
    const int bx = blockIdx.x * kDX, by = blockIdx.y * kDY;
    const int tid = threadIdx.y * kDX + threadIdx.x;
    // the block's pixels with a halo of R (cells outside the image are never read)
    const int tw = kDX + 2 * R, th = kDY + 2 * R;
    for (int k = tid; k < tw * th; k += kDX * kDY) {
        const int ty = k / tw, tx = k - ty * tw;
        const int gy = by - R + ty, gx = bx - R + tx;
        tile[ty][tx] = gy >= 0 && gy < ny && gx >= 0 && gx < nx ? img[(size_t)gy * nx + gx] : 0;
    }
    __syncthreads();
    const int i = by + threadIdx.y, j = bx + threadIdx.x;
    if (i >= ny || j >= nx) return;
    const int ci = threadIdx.y + R, cj = threadIdx.x + R;   // the pixel in the tile
    const int z = tile[ci][cj];
    int out = -1, zmed = z;
    for (int r = 1; r <= R; ++r) {
        // the window clipped to the image, in tile coordinates
        const int a0 = ci - (i - r < 0 ? i : r), a1 = ci + (i + r >= ny ? ny - 1 - i : r);
        const int b0 = cj - (j - r < 0 ? j : r), b1 = cj + (j + r >= nx ? nx - 1 - j : r);
        const int n = (a1 - a0 + 1) * (b1 - b0 + 1), m = (n - 1) / 2;
        int zmin = 255, zmax = 0, v = 0;
        for (int bit = 7; bit >= 0; --bit) {
            const int cand = v | (1 << bit);
            int below = 0;
            for (int a = a0; a <= a1; ++a)
                for (int b = b0; b <= b1; ++b) {
                    const int x = tile[a][b];
                    below += x < cand;
                    if (bit == 7) {
                        zmin = min(zmin, x);
                        zmax = max(zmax, x);
                    }
                }
            if (below <= m) v = cand;
        }
        zmed = v;
        if (zmin < zmed && zmed < zmax) {
            out = zmin < z && z < zmax ? z : zmed;
            break;
        }
    }
    if (out < 0) out = zmed;
    mask[(size_t)i * nx + j] = (unsigned char)(out != z);
    if (state) state[(size_t)i * nx + j] = (float)z;
}

__global__ void state_to_frame_kernel(const float *u, unsigned char *img, size_t n)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const float v = rintf(u[k]);
        img[k] = (unsigned char)(v >= 255.0f ? 255.0f : (v > 0.0f ? v : 0.0f));   // NaN -> 0
    }
}

}  // namespace
}  // namespace slr

extern "C" {

slr_status slr_detect_noise(const void *img, void *mask, void *state, int64_t nx, int64_t ny, int32_t wmax,
                            void *stream)
{
    if (!img || !mask) {
        slr::set_handleless_error("slr_detect_noise: img and mask must be device pointers");
        return SLR_ERR_INVALID_ARG;
    }
    if (nx < 1 || ny < 1 || nx >= (1ll << 31) || ny >= (1ll << 31)) {
        slr::set_handleless_error("slr_detect_noise: nx and ny must lie in [1, 2^31)");
        return SLR_ERR_INVALID_ARG;
    }
    if (wmax < 3 || wmax > slr::kMaxW || wmax % 2 == 0) {
        slr::set_handleless_error("slr_detect_noise: wmax must be odd, 3 .. 15");
        return SLR_ERR_INVALID_ARG;
    }
    const size_t bytes = (size_t)nx * (size_t)ny;
    const uintptr_t pi = (uintptr_t)img, pm = (uintptr_t)mask;
    const uintptr_t ps = (uintptr_t)state;
    if ((pi < pm + bytes && pm < pi + bytes) ||
        (state && ((ps < pi + bytes && pi < ps + 4 * bytes) || (ps < pm + bytes && pm < ps + 4 * bytes)))) {
        slr::set_handleless_error("slr_detect_noise: img, mask and state overlap");
        return SLR_ERR_INVALID_ARG;
    }
    if (ps % 4 != 0) {
        slr::set_handleless_error("slr_detect_noise: state must be 4-byte aligned");
        return SLR_ERR_INVALID_ARG;
    }
    const dim3 grid((unsigned)((nx + slr::kDX - 1) / slr::kDX), (unsigned)((ny + slr::kDY - 1) / slr::kDY));
    if (grid.y > 65535u) {
        slr::set_handleless_error("slr_detect_noise: ny above 524280 rows");
        return SLR_ERR_INVALID_ARG;
    }
    slr::amf_detect_kernel<<<grid, dim3(slr::kDX, slr::kDY), 0, (cudaStream_t)stream>>>(
        (const unsigned char *)img, (unsigned char *)mask, (float *)state, (int)nx, (int)ny, wmax);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        slr::set_handleless_error(std::string("slr_detect_noise: launch: ") + cudaGetErrorString(e));
        return SLR_ERR_CUDA;
    }
    return SLR_OK;
}

slr_status slr_state_to_frame(const void *state, void *img, int64_t n, void *stream)
{
    if (!state || !img || n < 0 || (uintptr_t)state % 4 != 0) {
        slr::set_handleless_error("slr_state_to_frame: state (4-byte aligned) and img must be device pointers, n >= 0");
        return SLR_ERR_INVALID_ARG;
    }
    if (n == 0) return SLR_OK;
    const int threads = 256;
    const long long want = (n + threads - 1) / threads;
    const unsigned blocks = (unsigned)(want < 152 * 8 ? want : 152 * 8);
    slr::state_to_frame_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>((const float *)state,
                                                                            (unsigned char *)img, (size_t)n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        slr::set_handleless_error(std::string("slr_state_to_frame: launch: ") + cudaGetErrorString(e));
        return SLR_ERR_CUDA;
    }
    return SLR_OK;
}

}  // extern "C"

// ---- Sobel edge detector (Sec. 4.2) --------------------------------------------
// One 3x3 stencil sweep with no reduce: the gradients
//   Gx = V1[j+1] - V1[j-1],  V1 = z[i-1] + 2 z[i] + z[i+1]   (per column)
//   Gy = V2[j-1] + 2 V2[j] + V2[j+1],  V2 = z[i+1] - z[i-1]
// in integers, out = min(255, floor(sqrt(Gx^2 + Gy^2))) inside, 0 on the
// image's border.  A warp owns a strip of 256 columns (8 consecutive pixels
// per lane, one 8-byte access per row) and marches down a segment of rows,
// keeping rows i-1, i, i+1 unpacked in registers (three rows per turn, no
// copies), each row's bytes loaded one row ahead of their use: each pixel is
// read from memory once and written once.  The
// neighbours across lanes come by shuffles of the column sums; the strip's two
// outer columns by single loads.  The clamped integer square root is the
// hardware estimate of sqrt(n + 1/2), truncated (exact: isqrt_clamp255).
namespace slr {
namespace {

constexpr int kPx = 8;                            // pixels per lane (one 8-byte access per row)
constexpr int kPW = kPx / 4;                      // 32-bit words per lane and row
constexpr int kSobelStrip = 32 * kPx;             // columns per warp
constexpr int kSobelWarps = 8;

// the lane's 8 bytes of row y (0 outside the image)
__device__ __forceinline__ uint2 sobel_raw(const unsigned char *img, int nx, int ny, int y, int x0, bool vec)
{
    if (y < 0 || y >= ny || x0 >= nx) return make_uint2(0u, 0u);
    const unsigned char *row = img + (size_t)y * nx;
    if (vec) return *(const uint2 *)(row + x0);
    uint32_t w[2] = {0u, 0u};
    for (int k = 0; k < kPx && x0 + k < nx; ++k) w[k >> 2] |= (uint32_t)row[x0 + k] << (8 * (k & 3));
    return make_uint2(w[0], w[1]);
}

__device__ __forceinline__ void unpack8(uint2 r, int (&v)[kPx])
{
#pragma unroll
    for (int k = 0; k < kPx; ++k) v[k] = ((k < 4 ? r.x : r.y) >> (8 * (k & 3))) & 0xFFu;
}

// output row y of the lane's pixels from rows y-1 (a), y (c), y+1 (b);
// keep[] clears the bytes of the image's first and last columns
__device__ __forceinline__ void sobel_row(const unsigned char *img, unsigned char *out, int nx, int ny, int y,
                                          int x0, bool vec, const uint32_t (&keep)[kPW], const int (&a)[kPx],
                                          const int (&c)[kPx], const int (&b)[kPx])
{
    const int lane = threadIdx.x & 31;
    int v1[kPx], v2[kPx];
#pragma unroll
    for (int k = 0; k < kPx; ++k) {
        v1[k] = a[k] + 2 * c[k] + b[k];
        v2[k] = b[k] - a[k];
    }
    // the column sums left of the lane's first pixel and right of its last
    int l1 = __shfl_up_sync(0xffffffffu, v1[kPx - 1], 1), l2 = __shfl_up_sync(0xffffffffu, v2[kPx - 1], 1);
    int r1 = __shfl_down_sync(0xffffffffu, v1[0], 1), r2 = __shfl_down_sync(0xffffffffu, v2[0], 1);
    if (y == 0 || y == ny - 1 || x0 >= nx) {
        if (x0 < nx) {
            unsigned char *o = out + (size_t)y * nx;
            if (vec) *(uint2 *)(o + x0) = make_uint2(0u, 0u);
            else
                for (int k = 0; k < kPx && x0 + k < nx; ++k) o[x0 + k] = 0;
        }
        return;
    }
    if (lane == 0 && x0 > 0) {
        const size_t i = (size_t)y * nx + x0 - 1;
        const int za = img[i - nx], zc = img[i], zb = img[i + nx];
        l1 = za + 2 * zc + zb;
        l2 = zb - za;
    }
    if (lane == 31 && x0 + kPx < nx) {
        const size_t i = (size_t)y * nx + x0 + kPx;
        const int za = img[i - nx], zc = img[i], zb = img[i + nx];
        r1 = za + 2 * zc + zb;
        r2 = zb - za;
    }
    uint32_t w[kPW];
#pragma unroll
    for (int q = 0; q < kPW; ++q) w[q] = 0u;
#pragma unroll
    for (int k = 0; k < kPx; ++k) {
        const int p1 = k > 0 ? v1[k - 1] : l1, n1 = k < kPx - 1 ? v1[k + 1] : r1;
        const int p2 = k > 0 ? v2[k - 1] : l2, n2 = k < kPx - 1 ? v2[k + 1] : r2;
        const int gx = n1 - p1, gy = p2 + 2 * v2[k] + n2;
        w[k >> 2] |= (uint32_t)isqrt_clamp255(gx * gx + gy * gy) << (8 * (k & 3));
    }
#pragma unroll
    for (int q = 0; q < kPW; ++q) w[q] &= keep[q];
    unsigned char *o = out + (size_t)y * nx;
    if (vec) {
        *(uint2 *)(o + x0) = make_uint2(w[0], w[1]);
    } else {
#pragma unroll
        for (int k = 0; k < kPx; ++k)
            if (x0 + k < nx) o[x0 + k] = (unsigned char)(w[k >> 2] >> (8 * (k & 3)));
    }
}

__global__ void __launch_bounds__(32 * kSobelWarps) sobel_kernel(const unsigned char *img, unsigned char *out,
                                                                 int nx, int ny, int seg_rows, int aligned)
{
    const int lane = threadIdx.x & 31;
    const long long unit = (long long)blockIdx.x * kSobelWarps + (threadIdx.x >> 5);
    const int strips = (nx + kSobelStrip - 1) / kSobelStrip;
    const long long units = (long long)strips * ((ny + seg_rows - 1) / seg_rows);
    if (unit >= units) return;
    const int strip = (int)(unit % strips), seg = (int)(unit / strips);
    const int x0 = strip * kSobelStrip + lane * kPx;
    const int y0 = seg * seg_rows, y1 = min(ny, y0 + seg_rows);
    // whole 8-byte groups inside the row, and 8-byte aligned rows
    const bool vec = aligned && x0 + kPx <= nx;
    uint32_t keep[kPW];
#pragma unroll
    for (int q = 0; q < kPW; ++q) keep[q] = ~0u;
#pragma unroll
    for (int k = 0; k < kPx; ++k)
        if (x0 + k == 0 || x0 + k == nx - 1) keep[k >> 2] &= ~(0xFFu << (8 * (k & 3)));
    int R0[kPx], R1[kPx], R2[kPx];
    unpack8(sobel_raw(img, nx, ny, y0 - 1, x0, vec), R0);
    unpack8(sobel_raw(img, nx, ny, y0, x0, vec), R1);
    // the next row's bytes are loaded one row ahead of their use
    uint2 nxt = sobel_raw(img, nx, ny, y0 + 1, x0, vec);
    for (int y = y0; y < y1; y += 3) {
        unpack8(nxt, R2);
        nxt = sobel_raw(img, nx, ny, y + 2, x0, vec);
        sobel_row(img, out, nx, ny, y, x0, vec, keep, R0, R1, R2);
        if (y + 1 >= y1) break;
        unpack8(nxt, R0);
        nxt = sobel_raw(img, nx, ny, y + 3, x0, vec);
        sobel_row(img, out, nx, ny, y + 1, x0, vec, keep, R1, R2, R0);
        if (y + 2 >= y1) break;
        unpack8(nxt, R1);
        nxt = sobel_raw(img, nx, ny, y + 4, x0, vec);
        sobel_row(img, out, nx, ny, y + 2, x0, vec, keep, R2, R0, R1);
    }
}

}  // namespace
}  // namespace slr

extern "C" {

slr_status slr_sobel(const void *img, void *out, int64_t nx, int64_t ny, void *stream)
{
    if (!img || !out) {
        slr::set_handleless_error("slr_sobel: img and out must be device pointers");
        return SLR_ERR_INVALID_ARG;
    }
    if (nx < 1 || ny < 1 || nx >= (1ll << 31) - 4096 || ny >= (1ll << 31)) {
        slr::set_handleless_error("slr_sobel: nx and ny must lie in [1, 2^31 - 4096)");
        return SLR_ERR_INVALID_ARG;
    }
    const size_t bytes = (size_t)nx * (size_t)ny;
    const uintptr_t pi = (uintptr_t)img, po = (uintptr_t)out;
    if (pi < po + bytes && po < pi + bytes) {
        slr::set_handleless_error("slr_sobel: img and out overlap");
        return SLR_ERR_INVALID_ARG;
    }
    // segments of rows: about four warps' worth of work per SM slot, at least 16 rows
    const long long strips = (nx + slr::kSobelStrip - 1) / slr::kSobelStrip;
    long long seg = ny * strips / (152 * 64 * 4);
    seg = seg < 16 ? 16 : (seg > 1024 ? 1024 : seg);
    const long long units = strips * ((ny + seg - 1) / seg);
    const long long blocks = (units + slr::kSobelWarps - 1) / slr::kSobelWarps;
    if (blocks > 0x7FFFFFFFll) {
        slr::set_handleless_error("slr_sobel: image too large");
        return SLR_ERR_INVALID_ARG;
    }
    const int aligned = nx % 8 == 0 && pi % 8 == 0 && po % 8 == 0;
    slr::sobel_kernel<<<(unsigned)blocks, 32 * slr::kSobelWarps, 0, (cudaStream_t)stream>>>(
        (const unsigned char *)img, (unsigned char *)out, (int)nx, (int)ny, (int)seg, aligned);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        slr::set_handleless_error(std::string("slr_sobel: launch: ") + cudaGetErrorString(e));
        return SLR_ERR_CUDA;
    }
    return SLR_OK;
}

}  // extern "C"
