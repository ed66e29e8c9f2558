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
