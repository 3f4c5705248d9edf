// Pyramid resize: level l is a bilinear resize of level l-1 (the pyramid of
// an ORB front end, Sec. 1; level sizes "decrease exponentially", Sec. 6.1).
//
// One launch resizes level l of every frame in the batch.  Each block owns a
// 128 x 16 output tile: it stages the tile's source window in shared memory
// with aligned 16-byte loads (direct loads when the window is larger than the
// buffer, i.e. scales above ~2), then each thread writes 4 consecutive output
// pixels with one 32-bit store.  Source coordinates come from per-axis tables computed on
// the host: (i0 << 12) | a, a in [0, 2048] the weight of sample i0 + 1 in
// units of 1/2048; one rounding at the end:
//   out = ((2048-ay)((2048-ax)p00 + ax p01) + ay((2048-ax)p10 + ax p11) + 2^21) >> 22.
// Exact int32 arithmetic: the largest intermediate is 2048*2048*255 < 2^31.
#include <cuda_runtime.h>

#include "of_internal.h"

namespace ofk {

__device__ __forceinline__ int find_job(const int32_t* __restrict__ prefix, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Shared-memory source window: up to RS_SW x RS_SH bytes (scale up to ~2).
constexpr int RS_SW = 288;
constexpr int RS_SH = 40;

__device__ __forceinline__ int bilerp(int p00, int p01, int p10, int p11, int ax, int ay) {
    const int top = (2048 - ax) * p00 + ax * p01;
    const int bot = (2048 - ax) * p10 + ax * p11;
    return ((2048 - ay) * top + ay * bot + (1 << 21)) >> 22;
}

__global__ void __launch_bounds__(RS_THREADS)
k_resize(const Resize* __restrict__ jobs, const int32_t* __restrict__ prefix, int n_jobs) {
    __shared__ __align__(16) uint8_t win[RS_SH * RS_SW];
    __shared__ int32_t xt[RS_TILE_W], yt[RS_TILE_H];
    const int b = blockIdx.x;
    const int j = find_job(prefix, n_jobs, b);
    const Resize J = jobs[j];
    const int t = b - __ldg(prefix + j);
    const int tx = t % J.tiles_x, ty = t / J.tiles_x;
    const int X0 = tx * RS_TILE_W, Y0 = ty * RS_TILE_H;
    const int nx = min(RS_TILE_W, J.dw - X0), ny = min(RS_TILE_H, J.dh - Y0);
    for (int i = threadIdx.x; i < RS_TILE_W + RS_TILE_H; i += blockDim.x) {
        if (i < RS_TILE_W) xt[i] = i < nx ? __ldg(J.xtab + X0 + i) : 0;
        else yt[i - RS_TILE_W] = (i - RS_TILE_W) < ny ? __ldg(J.ytab + Y0 + i - RS_TILE_W) : 0;
    }
    __syncthreads();
    // Source window of the tile: columns [sx0, sx1], rows [sy0, sy1].
    const int sx0 = (xt[0] >> 12) & ~15;
    const int sx1 = min((xt[nx - 1] >> 12) + 1, J.sw - 1);
    const int sy0 = yt[0] >> 12;
    const int sy1 = min((yt[ny - 1] >> 12) + 1, J.sh - 1);
    const int wbytes = ((sx1 - sx0) / 16 + 1) * 16;
    const int wrows = sy1 - sy0 + 1;
    const bool staged = wbytes <= RS_SW && wrows <= RS_SH;  // uniform per block
    if (staged) {
        const int cpr = wbytes / 16;
        for (int i = threadIdx.x; i < wrows * cpr; i += blockDim.x) {
            const int r = i / cpr, k = i - r * cpr;
            const int ix = sx0 + 16 * k;
            const uint8_t* p = J.src + (size_t)(sy0 + r) * J.spitch + ix;
            uint4 v;
            if (ix + 16 <= J.sw) {
                v = __ldg(reinterpret_cast<const uint4*>(p));  // src and spitch are 16-byte aligned
            } else {
                uint32_t wd[4] = {0u, 0u, 0u, 0u};
                for (int q = 0; q < 16 && ix + q < J.sw; ++q) wd[q >> 2] |= (uint32_t)__ldg(p + q) << (8 * (q & 3));
                v = make_uint4(wd[0], wd[1], wd[2], wd[3]);
            }
            *reinterpret_cast<uint4*>(win + r * RS_SW + 16 * k) = v;
        }
    }
    __syncthreads();

    const int lx = (threadIdx.x & 31) * 4, ly = threadIdx.x >> 5;
    if (ly >= ny || lx >= nx) return;
    const int y = Y0 + ly, x = X0 + lx;
    const int y0 = yt[ly] >> 12, ay = yt[ly] & 4095;
    const int y1 = min(y0 + 1, J.sh - 1);
    const int n = min(4, nx - lx);
    uint32_t packed = 0;
    if (staged) {
        const uint8_t* r0 = win + (y0 - sy0) * RS_SW - sx0;
        const uint8_t* r1 = win + (y1 - sy0) * RS_SW - sx0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < n) {
                const int e = xt[lx + i];
                const int x0 = e >> 12, ax = e & 4095, x1 = min(x0 + 1, J.sw - 1);
                packed |= (uint32_t)bilerp(r0[x0], r0[x1], r1[x0], r1[x1], ax, ay) << (8 * i);
            }
        }
    } else {
        const uint8_t* r0 = J.src + (size_t)y0 * J.spitch;
        const uint8_t* r1 = J.src + (size_t)y1 * J.spitch;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < n) {
                const int e = xt[lx + i];
                const int x0 = e >> 12, ax = e & 4095, x1 = min(x0 + 1, J.sw - 1);
                packed |= (uint32_t)bilerp(__ldg(r0 + x0), __ldg(r0 + x1), __ldg(r1 + x0), __ldg(r1 + x1), ax, ay)
                          << (8 * i);
            }
        }
    }
    uint8_t* d = J.dst + (size_t)y * J.dpitch + x;
    if (n == 4) {
        *reinterpret_cast<uint32_t*>(d) = packed;  // x % 4 == 0, dpitch % 16 == 0
    } else {
        for (int i = 0; i < n; ++i) d[i] = (uint8_t)(packed >> (8 * i));
    }
}

void launch_resize(const Resize* jobs, const int32_t* tile_prefix, int n_jobs, int n_tiles,
                   void* stream) {
    if (n_tiles <= 0) return;
    k_resize<<<n_tiles, RS_THREADS, 0, (cudaStream_t)stream>>>(jobs, tile_prefix, n_jobs);
}

}  // namespace ofk
