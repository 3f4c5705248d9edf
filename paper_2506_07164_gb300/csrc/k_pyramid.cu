// Pyramid resize: level l is a bilinear resize of level l-1 (the pyramid of
// an ORB front end, Sec. 1; level sizes "decrease exponentially", Sec. 6.1).
//
// One launch resizes level l of every frame in the batch.  Each block owns a
// 128 x TH output tile (TH = 32 or 64, chosen by the autotuner): it stages the tile's source window in shared memory
// with aligned 16-byte loads (direct loads when the window is larger than the
// buffer, i.e. scales above ~2), then each thread writes 4 consecutive output
// pixels of TH/16 rows, one 32-bit store per row, with its 4 column weights kept
// in registers.  Source coordinates come from per-axis tables computed on
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

// Shared-memory source window: up to RS_SW x RS_SH bytes (enough for scales
// up to 2 with a 128 x 64 output tile).
constexpr int RS_SW = 288;
constexpr int RS_SH = 136;

__device__ __forceinline__ int bilerp(int p00, int p01, int p10, int p11, int ax, int ay) {
    const int top = (2048 - ax) * p00 + ax * p01;
    const int bot = (2048 - ax) * p10 + ax * p11;
    return ((2048 - ay) * top + ay * bot + (1 << 21)) >> 22;
}

template <int TH>
__global__ void __launch_bounds__(RS_THREADS)
k_resize(const Resize* __restrict__ jobs, const int32_t* __restrict__ prefix, int n_jobs) {
    constexpr int RS_RPT = TH / (RS_THREADS / 32);  // output rows per thread
    __shared__ __align__(16) uint8_t win[RS_SH * RS_SW];
    __shared__ int32_t yt[TH];
    __shared__ int32_t sjob, sx0s, sy0s, sbytes, srows;
    const int b = blockIdx.x;
    if (threadIdx.x == 0) sjob = find_job(prefix, n_jobs, b);
    __syncthreads();
    const int j = sjob;
    const Resize& J = jobs[j];
    const int t = b - __ldg(prefix + j);
    const int tx = t % J.tiles_x, ty = t / J.tiles_x;
    const int X0 = tx * RS_TILE_W, Y0 = ty * TH;
    const int nx = min(RS_TILE_W, J.dw - X0), ny = min(TH, J.dh - Y0);
    const int sw = J.sw, sh = J.sh;
    for (int i = threadIdx.x; i < TH; i += blockDim.x) yt[i] = i < ny ? __ldg(J.ytab + Y0 + i) : 0;
    if (threadIdx.x == 0) {
        // Source window of the tile: columns [sx0, sx1], rows [sy0, sy1].
        const int sx0 = (__ldg(J.xtab + X0) >> 12) & ~15;
        const int sx1 = min((__ldg(J.xtab + X0 + nx - 1) >> 12) + 1, sw - 1);
        const int sy0 = __ldg(J.ytab + Y0) >> 12;
        const int sy1 = min((__ldg(J.ytab + Y0 + ny - 1) >> 12) + 1, sh - 1);
        sx0s = sx0;
        sy0s = sy0;
        sbytes = ((sx1 - sx0) / 16 + 1) * 16;
        srows = sy1 - sy0 + 1;
    }
    __syncthreads();
    const int sx0 = sx0s, sy0 = sy0s, wbytes = sbytes, wrows = srows;
    const bool staged = wbytes <= RS_SW && wrows <= RS_SH;  // uniform per block
    if (staged) {
        const int cpr = wbytes / 16;
        for (int i = threadIdx.x; i < wrows * cpr; i += blockDim.x) {
            const int r = i / cpr, k = i - r * cpr;
            const int ix = sx0 + 16 * k;
            const uint8_t* p = J.src + (size_t)(sy0 + r) * J.spitch + ix;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (ix + 16 <= sw) {
                v = __ldg(reinterpret_cast<const uint4*>(p));  // src and spitch are 16-byte aligned
            } else {
                // Ragged end of the row: bytewise, in bounds.
                uint32_t w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
                for (int q = 0; q < 16 && ix + q < sw; ++q) {
                    const uint32_t byte = (uint32_t)__ldg(p + q) << (8 * (q & 3));
                    if (q < 4) w0 |= byte; else if (q < 8) w1 |= byte; else if (q < 12) w2 |= byte; else w3 |= byte;
                }
                v = make_uint4(w0, w1, w2, w3);
            }
            *reinterpret_cast<uint4*>(win + r * RS_SW + 16 * k) = v;
        }
    }
    __syncthreads();

    // Each thread: 4 consecutive columns, rows ly, ly + 16, ...
    const int lx = (threadIdx.x & 31) * 4, ly0 = threadIdx.x >> 5;
    if (lx >= nx) return;
    const int n = min(4, nx - lx);
    int x0[4], x1[4], ax[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int e = i < n ? __ldg(J.xtab + X0 + lx + i) : __ldg(J.xtab + X0 + lx);
        x0[i] = e >> 12;
        ax[i] = e & 4095;
        x1[i] = min(x0[i] + 1, sw - 1);
    }
#pragma unroll
    for (int rr = 0; rr < RS_RPT; ++rr) {
        const int ly = ly0 + rr * (RS_THREADS / 32);
        if (ly >= ny) break;
        const int y0 = yt[ly] >> 12, ay = yt[ly] & 4095;
        const int y1 = min(y0 + 1, sh - 1);
        uint32_t packed = 0;
        if (staged) {
            const uint8_t* r0 = win + (y0 - sy0) * RS_SW - sx0;
            const uint8_t* r1 = win + (y1 - sy0) * RS_SW - sx0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                packed |= (uint32_t)bilerp(r0[x0[i]], r0[x1[i]], r1[x0[i]], r1[x1[i]], ax[i], ay) << (8 * i);
        } else {
            const uint8_t* r0 = J.src + (size_t)y0 * J.spitch;
            const uint8_t* r1 = J.src + (size_t)y1 * J.spitch;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                packed |= (uint32_t)bilerp(__ldg(r0 + x0[i]), __ldg(r0 + x1[i]), __ldg(r1 + x0[i]),
                                           __ldg(r1 + x1[i]), ax[i], ay)
                          << (8 * i);
        }
        uint8_t* d = J.dst + (size_t)(Y0 + ly) * J.dpitch + X0 + lx;
        if (n == 4) {
            *reinterpret_cast<uint32_t*>(d) = packed;  // X0 + lx is a multiple of 4, dpitch of 16
        } else {
            for (int i = 0; i < n; ++i) d[i] = (uint8_t)(packed >> (8 * i));
        }
    }
}

void launch_resize(const Resize* jobs, const int32_t* tile_prefix, int n_jobs, int n_tiles, int tile_h,
                   void* stream) {
    if (n_tiles <= 0) return;
    if (tile_h == 32)
        k_resize<32><<<n_tiles, RS_THREADS, 0, (cudaStream_t)stream>>>(jobs, tile_prefix, n_jobs);
    else
        k_resize<64><<<n_tiles, RS_THREADS, 0, (cudaStream_t)stream>>>(jobs, tile_prefix, n_jobs);
}

}  // namespace ofk
