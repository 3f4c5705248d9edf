// Pyramid resize: level l is a bilinear resize of level l-1 (the pyramid of
// an ORB front end, Sec. 1; level sizes "decrease exponentially", Sec. 6.1).
//
// One launch resizes level l of every frame in the batch.  Each block owns a
// 128 x 16 output tile; each thread writes 4 consecutive output pixels with
// one 32-bit store.  Source coordinates come from per-axis tables computed on
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

__global__ void __launch_bounds__(RS_THREADS)
k_resize(const Resize* __restrict__ jobs, const int32_t* __restrict__ prefix, int n_jobs) {
    const int b = blockIdx.x;
    const int j = find_job(prefix, n_jobs, b);
    const Resize J = jobs[j];
    const int t = b - __ldg(prefix + j);
    const int tx = t % J.tiles_x, ty = t / J.tiles_x;
    const int x = tx * RS_TILE_W + (threadIdx.x & 31) * 4;
    const int y = ty * RS_TILE_H + (threadIdx.x >> 5);
    if (y >= J.dh || x >= J.dw) return;

    const int yt = __ldg(J.ytab + y);
    const int y0 = yt >> 12, ay = yt & 4095;
    const int y1 = min(y0 + 1, J.sh - 1);
    const uint8_t* r0 = J.src + (size_t)y0 * J.spitch;
    const uint8_t* r1 = J.src + (size_t)y1 * J.spitch;
    const int n = min(4, J.dw - x);
    uint32_t packed = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i < n) {
            const int xt = __ldg(J.xtab + x + i);
            const int x0 = xt >> 12, ax = xt & 4095;
            const int x1 = min(x0 + 1, J.sw - 1);
            const int p00 = __ldg(r0 + x0), p01 = __ldg(r0 + x1);
            const int p10 = __ldg(r1 + x0), p11 = __ldg(r1 + x1);
            const int top = (2048 - ax) * p00 + ax * p01;
            const int bot = (2048 - ax) * p10 + ax * p11;
            const int v = ((2048 - ay) * top + ay * bot + (1 << 21)) >> 22;
            packed |= (uint32_t)v << (8 * i);
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
