// Device helpers shared by the detect-stage kernels: job lookup, tile
// staging into shared memory with 16-byte loads, and 4-pixel byte windows.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "of_internal.h"

namespace ofk {

// Index of the job that owns block `b`: the largest i with prefix[i] <= b.
__device__ __forceinline__ int find_tile_job(const int32_t* __restrict__ prefix, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Stage rows [y_first, y_first + rows) x columns [x_first, x_first + SROW) of a
// w x h uint8 image into shared memory (row stride SROW).  x_first is a
// multiple of 16, as are the image address and pitch, so every 16-byte chunk
// that lies inside the row is one aligned vector load.  Pixels outside the
// image are staged as 0 (they are never used by in-region outputs).
__device__ __forceinline__ void stage_tile(uint8_t* __restrict__ s, const uint8_t* __restrict__ img,
                                           int w, int h, int pitch, int x_first, int y_first,
                                           int rows) {
    constexpr int CPR = SROW / 16;  // chunks per row
    const int n = rows * CPR;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int r = i / CPR, k = i - r * CPR;
        const int iy = y_first + r, ix = x_first + 16 * k;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (iy >= 0 && iy < h && ix + 16 > 0 && ix < w) {
            const uint8_t* p = img + (size_t)iy * pitch + ix;
            if (ix >= 0 && ix + 16 <= w) {
                v = __ldg(reinterpret_cast<const uint4*>(p));
            } else {
                uint32_t wd[4] = {0u, 0u, 0u, 0u};
                for (int q = 0; q < 16; ++q) {
                    const int xx = ix + q;
                    if (xx >= 0 && xx < w) wd[q >> 2] |= (uint32_t)__ldg(p + q) << (8 * (q & 3));
                }
                v = make_uint4(wd[0], wd[1], wd[2], wd[3]);
            }
        }
        *reinterpret_cast<uint4*>(s + r * SROW + 16 * k) = v;
    }
}

// Four consecutive bytes starting `dx` bytes (-4..4) from the word `c`, given
// the words before (m) and after (p) it.
template <int DX>
__device__ __forceinline__ uint32_t win4(uint32_t m, uint32_t c, uint32_t p) {
    if constexpr (DX < 0) return __funnelshift_r(m, c, 8 * (4 + DX));
    else if constexpr (DX == 0) return c;
    else return __funnelshift_r(c, p, 8 * DX);
}

// Byte mask (0xFF per byte) of the bytes x..x+3 that fall inside [lo, hi).
__device__ __forceinline__ uint32_t range_mask4(int x, int lo, int hi) {
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (x + i >= lo && x + i < hi) m |= 0xFFu << (8 * i);
    return m;
}

// 0xFF in each byte of v that is >= t, for 1 <= t <= 128: (b | 0x80) - t has
// no borrow out of its byte and bit 7 set exactly when the low seven bits are
// >= t; a byte with bit 7 set is >= 128 >= t itself.  Five instructions.
__device__ __forceinline__ uint32_t bytes_ge(uint32_t v, uint32_t t) {
    const uint32_t g = (((v | 0x80808080u) - t * 0x01010101u) | v) & 0x80808080u;
    return (g >> 7) * 0xFFu;
}

// The same for any t <= 255, in 16-bit lanes.
__device__ __forceinline__ uint32_t bytes_ge_any(uint32_t v, uint32_t t) {
    const uint32_t tt = (0x8000u - t) * 0x00010001u;
    const uint32_t lo = __byte_perm(v, 0u, 0x4140) + tt, hi = __byte_perm(v, 0u, 0x4342) + tt;
    return __byte_perm((lo >> 15 & 0x00010001u) * 0xFFu, (hi >> 15 & 0x00010001u) * 0xFFu, 0x6420);
}

// Per-cell threshold on a word of offset scores: the bytes of v below t are
// cleared where fm is 0xFF (flagged cells).
__device__ __forceinline__ uint32_t apply_cell_threshold(uint32_t v, uint32_t fm, uint32_t t) {
    return v & ((t <= 128u ? bytes_ge(v, t) : bytes_ge_any(v, t)) | ~fm);
}

}  // namespace ofk
