// FAST-9 segment test with a score (Eq. 1, Sec. 3.1; binary encoding of
// Alg. 2 / Fig. 3), byte-parallel: one 32-bit register carries the same ring
// pixel of 4 horizontally adjacent centres.
//
// Score.  Eq. 1 calls ring pixel I_i bright when I_i >= I_p + t and dark when
// I_i <= I_p - t; p is a corner at t when 9 contiguous ring pixels are all
// bright or all dark.  The largest such t is
//   s(p) = max( max_j min_{k<9} I_{j+k} - I_p ,  I_p - min_j max_{k<9} I_{j+k} )
// (the I_p terms leave the min/max), so corner(t) <=> s(p) >= t for t >= 1.
// Both arc terms are computed once for all 4 pixels with byte-wise min/max:
// minima of 2, 4, 8 contiguous pixels by doubling, then the 9th pixel.  The
// map stores s(p) where s(p) >= t_lo (the lowest threshold in use), else 0.
//
// Per-cell fallback: a cell with any pixel scoring >= t_hi is flagged
// (shared-memory flags per tile, then one global atomicOr per flagged cell).
#include <cuda_runtime.h>

#include "of_internal.h"
#include "of_tile.cuh"

namespace ofk {

// The 16 ring offsets of Fig. 2(a) in cyclic order.
#define OF_RING(R)                                                                        \
    R(0, 0, -3) R(1, 1, -3) R(2, 2, -2) R(3, 3, -1) R(4, 3, 0) R(5, 3, 1) R(6, 2, 2)      \
    R(7, 1, 3) R(8, 0, 3) R(9, -1, 3) R(10, -2, 2) R(11, -3, 1) R(12, -3, 0) R(13, -3, -1) \
    R(14, -2, -2) R(15, -1, -3)

// s(p) for 4 adjacent centres.  q[i] = ring pixel i of the 4 centres, c = centres.
__device__ __forceinline__ uint32_t fast_score4(const uint32_t (&q)[16], uint32_t c) {
    uint32_t lo2[16], hi2[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        lo2[i] = __vminu4(q[i], q[(i + 1) & 15]);
        hi2[i] = __vmaxu4(q[i], q[(i + 1) & 15]);
    }
    uint32_t lo4[16], hi4[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        lo4[i] = __vminu4(lo2[i], lo2[(i + 2) & 15]);
        hi4[i] = __vmaxu4(hi2[i], hi2[(i + 2) & 15]);
    }
    uint32_t lo8[16], hi8[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        lo8[i] = __vminu4(lo4[i], lo4[(i + 4) & 15]);
        hi8[i] = __vmaxu4(hi4[i], hi4[(i + 4) & 15]);
    }
    uint32_t arc_min_max = 0u, arc_max_min = 0xFFFFFFFFu;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        arc_min_max = __vmaxu4(arc_min_max, __vminu4(lo8[i], q[(i + 8) & 15]));
        arc_max_min = __vminu4(arc_max_min, __vmaxu4(hi8[i], q[(i + 8) & 15]));
    }
    return __vmaxu4(__vsubus4(arc_min_max, c), __vsubus4(c, arc_max_min));
}

__global__ void __launch_bounds__(DET_THREADS)
k_fast(const Img* __restrict__ imgs, const int32_t* __restrict__ list,
       const int32_t* __restrict__ prefix, int n_list, int t_hi, int t_lo, int border, int cell) {
    __shared__ __align__(16) uint8_t s[(TILE_H + 6) * SROW];
    __shared__ uint32_t sflag[MAX_CELLS_LOCAL];

    const int b = blockIdx.x;
    const int j = find_tile_job(prefix, n_list, b);
    const Img& I = imgs[__ldg(list + j)];
    const int w = I.w, h = I.h;
    const int t = b - __ldg(prefix + j);
    const int tx = t % I.tiles_x, ty_tile = t / I.tiles_x;
    const int X0 = I.tile_x0 + tx * TILE_W;
    const int Y0 = border + ty_tile * TILE_H;
    const bool cells = t_hi != t_lo;

    // Cells overlapping this tile: columns [cx0, ...), rows [cy0, ...).
    const int rx0 = border, rx1 = w - border, ry1 = h - border;
    const int cx0 = (max(X0, rx0) - rx0) / cell;
    const int cy0 = (Y0 - border) / cell;
    const int lcw = TILE_W / cell + 2;
    if (cells) {
        for (int i = threadIdx.x; i < MAX_CELLS_LOCAL; i += blockDim.x) sflag[i] = 0u;
    }
    stage_tile(s, I.img, w, h, I.pitch, X0 - HALO_X, Y0 - 3, TILE_H + 6);
    __syncthreads();

    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int x = X0 + 4 * lane;
    uint32_t wm[RPT + 6], wc[RPT + 6], wp[RPT + 6];
#pragma unroll
    for (int k = 0; k < RPT + 6; ++k) {
        const uint8_t* row = s + (ty * RPT + k) * SROW + HALO_X + 4 * lane;
        wm[k] = *reinterpret_cast<const uint32_t*>(row - 4);
        wc[k] = *reinterpret_cast<const uint32_t*>(row);
        wp[k] = *reinterpret_cast<const uint32_t*>(row + 4);
    }
    const uint32_t colmask = range_mask4(x, rx0, rx1);
    const uint32_t tlo4 = 0x01010101u * (uint32_t)t_lo;
    const uint32_t thi4 = 0x01010101u * (uint32_t)t_hi;

#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int y = Y0 + ty * RPT + r;
        uint32_t q[16];
#define OF_LOAD_RING(i, dx, dy) q[i] = win4<dx>(wm[r + 3 + (dy)], wc[r + 3 + (dy)], wp[r + 3 + (dy)]);
        OF_RING(OF_LOAD_RING)
#undef OF_LOAD_RING
        const uint32_t c = wc[r + 3];
        uint32_t sc = fast_score4(q, c);
        const uint32_t m = (y < ry1) ? colmask : 0u;
        sc &= __vcmpgeu4(sc, tlo4) & m;
        if (m != 0u) *reinterpret_cast<uint32_t*>(I.score + (size_t)y * I.spitch + x) = sc;
        if (cells) {
            const uint32_t strong = __vcmpgeu4(sc, thi4) & m;
            if (strong) {
                const int cyl = (y - border) / cell - cy0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if ((strong >> (8 * i)) & 1u) {
                        const int cxl = (x + i - rx0) / cell - cx0;
                        atomicOr(&sflag[cyl * lcw + cxl], 1u);
                    }
                }
            }
        }
    }
    if (cells) {
        __syncthreads();
        const int lch = TILE_H / cell + 2;
        for (int i = threadIdx.x; i < lcw * lch; i += blockDim.x) {
            if (sflag[i]) {
                const int cx = cx0 + i % lcw, cy = cy0 + i / lcw;
                if (cx < I.ncx && cy < I.ncy) atomicOr(&I.cell[cy * I.ncx + cx], 1u);
            }
        }
    }
}

void launch_fast(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix, int n_list,
                 int n_tiles, const Call*, int t_hi, int t_lo, int border, int cell, void* stream) {
    if (n_tiles <= 0) return;
    k_fast<<<n_tiles, DET_THREADS, 0, (cudaStream_t)stream>>>(imgs, img_list, tile_prefix, n_list,
                                                               t_hi, t_lo, border, cell);
}

}  // namespace ofk
