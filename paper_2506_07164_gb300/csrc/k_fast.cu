// FAST-9 segment test with a score (Eq. 1, Sec. 3.1; binary encoding of
// Alg. 2 / Fig. 3), two pixels per 32-bit register in 16-bit lanes.
//
// Score.  Eq. 1 calls ring pixel I_i bright when I_i >= I_p + t and dark when
// I_i <= I_p - t; p is a corner at t when 9 contiguous ring pixels are all
// bright or all dark.  The largest such t is
//   s(p) = max( max_j min_{k<9} I_{j+k} - I_p ,  I_p - min_j max_{k<9} I_{j+k} )
// (the I_p terms leave the min/max), so corner(t) <=> s(p) >= t for t >= 1.
// The arc terms use the three-input packed min/max of sm_90+ (DPX):
// minima of 3 contiguous ring pixels, then of 9 = three 3-runs 3 apart, then
// the maximum over the 16 starts -- 40 instructions per side for 2 pixels,
// no branches.  The map stores s(p) where s(p) >= t_lo (the lowest threshold
// in use), else 0.
//
// Data movement.  A thread owns 4 adjacent pixels x..x+3 over RPT rows.  Each
// staged row gives it three 32-bit words (bytes x-4..x+7); one byte permute
// per pair turns them into six 16-bit-lane words (pixel pairs x-4.., x-2..,
// x.., x+2.., x+4.., x+6..).  A ring pixel at an even column offset is one of
// those words; at an odd offset one more permute joins two of them.
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

// The pair (x+o, x+o+1) in 16-bit lanes, o in -4..6, from the six pair words
// h[j] = (x-4+2j, x-3+2j).
template <int O>
__device__ __forceinline__ uint32_t pair_at(const uint32_t (&h)[6]) {
    constexpr int j = (O + 4) >> 1;
    if constexpr (((O + 4) & 1) == 0) return h[j];
    else return __byte_perm(h[j], h[j + 1], 0x5432);  // high lane of h[j], low lane of h[j+1]
}

// Largest arc minimum and smallest arc maximum over the 16 nine-pixel arcs,
// for the two pixels in the lanes of q[].
__device__ __forceinline__ void arc_extrema(const uint32_t (&q)[16], uint32_t& amax, uint32_t& amin) {
    uint32_t m3[16], M3[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        m3[i] = __vimin3_u16x2(q[i], q[(i + 1) & 15], q[(i + 2) & 15]);
        M3[i] = __vimax3_u16x2(q[i], q[(i + 1) & 15], q[(i + 2) & 15]);
    }
    uint32_t m9[16], M9[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        m9[i] = __vimin3_u16x2(m3[i], m3[(i + 3) & 15], m3[(i + 6) & 15]);
        M9[i] = __vimax3_u16x2(M3[i], M3[(i + 3) & 15], M3[(i + 6) & 15]);
    }
    const uint32_t a0 = __vimax3_u16x2(m9[0], m9[1], m9[2]), a1 = __vimax3_u16x2(m9[3], m9[4], m9[5]);
    const uint32_t a2 = __vimax3_u16x2(m9[6], m9[7], m9[8]), a3 = __vimax3_u16x2(m9[9], m9[10], m9[11]);
    const uint32_t a4 = __vimax3_u16x2(m9[12], m9[13], m9[14]);
    const uint32_t b0 = __vimin3_u16x2(M9[0], M9[1], M9[2]), b1 = __vimin3_u16x2(M9[3], M9[4], M9[5]);
    const uint32_t b2 = __vimin3_u16x2(M9[6], M9[7], M9[8]), b3 = __vimin3_u16x2(M9[9], M9[10], M9[11]);
    const uint32_t b4 = __vimin3_u16x2(M9[12], M9[13], M9[14]);
    amax = __vimax3_u16x2(__vimax3_u16x2(a0, a1, a2), a3, __vimax3_u16x2(a4, m9[15], 0u));
    amin = __vimin3_u16x2(__vimin3_u16x2(b0, b1, b2), b3, __vimin3_u16x2(b4, M9[15], 0xFFFFFFFFu));
}

// s(p) for the two pixels of a pair: lanes of max(amax - c, c - amin, 0).
__device__ __forceinline__ uint32_t pair_score(const uint32_t (&q)[16], uint32_t c) {
    uint32_t amax, amin;
    arc_extrema(q, amax, amin);
    constexpr uint32_t B = 0x01000100u;  // +256 per lane keeps each difference positive
    return __vimax3_u16x2(amax + B - c, c + B - amin, B) - B;
}

// 0xFFFF in each 16-bit lane whose value is >= t (values and t below 2^15).
__device__ __forceinline__ uint32_t lanes_ge(uint32_t v, uint32_t t) {
    const uint32_t d = v + (0x8000u - t) * 0x00010001u;
    return ((d >> 15) & 0x00010001u) * 0xFFFFu;
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
    // Six pair words per staged row (RPT + 6 rows).
    uint32_t hw[RPT + 6][6];
#pragma unroll
    for (int k = 0; k < RPT + 6; ++k) {
        const uint8_t* row = s + (ty * RPT + k) * SROW + HALO_X + 4 * lane;
        const uint32_t wm = *reinterpret_cast<const uint32_t*>(row - 4);
        const uint32_t wc = *reinterpret_cast<const uint32_t*>(row);
        const uint32_t wp = *reinterpret_cast<const uint32_t*>(row + 4);
        hw[k][0] = __byte_perm(wm, 0u, 0x4140);
        hw[k][1] = __byte_perm(wm, 0u, 0x4342);
        hw[k][2] = __byte_perm(wc, 0u, 0x4140);
        hw[k][3] = __byte_perm(wc, 0u, 0x4342);
        hw[k][4] = __byte_perm(wp, 0u, 0x4140);
        hw[k][5] = __byte_perm(wp, 0u, 0x4342);
    }
    const uint32_t colmask = range_mask4(x, rx0, rx1);

#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int y = Y0 + ty * RPT + r;
        uint32_t q0[16], q1[16];
#define OF_LOAD_RING(i, dx, dy)                        \
    q0[i] = pair_at<(dx)>(hw[r + 3 + (dy)]);          \
    q1[i] = pair_at<(dx) + 2>(hw[r + 3 + (dy)]);
        OF_RING(OF_LOAD_RING)
#undef OF_LOAD_RING
        uint32_t s0 = pair_score(q0, hw[r + 3][2]);
        uint32_t s1 = pair_score(q1, hw[r + 3][3]);
        s0 &= lanes_ge(s0, (uint32_t)t_lo);
        s1 &= lanes_ge(s1, (uint32_t)t_lo);
        const uint32_t m = (y < ry1) ? colmask : 0u;
        const uint32_t sc = __byte_perm(s0, s1, 0x6420) & m;
        if (m != 0u) *reinterpret_cast<uint32_t*>(I.score + (size_t)y * I.spitch + x) = sc;
        if (cells && sc) {
            const uint32_t strong = __byte_perm(lanes_ge(s0, (uint32_t)t_hi), lanes_ge(s1, (uint32_t)t_hi),
                                                0x6420) & m;
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
