// Candidate selection, strict 3x3 non-maximum suppression and the Harris key
// of every survivor, fused per 128 x 32 tile (the FAST -> Harris fusion of
// Sec. 5.2: the survivors' Harris sums are computed from the same shared
// memory tile, with no round trip of points through global memory).
//
// 1. Stage the score tile (+1 pixel halo) and turn it into S(p): s(p) when p is
//    a candidate at its cell's threshold, else 0; 0 outside the detect region.
//    A per-tile table gives, for each staged word and cell row, the bytes that
//    lie in cells whose threshold is t_hi.
// 2. NMS, two pixels per register in 16-bit lanes: p survives when S(p) > the
//    three-input maximum of its 8 neighbours.
// 3. Survivors go to a shared-memory queue; the image tile (+4 pixel halo) is
//    staged only when the queue is not empty.
// 4. Harris (Eqs. 2-4, Alg. 3): one thread per survivor slides down the 9 x 9
//    footprint keeping three rows of the horizontal Sobel passes (difference
//    [-1 0 1] and smoothing [1 2 1]) in registers -- the circular buffer of
//    Alg. 3 -- and combines them vertically into gx, gy, accumulating the
//    exact int32 sums A = sum gx^2, B = sum gy^2, C = sum gx gy over 7 x 7.
//    key = kden (AB - C^2) - knum (A+B)^2 (int64, exact for k = knum/kden).
// 5. One atomicAdd per tile reserves the survivors' slots in the image's list.
#include <cuda_runtime.h>

#include "of_internal.h"
#include "of_tile.cuh"

namespace ofk {

constexpr int QCAP = TILE_W * TILE_H / 4;  // strict maxima are never adjacent
constexpr int WPR = SROW / 4;               // staged words per row
constexpr int LCH_MAX = (TILE_H + 2) / 8 + 2;  // cell rows touched by a tile (cell >= 8)

// 0xFF in each byte of v that is below t (t <= 255).
__device__ __forceinline__ uint32_t bytes_lt(uint32_t v, uint32_t t) {
    const uint32_t tt = (0x8000u - t) * 0x00010001u;
    const uint32_t lo = __byte_perm(v, 0u, 0x4140) + tt, hi = __byte_perm(v, 0u, 0x4342) + tt;
    // bit 15 of a lane set <=> byte >= t
    return ~__byte_perm((lo >> 15 & 0x00010001u) * 0xFFu, (hi >> 15 & 0x00010001u) * 0xFFu, 0x6420);
}

__device__ __forceinline__ void harris_sums(const uint8_t* __restrict__ s, int lx, int ly,
                                            int32_t& A, int32_t& B, int32_t& C) {
    // s: image tile, row 0 = tile row -4, column HALO_X = tile column 0.
    int hd[3][7], hsm[3][7];
    int a = 0, bb = 0, c = 0;
#pragma unroll
    for (int v = -4; v <= 4; ++v) {
        const uint8_t* row = s + (ly + 4 + v) * SROW + HALO_X + lx - 4;
        int p[9];
#pragma unroll
        for (int u = 0; u < 9; ++u) p[u] = row[u];
        const int slot = (v + 4) % 3;
#pragma unroll
        for (int u = 0; u < 7; ++u) {
            hd[slot][u] = p[u + 2] - p[u];
            hsm[slot][u] = p[u] + 2 * p[u + 1] + p[u + 2];
        }
        if (v >= -2) {
            const int s0 = (v + 2) % 3, s1 = (v + 3) % 3;  // rows v-2, v-1
#pragma unroll
            for (int u = 0; u < 7; ++u) {
                const int gx = hd[s0][u] + 2 * hd[s1][u] + hd[slot][u];
                const int gy = hsm[slot][u] - hsm[s0][u];
                a += gx * gx;
                bb += gy * gy;
                c += gx * gy;
            }
        }
    }
    A = a;
    B = bb;
    C = c;
}

__global__ void __launch_bounds__(DET_THREADS)
k_nms_harris(const Img* __restrict__ imgs, const int32_t* __restrict__ list,
             const int32_t* __restrict__ prefix, int n_list, const Call* __restrict__ call,
             int t_hi, int t_lo, int border, int cell) {
    __shared__ __align__(16) uint8_t sS[(TILE_H + 2) * SROW];
    __shared__ __align__(16) uint8_t sI[(TILE_H + 8) * SROW];
    __shared__ uint32_t sflag[MAX_CELLS_LOCAL];
    __shared__ uint32_t fmask[LCH_MAX * WPR];
    __shared__ uint32_t queue[QCAP];
    __shared__ int nq, qbase;

    const int b = blockIdx.x;
    const int j = find_tile_job(prefix, n_list, b);
    const Img& I = imgs[__ldg(list + j)];
    const int w = I.w, h = I.h;
    const int t = b - __ldg(prefix + j);
    const int tx = t % I.tiles_x, ty_tile = t / I.tiles_x;
    const int X0 = I.tile_x0 + tx * TILE_W;
    const int Y0 = border + ty_tile * TILE_H;
    const int rx0 = border, rx1 = w - border, ry0 = border, ry1 = h - border;
    const bool cells = t_hi != t_lo;

    // Cells touched by the tile and its 1-pixel halo.
    const int cx0 = (max(X0 - 1, rx0) - rx0) / cell;
    const int cy0 = (max(Y0 - 1, ry0) - ry0) / cell;
    const int lcw = (TILE_W + 2) / cell + 2;
    const int lch = (TILE_H + 2) / cell + 2;
    // Only columns X0-1 .. X0+TILE_W feed the 3x3 test; the rest stay 0.
    const int lox = max(rx0, X0 - 1), hix = min(rx1, X0 + TILE_W + 1);
    if (threadIdx.x == 0) nq = 0;
    if (cells) {
        for (int i = threadIdx.x; i < lcw * lch; i += blockDim.x) {
            const int cx = cx0 + i % lcw, cy = cy0 + i / lcw;
            sflag[i] = (cx < I.ncx && cy < I.ncy) ? I.cell[cy * I.ncx + cx] : 0u;
        }
        __syncthreads();
        // fmask[cyl][k]: 0xFF for each byte of staged word k in a flagged cell of cell row cyl.
        for (int i = threadIdx.x; i < lch * WPR; i += blockDim.x) {
            const int cyl = i / WPR, k = i - cyl * WPR;
            uint32_t m = 0u;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int xx = X0 - HALO_X + 4 * k + e;
                if (xx >= lox && xx < hix && sflag[cyl * lcw + (xx - rx0) / cell - cx0])
                    m |= 0xFFu << (8 * e);
            }
            fmask[i] = m;
        }
        __syncthreads();
    }

    // 1. S(p) for rows Y0-1 .. Y0+TILE_H, columns X0-16 .. X0+TILE_W+16.
    {
        constexpr int CPR = SROW / 16;
        const int n = (TILE_H + 2) * CPR;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int r = i / CPR, k = i - r * CPR;
            const int iy = Y0 - 1 + r, ix = X0 - HALO_X + 16 * k;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (iy >= ry0 && iy < ry1 && ix + 16 > lox && ix < hix) {
                v = __ldg(reinterpret_cast<const uint4*>(I.score + (size_t)iy * I.spitch + ix));
                uint32_t wd[4] = {v.x, v.y, v.z, v.w};
                const uint32_t* fm = fmask + ((iy - ry0) / cell - cy0) * WPR + 4 * k;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t val = wd[q] & range_mask4(ix + 4 * q, lox, hix);
                    // Bytes below t_hi survive only when their cell has no strong pixel.
                    if (cells && val) val &= ~(fm[q] & bytes_lt(val, (uint32_t)t_hi));
                    wd[q] = val;
                }
                v = make_uint4(wd[0], wd[1], wd[2], wd[3]);
            }
            *reinterpret_cast<uint4*>(sS + r * SROW + 16 * k) = v;
        }
    }
    __syncthreads();

    // 2. Strict 3x3 maxima, two pixels per register.
    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    {
        uint32_t hw[RPT + 2][6];
#pragma unroll
        for (int k = 0; k < RPT + 2; ++k) {
            const uint8_t* row = sS + (ty * RPT + k) * SROW + HALO_X + 4 * lane;
            const uint32_t wm = *reinterpret_cast<const uint32_t*>(row - 4);
            const uint32_t wc = *reinterpret_cast<const uint32_t*>(row);
            const uint32_t wp = *reinterpret_cast<const uint32_t*>(row + 4);
            hw[k][1] = __byte_perm(wm, 0u, 0x4342);  // (x-2, x-1)
            hw[k][2] = __byte_perm(wc, 0u, 0x4140);  // (x, x+1)
            hw[k][3] = __byte_perm(wc, 0u, 0x4342);  // (x+2, x+3)
            hw[k][4] = __byte_perm(wp, 0u, 0x4140);  // (x+4, x+5)
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) {
                // Pair (x+2pr, x+2pr+1): neighbours at column offsets -1, 0, +1.
                const uint32_t* a = hw[r];
                const uint32_t* c = hw[r + 1];
                const uint32_t* d = hw[r + 2];
                const int j = 2 + pr;
                const uint32_t am = __byte_perm(a[j - 1], a[j], 0x5432), ap = __byte_perm(a[j], a[j + 1], 0x5432);
                const uint32_t cm = __byte_perm(c[j - 1], c[j], 0x5432), cp = __byte_perm(c[j], c[j + 1], 0x5432);
                const uint32_t dm = __byte_perm(d[j - 1], d[j], 0x5432), dp = __byte_perm(d[j], d[j + 1], 0x5432);
                const uint32_t nb = __vimax3_u16x2(__vimax3_u16x2(am, a[j], ap), __vimax3_u16x2(cm, cp, dm),
                                                   __vimax3_u16x2(d[j], dp, dp));
                // Lane bit 15 set when centre > neighbours (values <= 255).
                const uint32_t keep = (c[j] + 0x7FFF7FFFu - nb) & 0x80008000u;
                if (keep) {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if ((keep >> (16 * e + 15)) & 1u) {
                            const int slot = atomicAdd(&nq, 1);
                            queue[slot] = ((uint32_t)(ty * RPT + r) << 16) | (uint32_t)(4 * lane + 2 * pr + e);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    const int count = nq;
    if (count == 0) return;
    if (threadIdx.x == 0) qbase = atomicAdd(&I.ctr[0], count);

    // 3. Image tile for the survivors' 9 x 9 footprints.
    stage_tile(sI, I.img, w, h, I.pitch, X0 - HALO_X, Y0 - 4, TILE_H + 8);
    __syncthreads();

    const int base = qbase;
    const int64_t knum = call->knum, kden = call->kden;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const uint32_t e = queue[i];
        const int lx = (int)(e & 0xFFFFu), ly = (int)(e >> 16);
        int32_t A, B, C;
        harris_sums(sI, lx, ly, A, B, C);
        const int64_t det = (int64_t)A * B - (int64_t)C * C;
        const int64_t tr = (int64_t)A + B;
        const int64_t key = kden * det - knum * tr * tr;
        const int slot = base + i;
        if (slot < I.cand_cap) {
            I.ckey[slot] = (uint64_t)key ^ 0x8000000000000000ull;
            I.cyx[slot] = ((uint32_t)(Y0 + ly) << 16) | (uint32_t)(X0 + lx);
        } else {
            I.ctr[2] = 1;  // cannot happen: survivors are an independent set
        }
    }
}

void launch_nms_harris(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix,
                       int n_list, int n_tiles, const Call* call, int t_hi, int t_lo, int border,
                       int cell, void* stream) {
    if (n_tiles <= 0) return;
    k_nms_harris<<<n_tiles, DET_THREADS, 0, (cudaStream_t)stream>>>(
        imgs, img_list, tile_prefix, n_list, call, t_hi, t_lo, border, cell);
}

}  // namespace ofk
