// Candidate selection, strict 3x3 non-maximum suppression and the Harris key
// of every survivor, fused per 128 x 32 tile (the FAST -> Harris fusion of
// Sec. 5.2: the survivors' Harris sums are computed from the same shared
// memory tile, with no round trip of points through global memory).
//
// 1. Stage the score tile (+1 pixel halo) and turn it into S(p): s(p) when p is
//    a candidate at its cell's threshold, else 0; 0 outside the detect region.
// 2. NMS, 4 pixels per register: p survives when S(p) > max of its 8
//    neighbours (byte-wise max of 8 shifted words, one byte-wise compare).
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
    if (threadIdx.x == 0) nq = 0;
    if (cells) {
        for (int i = threadIdx.x; i < lcw * lch; i += blockDim.x) {
            const int cx = cx0 + i % lcw, cy = cy0 + i / lcw;
            sflag[i] = (cx < I.ncx && cy < I.ncy) ? I.cell[cy * I.ncx + cx] : 0u;
        }
        __syncthreads();
    }

    // 1. S(p) for rows Y0-1 .. Y0+TILE_H, columns X0-16 .. X0+TILE_W+16.
    {
        constexpr int CPR = SROW / 16;
        const uint32_t thi4 = 0x01010101u * (uint32_t)t_hi;
        // Only columns X0-1 .. X0+TILE_W feed the 3x3 test; the rest stay 0.
        const int lox = max(rx0, X0 - 1), hix = min(rx1, X0 + TILE_W + 1);
        const int n = (TILE_H + 2) * CPR;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int r = i / CPR, k = i - r * CPR;
            const int iy = Y0 - 1 + r, ix = X0 - HALO_X + 16 * k;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (iy >= ry0 && iy < ry1 && ix + 16 > lox && ix < hix) {
                v = __ldg(reinterpret_cast<const uint4*>(I.score + (size_t)iy * I.spitch + ix));
                uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t m = range_mask4(ix + 4 * q, lox, hix);
                    uint32_t val = wd[q] & m;
                    if (cells && val) {
                        // Bytes below t_hi survive only when their cell has no strong pixel.
                        const uint32_t weak = __vcmpltu4(val, thi4) & __vcmpne4(val, 0u);
                        if (weak) {
                            const int cyl = (iy - ry0) / cell - cy0;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                if ((weak >> (8 * e)) & 1u) {
                                    const int cxl = (ix + 4 * q + e - rx0) / cell - cx0;
                                    if (sflag[cyl * lcw + cxl]) val &= ~(0xFFu << (8 * e));
                                }
                            }
                        }
                    }
                    wd[q] = val;
                }
                v = make_uint4(wd[0], wd[1], wd[2], wd[3]);
            }
            *reinterpret_cast<uint4*>(sS + r * SROW + 16 * k) = v;
        }
    }
    __syncthreads();

    // 2. Strict 3x3 maxima.
    const int lane = threadIdx.x & 31, ty = threadIdx.x >> 5;
    {
        uint32_t wm[RPT + 2], wc[RPT + 2], wp[RPT + 2];
#pragma unroll
        for (int k = 0; k < RPT + 2; ++k) {
            const uint8_t* row = sS + (ty * RPT + k) * SROW + HALO_X + 4 * lane;
            wm[k] = *reinterpret_cast<const uint32_t*>(row - 4);
            wc[k] = *reinterpret_cast<const uint32_t*>(row);
            wp[k] = *reinterpret_cast<const uint32_t*>(row + 4);
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            uint32_t nb = win4<-1>(wm[r], wc[r], wp[r]);
            nb = __vmaxu4(nb, wc[r]);
            nb = __vmaxu4(nb, win4<1>(wm[r], wc[r], wp[r]));
            nb = __vmaxu4(nb, win4<-1>(wm[r + 1], wc[r + 1], wp[r + 1]));
            nb = __vmaxu4(nb, win4<1>(wm[r + 1], wc[r + 1], wp[r + 1]));
            nb = __vmaxu4(nb, win4<-1>(wm[r + 2], wc[r + 2], wp[r + 2]));
            nb = __vmaxu4(nb, wc[r + 2]);
            nb = __vmaxu4(nb, win4<1>(wm[r + 2], wc[r + 2], wp[r + 2]));
            const uint32_t keep = __vcmpgtu4(wc[r + 1], nb);
            if (keep) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if ((keep >> (8 * e)) & 1u) {
                        const int slot = atomicAdd(&nq, 1);
                        queue[slot] = ((uint32_t)(ty * RPT + r) << 16) | (uint32_t)(4 * lane + e);
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
