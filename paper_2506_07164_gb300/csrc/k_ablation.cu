// The paper's ablation variants (Table 2, Sec. 6.2) on GB300, for measuring
// whether their ordering holds on Blackwell.  Not on the hot path: the
// detector's own kernels (k_fast, k_nms_harris) compute a threshold-free
// score and Harris for NMS survivors only.
//
// Every variant finds the FAST points at threshold t (Eq. 1: 9 contiguous
// ring pixels all >= I_p + t or all <= I_p - t) in the detect region and,
// for the Harris variants, the exact Sobel sums A, B, C over the 7 x 7 window
// (Eqs. 2-4) and the integer key of each point -- the same numbers whichever
// variant runs.  One thread per pixel, blocks of 32 x 8 pixels.
//
// FAST variants (one launch; points appended to a list):
//   baseline  global loads; 8 opposite ring pairs decide which tones are
//             possible (a 9-arc holds one pixel of every opposite pair), then
//             a run-length scan over 16 + 8 ring positions with early exit
//             (the CUDA_ORB form of Alg. 1)
//   binary    global loads; the 16 bright and 16 dark tests packed in a word,
//             each half extended to 24 bits by its low 8, then 16 shifted
//             9-bit windows compared with 0x1FF (Alg. 2)
//   sm        the baseline logic on a shared-memory tile
//   sm_binary the binary logic on a shared-memory tile
// Harris variants (each fused after sm_binary in one kernel, as the paper
// pairs them, except the baseline):
//   baseline  a second launch over the point list: 2-D 3 x 3 Sobel at each of
//             the 49 window pixels, global loads
//   sep       one thread per point: separable Sobel over its own 9 x 9
//             footprint (the [-1 0 1] / [1 2 1] row passes, then the column
//             passes), from the shared tile
//   para_sep  the block computes every row pass, then every gx, gy of the tile
//             into shared memory; each point sums its 7 x 7 products
//   semi_sep  Alg. 3: a warp whose row holds a point computes, per column, the
//             vertical 7-row sums of gx^2, gy^2, gx gy with a three-row
//             register ring, stores them in shared memory, and each point
//             adds its 7 columns
#include <cuda_runtime.h>
#include <stdint.h>

#include "of_internal.h"

namespace ofk {

constexpr int AB_W = 32, AB_H = 8;             // pixels per block
constexpr int AB_HALO = 4;                     // Sobel at window edge +- 1
constexpr int AB_SW = AB_W + 2 * AB_HALO;      // 40 staged columns
constexpr int AB_SH = AB_H + 2 * AB_HALO;      // 16 staged rows

__constant__ int8_t c_ring_dx[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
__constant__ int8_t c_ring_dy[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};

// Pixel fetchers: global (read-only cache) or the block's shared tile.
struct GlobalPix {
    const uint8_t* img;
    int pitch;
    __device__ __forceinline__ int operator()(int x, int y) const { return __ldg(img + (size_t)y * pitch + x); }
};
struct SharedPix {
    const uint8_t* s;  // staged tile, row 0 = y0 - AB_HALO, column 0 = x0 - AB_HALO
    int x0, y0;
    __device__ __forceinline__ int operator()(int x, int y) const {
        return s[(y - y0 + AB_HALO) * AB_SW + (x - x0 + AB_HALO)];
    }
};

template <class Pix>
__device__ bool fast_baseline(const Pix& P, int x, int y, int t) {
    const int c = P(x, y), hi = c + t, lo = c - t;
    bool can_b = true, can_d = true;
    for (int i = 0; i < 8; ++i) {
        const int v1 = P(x + c_ring_dx[i], y + c_ring_dy[i]);
        const int v2 = P(x + c_ring_dx[i + 8], y + c_ring_dy[i + 8]);
        can_b = can_b && (v1 >= hi || v2 >= hi);
        can_d = can_d && (v1 <= lo || v2 <= lo);
    }
    if (!can_b && !can_d) return false;
    for (int tone = 0; tone < 2; ++tone) {
        if (tone == 0 ? !can_d : !can_b) continue;
        int count = 0;
        for (int k = 0; k < 24; ++k) {
            const int v = P(x + c_ring_dx[k & 15], y + c_ring_dy[k & 15]);
            if (tone == 0 ? v <= lo : v >= hi) {
                if (++count >= 9) return true;
            } else {
                count = 0;
            }
        }
    }
    return false;
}

template <class Pix>
__device__ bool fast_binary(const Pix& P, int x, int y, int t) {
    const int c = P(x, y), hi = c + t, lo = c - t;
    uint32_t buf = 0u;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int v = P(x + c_ring_dx[i], y + c_ring_dy[i]);
        buf |= (v >= hi ? 1u : 0u) << i;
        buf |= (v <= lo ? 1u : 0u) << (16 + i);
    }
    const uint32_t bright = buf & 0xFFFFu, dark = buf >> 16;
    const uint32_t b24 = bright | ((bright & 0xFFu) << 16), d24 = dark | ((dark & 0xFFu) << 16);
    for (int k = 0; k < 16; ++k)
        if (((d24 >> k) & 0x1FFu) == 0x1FFu) return true;
    for (int k = 0; k < 16; ++k)
        if (((b24 >> k) & 0x1FFu) == 0x1FFu) return true;
    return false;
}

__device__ __forceinline__ void stage_ab(uint8_t* s, const uint8_t* img, int w, int h, int pitch, int x0, int y0) {
    for (int i = threadIdx.y * AB_W + threadIdx.x; i < AB_SW * AB_SH; i += AB_W * AB_H) {
        const int r = i / AB_SW, c = i - r * AB_SW;
        const int x = x0 - AB_HALO + c, y = y0 - AB_HALO + r;
        s[i] = (x >= 0 && x < w && y >= 0 && y < h) ? __ldg(img + (size_t)y * pitch + x) : 0;
    }
}

__device__ __forceinline__ int64_t harris_key_of(int32_t A, int32_t B, int32_t C, int64_t knum, int64_t kden) {
    const int64_t det = (int64_t)A * B - (int64_t)C * C, tr = (int64_t)A + B;
    return kden * det - knum * tr * tr;
}

__device__ __forceinline__ void emit(of_var_point* out, int32_t* count, int cap, int x, int y, int32_t A, int32_t B,
                                     int32_t C, int64_t key) {
    const int i = atomicAdd(count, 1);
    if (i < cap) {
        of_var_point p;
        p.x = x;
        p.y = y;
        p.A = A;
        p.B = B;
        p.C = C;
        p.reserved = 0;
        p.key = key;
        out[i] = p;
    }
}

// FAST-only variants 0..3; points appended with zero sums.
template <int V>
__global__ void __launch_bounds__(AB_W * AB_H)
k_var_fast(const uint8_t* __restrict__ img, int w, int h, int pitch, int t, int border, of_var_point* out,
           int32_t* count, int cap) {
    __shared__ uint8_t s[AB_SW * AB_SH];
    const int x0 = border + blockIdx.x * AB_W, y0 = border + blockIdx.y * AB_H;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if constexpr (V >= 2) {
        stage_ab(s, img, w, h, pitch, x0, y0);
        __syncthreads();
    }
    if (x >= w - border || y >= h - border) return;
    bool pt;
    if constexpr (V == 0) pt = fast_baseline(GlobalPix{img, pitch}, x, y, t);
    else if constexpr (V == 1) pt = fast_binary(GlobalPix{img, pitch}, x, y, t);
    else if constexpr (V == 2) pt = fast_baseline(SharedPix{s, x0, y0}, x, y, t);
    else pt = fast_binary(SharedPix{s, x0, y0}, x, y, t);
    if (pt) emit(out, count, cap, x, y, 0, 0, 0, 0);
}

// Harris baseline: second launch over the point list, 2-D Sobel from global memory.
__global__ void k_var_harris_base(const uint8_t* __restrict__ img, int pitch, of_var_point* pts,
                                  const int32_t* __restrict__ count, int cap, int64_t knum, int64_t kden) {
    const int n = min(*count, cap);
    const GlobalPix P{img, pitch};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = pts[i].x, y = pts[i].y;
        int32_t A = 0, B = 0, C = 0;
        for (int dy = -3; dy <= 3; ++dy) {
            for (int dx = -3; dx <= 3; ++dx) {
                const int u = x + dx, v = y + dy;
                const int gx = (P(u + 1, v - 1) - P(u - 1, v - 1)) + 2 * (P(u + 1, v) - P(u - 1, v)) +
                               (P(u + 1, v + 1) - P(u - 1, v + 1));
                const int gy = (P(u - 1, v + 1) - P(u - 1, v - 1)) + 2 * (P(u, v + 1) - P(u, v - 1)) +
                               (P(u + 1, v + 1) - P(u + 1, v - 1));
                A += gx * gx;
                B += gy * gy;
                C += gx * gy;
            }
        }
        pts[i].A = A;
        pts[i].B = B;
        pts[i].C = C;
        pts[i].key = harris_key_of(A, B, C, knum, kden);
    }
}

// sm_binary FAST fused with Harris variant H (1 sep, 2 para_sep, 3 semi_sep).
template <int H>
__global__ void __launch_bounds__(AB_W * AB_H)
k_var_fused(const uint8_t* __restrict__ img, int w, int h, int pitch, int t, int border, int64_t knum, int64_t kden,
            of_var_point* out, int32_t* count, int cap) {
    __shared__ uint8_t s[AB_SW * AB_SH];
    // para_sep: row passes, then gradients, of the whole tile (int16 is exact:
    // |[-1 0 1]| <= 255, [1 2 1] <= 1020, |g| <= 1020).
    __shared__ int16_t hd[H == 2 ? AB_SH : 1][AB_SW], hs[H == 2 ? AB_SH : 1][AB_SW];
    __shared__ int16_t gxs[H == 2 ? AB_H + 6 : 1][AB_SW], gys[H == 2 ? AB_H + 6 : 1][AB_SW];
    // semi_sep: per-warp column sums of the 38 columns x0-3 .. x0+34.
    __shared__ int32_t sxx[H == 3 ? AB_H : 1][AB_W + 6], syy[H == 3 ? AB_H : 1][AB_W + 6],
        sxy[H == 3 ? AB_H : 1][AB_W + 6];
    const int x0 = border + blockIdx.x * AB_W, y0 = border + blockIdx.y * AB_H;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = x0 + tx, y = y0 + ty;
    stage_ab(s, img, w, h, pitch, x0, y0);
    __syncthreads();
    const SharedPix P{s, x0, y0};
    const bool in = x < w - border && y < h - border;
    const bool pt = in && fast_binary(P, x, y, t);
    int32_t A = 0, B = 0, C = 0;
    if constexpr (H == 1) {
        if (pt) {
            int rd[9][7], rs[9][7];
            for (int r = 0; r < 9; ++r)
                for (int u = 0; u < 7; ++u) {
                    const int a = P(x + u - 4, y + r - 4), b = P(x + u - 3, y + r - 4), c = P(x + u - 2, y + r - 4);
                    rd[r][u] = c - a;
                    rs[r][u] = a + 2 * b + c;
                }
            for (int v = 0; v < 7; ++v)
                for (int u = 0; u < 7; ++u) {
                    const int gx = rd[v][u] + 2 * rd[v + 1][u] + rd[v + 2][u];
                    const int gy = rs[v + 2][u] - rs[v][u];
                    A += gx * gx;
                    B += gy * gy;
                    C += gx * gy;
                }
        }
    } else if constexpr (H == 2) {
        // Row passes at staged columns 1..38, all staged rows.
        for (int i = ty * AB_W + tx; i < AB_SH * (AB_SW - 2); i += AB_W * AB_H) {
            const int r = i / (AB_SW - 2), c = 1 + i % (AB_SW - 2);
            const int a = s[r * AB_SW + c - 1], b = s[r * AB_SW + c], d = s[r * AB_SW + c + 1];
            hd[r][c] = (int16_t)(d - a);
            hs[r][c] = (int16_t)(a + 2 * b + d);
        }
        __syncthreads();
        // Gradients at staged rows 1..14 (tile rows -3..AB_H+2), columns 1..38.
        for (int i = ty * AB_W + tx; i < (AB_H + 6) * (AB_SW - 2); i += AB_W * AB_H) {
            const int g = i / (AB_SW - 2), c = 1 + i % (AB_SW - 2), r = g + 1;
            gxs[g][c] = (int16_t)(hd[r - 1][c] + 2 * hd[r][c] + hd[r + 1][c]);
            gys[g][c] = (int16_t)(hs[r + 1][c] - hs[r - 1][c]);
        }
        __syncthreads();
        if (pt) {
            for (int v = 0; v < 7; ++v)
                for (int u = 0; u < 7; ++u) {
                    const int gx = gxs[ty + v][tx + AB_HALO - 3 + u], gy = gys[ty + v][tx + AB_HALO - 3 + u];
                    A += gx * gx;
                    B += gy * gy;
                    C += gx * gy;
                }
        }
    } else {
        // Alg. 3: a warp is one tile row; skip it when no lane has a point.
        if (__any_sync(0xFFFFFFFFu, pt)) {
            for (int c = tx; c < AB_W + 6; c += AB_W) {
                const int cx = x0 - 3 + c;  // image column of this column sum
                int rdv[3], rsv[3];
                int32_t a = 0, b = 0, cc = 0;
#pragma unroll
                for (int k = 0; k < 9; ++k) {  // image rows y-4 .. y+4
                    const int row = y - 4 + k;
                    const int l = P(cx - 1, row), m = P(cx, row), r = P(cx + 1, row);
                    rdv[k % 3] = r - l;
                    rsv[k % 3] = l + 2 * m + r;
                    if (k >= 2) {
                        const int gx = rdv[(k + 1) % 3] + 2 * rdv[(k + 2) % 3] + rdv[k % 3];
                        const int gy = rsv[k % 3] - rsv[(k + 1) % 3];
                        a += gx * gx;
                        b += gy * gy;
                        cc += gx * gy;
                    }
                }
                sxx[ty][c] = a;
                syy[ty][c] = b;
                sxy[ty][c] = cc;
            }
            __syncwarp();
            if (pt) {
                for (int j = 0; j < 7; ++j) {
                    A += sxx[ty][tx + j];
                    B += syy[ty][tx + j];
                    C += sxy[ty][tx + j];
                }
            }
        }
    }
    if (pt) emit(out, count, cap, x, y, A, B, C, harris_key_of(A, B, C, knum, kden));
}

int launch_variant(int fast_v, int harris_v, const uint8_t* img, int w, int h, int pitch, int t, int border,
                   int64_t knum, int64_t kden, of_var_point* out, int32_t* count, int cap, int n_sms, void* stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    const int rw = w - 2 * border, rh = h - 2 * border;
    if (rw <= 0 || rh <= 0) return 0;
    const dim3 block(AB_W, AB_H), grid((rw + AB_W - 1) / AB_W, (rh + AB_H - 1) / AB_H);
    if (harris_v >= 1) {
        if (harris_v == 1)
            k_var_fused<1><<<grid, block, 0, st>>>(img, w, h, pitch, t, border, knum, kden, out, count, cap);
        else if (harris_v == 2)
            k_var_fused<2><<<grid, block, 0, st>>>(img, w, h, pitch, t, border, knum, kden, out, count, cap);
        else
            k_var_fused<3><<<grid, block, 0, st>>>(img, w, h, pitch, t, border, knum, kden, out, count, cap);
        return 1;
    }
    switch (fast_v) {
        case 0: k_var_fast<0><<<grid, block, 0, st>>>(img, w, h, pitch, t, border, out, count, cap); break;
        case 1: k_var_fast<1><<<grid, block, 0, st>>>(img, w, h, pitch, t, border, out, count, cap); break;
        case 2: k_var_fast<2><<<grid, block, 0, st>>>(img, w, h, pitch, t, border, out, count, cap); break;
        default: k_var_fast<3><<<grid, block, 0, st>>>(img, w, h, pitch, t, border, out, count, cap); break;
    }
    if (harris_v == 0) {
        k_var_harris_base<<<n_sms * 4, 256, 0, st>>>(img, pitch, out, count, cap, knum, kden);
        return 2;
    }
    return 1;
}

}  // namespace ofk
