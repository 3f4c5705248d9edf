// Orientation by intensity centroid (Fig. 1 "Centroid") and the output
// records.  One warp per output slot (frame, level, rank):
//   - Harris sums A, B, C of the kept keypoint (Eqs. 2-4), lanes over the 49
//     window positions, warp reduction;
//   - moments m10 = sum u I, m01 = sum v I over the disc u^2 + v^2 <= r^2,
//     lane = column u, loop over rows v, warp reduction;
//   - angle = atan2f(m01, m10) (both moments are exact int32, |m| < 2^24, so
//     their float conversion is exact);
//   - response = key / kden * (1 / (4*7*255))^4, as key (float) times the
//     host-rounded float (1/(4*7*255))^4 / kden (relative error below 3e-7);
//   - level-0 coordinates from the plan's tables (x * scale^level rounded once).
// Records are level-major in rank order: the slot of a kept keypoint is the
// number of keypoints kept by the frame's earlier levels plus its rank.
#include <cuda_runtime.h>

#include "of_internal.h"

namespace ofk {

__global__ void __launch_bounds__(ORIENT_WARPS * 32)
k_orient(const Img* __restrict__ imgs, int img_begin, int n_img, int slot_begin, int slot_end,
         const Call* __restrict__ call, const uint16_t* __restrict__ slot_img) {
    const int slot = slot_begin + blockIdx.x * ORIENT_WARPS + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (slot >= slot_end) return;
    // The slot's image: from the plan's slot table, else a search over slot0.
    int lo = img_begin, hi = img_begin + n_img - 1;
    if (slot_img) {
        lo = __ldg(slot_img + slot);
    } else {
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (imgs[mid].slot0 <= slot) lo = mid; else hi = mid - 1;
        }
    }
    const Img& I = imgs[lo];
    const int rank = slot - I.slot0;
    const int levels = call->levels;
    const Img* F = imgs + I.frame * levels;

    // The frame's first slot publishes its keypoint count.
    if (slot == I.frame * call->n_features) {
        if (lane == 0) {
            int total = 0;
            for (int l = 0; l < levels; ++l) total += F[l].ctr[1];
            // A detect-stage wait that expired leaves partial results: report it instead.
            call->counts[I.frame] = *call->status ? OF_ERR_TIMEOUT : total;
        }
    }
    if (rank >= I.quota || rank >= I.ctr[1]) return;
    int base = 0;
    for (int l = 0; l < I.level; ++l) base += F[l].ctr[1];

    const uint32_t yx = I.kyx[rank];
    const int x = (int)(yx & 0xFFFFu), y = (int)(yx >> 16);
    const uint8_t* img = I.img;
    const int pitch = I.pitch;

    // Harris sums over the 7 x 7 window.
    int a = 0, b = 0, c = 0;
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
        const int p = lane + 32 * rep;
        if (p < 49) {
            const int u = p % 7 - 3, v = p / 7 - 3;
            const uint8_t* q = img + (size_t)(y + v) * pitch + (x + u);
            const int l0 = __ldg(q - pitch - 1), c0 = __ldg(q - pitch), r0 = __ldg(q - pitch + 1);
            const int l1 = __ldg(q - 1), r1 = __ldg(q + 1);
            const int l2 = __ldg(q + pitch - 1), c2 = __ldg(q + pitch), r2 = __ldg(q + pitch + 1);
            const int gx = (r0 - l0) + 2 * (r1 - l1) + (r2 - l2);
            const int gy = (l2 - l0) + 2 * (c2 - c0) + (r2 - r0);
            a += gx * gx;
            b += gy * gy;
            c += gx * gy;
        }
    }
    a = __reduce_add_sync(0xFFFFFFFFu, a);
    b = __reduce_add_sync(0xFFFFFFFFu, b);
    c = __reduce_add_sync(0xFFFFFFFFu, c);

    // Centroid moments.
    const int R = call->radius;
    const int u = lane - 15;
    int m10 = 0, m01 = 0;
    if (u >= -R && u <= R) {
        // Rows in groups of 8 so that each lane has 8 loads in flight.
        const uint8_t* col = img + (size_t)y * pitch + (x + u);
        for (int v0 = -R; v0 <= R; v0 += 8) {
            int iv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int v = v0 + k;
                iv[k] = (v <= R && u * u + v * v <= R * R) ? __ldg(col + (ptrdiff_t)v * pitch) : 0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                m10 += u * iv[k];
                m01 += (v0 + k) * iv[k];
            }
        }
    }
    m10 = __reduce_add_sync(0xFFFFFFFFu, m10);
    m01 = __reduce_add_sync(0xFFFFFFFFu, m01);

    if (lane == 0) {
        const uint64_t okey = I.kkey[rank];
        const int64_t key = (int64_t)(okey ^ 0x8000000000000000ull);
        // response = key / kden * (1/(4*7*255))^4 in float: key as hi * 2^32 + lo
        // (two 32-bit conversions), times the host-rounded scale -- no float64 here
        // (the FP64 pipe was the orientation kernel's busiest unit).
        const float keyf = fmaf((float)(int32_t)(key >> 32), 4294967296.0f, (float)(uint32_t)key);
        of_keypoint k;
        if (I.fx) {
            k.x = I.fx[x];
            k.y = I.fy[y];
        } else {  // no tables: a level-0 image (scale^0 = 1; the allocation-free entry point)
            k.x = (float)x;
            k.y = (float)y;
        }
        k.x_l = x;
        k.y_l = y;
        k.level = I.level;
        k.fast_score = I.score[(size_t)y * I.spitch + x] + (call->t_lo - 1);  // the map holds s - (t_lo - 1)
        k.response = keyf * call->resp_scale;
        k.angle = (m10 == 0 && m01 == 0) ? 0.0f : atan2f((float)m01, (float)m10);
        k.A = a;
        k.B = b;
        k.C = c;
        k.m10 = m10;
        k.m01 = m01;
        k.reserved = 0;
        k.key = key;
        of_keypoint* dst = call->out + (size_t)I.frame * call->n_features + base + rank;
        const uint4* src = reinterpret_cast<const uint4*>(&k);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
        for (int i = 0; i < 4; ++i) d4[i] = src[i];
    }
}

void launch_orient_range(const Img* imgs, int img_begin, int n_img, int slot_begin, int slot_end, const Call* call,
                         void* stream, const uint16_t* slot_img) {
    if (slot_end <= slot_begin || n_img <= 0) return;
    const int blocks = (slot_end - slot_begin + ORIENT_WARPS - 1) / ORIENT_WARPS;
    k_orient<<<blocks, ORIENT_WARPS * 32, 0, (cudaStream_t)stream>>>(imgs, img_begin, n_img, slot_begin, slot_end,
                                                                       call, slot_img);
}

void launch_orient(const Img* imgs, int n_img, const Call* call, int total_slots, void* stream) {
    launch_orient_range(imgs, 0, n_img, 0, total_slots, call, stream, nullptr);
}

// ---------------------------------------------------------------- inspect
__global__ void k_inspect_cells(const Img* imgs, int img, int t_hi, int t_lo, uint8_t* dst) {
    const Img& I = imgs[img];
    const int n = I.ncx * I.ncy;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = (uint8_t)((t_hi != t_lo && I.cell[i]) ? t_hi : t_lo);
}

__global__ void k_inspect_cands(const Img* imgs, int img, int n, uint8_t* dst) {
    const Img& I = imgs[img];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int64_t* d = reinterpret_cast<int64_t*>(dst + 16 * (size_t)i);
        int32_t* d32 = reinterpret_cast<int32_t*>(dst + 16 * (size_t)i + 8);
        d[0] = (int64_t)(I.ckey[i] ^ 0x8000000000000000ull);
        d32[0] = (int32_t)(I.cyx[i] & 0xFFFFu);
        d32[1] = (int32_t)(I.cyx[i] >> 16);
    }
}

void launch_inspect_cells(const Img* imgs, int img, int t_hi, int t_lo, uint8_t* dst,
                          void* stream) {
    k_inspect_cells<<<64, 256, 0, (cudaStream_t)stream>>>(imgs, img, t_hi, t_lo, dst);
}

// S(p) from a dense copy of a map: 0 outside proposed tiles and below t_hi in
// flagged cells, else the offset score + t_lo - 1 (idempotent on final maps).
__global__ void k_inspect_score_final(const Img* imgs, int img, uint8_t* d, int w, int h, int t_hi, int t_lo,
                                      int border, int cell) {
    const Img& I = imgs[img];
    const int rw = w - 2 * border, rh = h - 2 * border;
    if (rw <= 0 || rh <= 0) return;
    const int64_t n = (int64_t)rw * rh;
    const int th = t_hi - t_lo + 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = border + (int)(i % rw), y = border + (int)(i / rw);
        uint8_t* p = d + (size_t)y * w + x;
        int v = *p;
        if (v == 0) continue;
        if (t_hi != t_lo && v < th && I.cell[(size_t)((y - border) / cell) * I.ncx + (x - border) / cell]) v = 0;
        if (I.pmask && I.pmask[(size_t)((y - border) >> 5) * 4 * I.tiles_x + ((x - I.tile_x0) >> 5)] == 0) v = 0;
        *p = (uint8_t)(v ? v + t_lo - 1 : 0);
    }
}

void launch_inspect_score_final(const Img* imgs, int img, uint8_t* d, int w, int h, int t_hi, int t_lo, int border,
                                int cell, void* stream) {
    k_inspect_score_final<<<256, 256, 0, (cudaStream_t)stream>>>(imgs, img, d, w, h, t_hi, t_lo, border, cell);
}

void launch_inspect_cands(const Img* imgs, int img, int n, uint8_t* dst, void* stream) {
    if (n <= 0) return;
    k_inspect_cands<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(imgs, img, n, dst);
}

}  // namespace ofk
