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
#include "of_tma.cuh"

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

// ---------------------------------------------------------------------------
// Persistent TMA resize, separable and exact.
//
// The bilinear value above factors into a horizontal and a vertical step,
// both exact in unsigned 32-bit arithmetic when every weight is doubled:
//   h(r, x) = (4096 - 2ax) S[r][x0] + 2ax S[r][x0 + 1]           (< 2^20)
//   v       = (4096 - 2ay) h(y0, x) + 2ay h(y0 + 1, x) + 2^23    (< 2^32)
//   out     = v >> 24 = ((sum of the original products) + 2^21) >> 22.
// h is one __dp2a_lo or __dp2a_hi (two 16 x 8-bit products) on a byte pair;
// one __byte_perm picks the byte pairs of two outputs into the low and high
// halves of a word; out is byte 3 of v, so four outputs pack with three byte
// permutes.  Where a source index is clamped (x0 = w - 1, y0 = h - 1) the
// tables give that sample's partner weight 0, so the zero fill of the TMA
// box past the image edge never contributes.
//
// Each block walks 128 x 64 output tiles (all frames of one level) and
// fetches the next tile's source window by TMA into the other buffer while
// it filters the current one.  Warp w owns output rows 8w .. 8w + 7; each
// lane owns 4 consecutive output columns and keeps the horizontal values of
// the two source rows under the current output row in registers, computing
// each source row once as the warp moves down.

struct RsTile {
    int32_t job, x0, y0, sx0, sy0;
};

// Horizontal pass of one staged source row for a lane's 4 columns.
__device__ __forceinline__ void hrow(const uint8_t* __restrict__ row, int wa, int wb, const uint32_t (&sel)[4],
                                     const uint32_t (&wgt)[4], uint32_t (&h)[4]) {
    const uint32_t* rp = reinterpret_cast<const uint32_t*>(row);
    const uint32_t a0 = rp[wa], a1 = rp[wa + 1], b0 = rp[wb], b1 = rp[wb + 1];
    // sel[0]: the byte pairs of outputs 0 and 1 in one word (low half, high half); sel[2]: outputs 2 and 3.
    const uint32_t p01 = __byte_perm(a0, a1, sel[0]), p23 = __byte_perm(b0, b1, sel[2]);
    h[0] = __dp2a_lo(wgt[0], p01, 0u);
    h[1] = __dp2a_hi(wgt[1], p01, 0u);
    h[2] = __dp2a_lo(wgt[2], p23, 0u);
    h[3] = __dp2a_hi(wgt[3], p23, 0u);
}

__global__ void __launch_bounds__(RT_THREADS)
k_resize_tma(const Resize* __restrict__ jobs, const uint2* __restrict__ items, int n_tiles,
             const CUtensorMap* __restrict__ maps, const Call* __restrict__ call, int buf_bytes) {
    extern __shared__ __align__(128) uint8_t rdyn[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ RsTile tinfo[2];
    // Two buffers of buf_bytes (a multiple of 128) from a 128-byte boundary;
    // the launch reserves 128 bytes of slack for the rounding.
    uint8_t* rbuf = rdyn + ((128u - (smem_u32(rdyn) & 127u)) & 127u);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](int t, int b) {
        // Tile t from the plan's item table: (job, (Y0 << 16) | X0).
        const uint2 e = __ldg(items + t);
        const int j = (int)e.x;
        const Resize& J = jobs[j];
        const int X0 = (int)(e.y & 0xFFFFu), Y0 = (int)(e.y >> 16);
        const int sx0 = (__ldg(J.xtab + X0) >> 12) & ~15;
        const int sy0 = __ldg(J.ytab + Y0) >> 12;
        tinfo[b] = RsTile{j, X0, Y0, sx0, sy0};
        tensormap_acquire(maps + j);
        mbar_arrive_expect_tx(&mbar[b], (uint32_t)(J.box_w * J.box_h));
        tma_load_2d(rbuf + b * buf_bytes, maps + j, sx0, sy0, &mbar[b]);
    };
    const int g = gridDim.x;
    if (tid == 0 && (int)blockIdx.x < n_tiles) issue(blockIdx.x, 0);

    const int lane = tid & 31, warp = tid >> 5;
    for (int it = 0;; ++it) {
        const int t = blockIdx.x + it * g;
        if (t >= n_tiles) break;
        const int tn = t + g;
        const int b = it & 1;
        if (tid == 0 && tn < n_tiles) {
            fence_proxy_async_smem();
            issue(tn, b ^ 1);
        }
        const bool ok = mbar_wait(&mbar[b], (it >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(call->status, OF_DEV_TIMEOUT);
                mbar_wait(&mbar[b], (it >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
                if (tn < n_tiles) mbar_wait(&mbar[b ^ 1], ((it + 1) >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
            }
            return;
        }
        const RsTile ti = tinfo[b];
        const Resize& J = jobs[ti.job];
        const uint8_t* s = rbuf + b * buf_bytes;
        const int bw = J.box_w;
        const int nx = min(RS_TILE_W, J.dw - ti.x0), ny = min(RT_TILE_H, J.dh - ti.y0);
        const int lx = 4 * lane;
        if (lx < nx) {
            const int n = min(4, nx - lx);
            int xo[4];
            uint32_t wgt[4], sel[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = __ldg(J.xtab + ti.x0 + lx + min(i, n - 1));
                xo[i] = (e >> 12) - ti.sx0;  // byte offset of x0 in the staged row
                const uint32_t a2 = 2u * (uint32_t)(e & 4095);
                wgt[i] = (4096u - a2) | (a2 << 16);
            }
            // Columns 0-1 read the word pair at wa, columns 2-3 the pair at wb;
            // consecutive x0 differ by at most 3, so each byte pair lies in its 8 bytes.
            const int wa = xo[0] >> 2, wb = xo[2] >> 2;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t o = (uint32_t)(xo[i] - 4 * (i < 2 ? wa : wb));
                sel[i] = o | ((o + 1u) << 4);
            }
            sel[0] |= sel[1] << 8;  // outputs 0 and 1 share one permute
            sel[2] |= sel[3] << 8;
            // The job's fields, read once (the stores below could alias them).
            const int dpitch = J.dpitch;
            const int32_t* ytab = J.ytab + ti.y0;
            uint8_t* d = J.dst + (size_t)ti.y0 * dpitch + ti.x0 + lx;
            uint32_t ha[4], hb[4];
            int cur = -4;
            const int ly_end = min(8 * warp + 8, ny);
#pragma unroll
            for (int k = 0; k < 8; ++k) {  // unrolled: the row-table loads are issued together
                const int ly = 8 * warp + k;
                if (ly >= ly_end) break;
                const int e = __ldg(ytab + ly);
                const int r0 = (e >> 12) - ti.sy0;
                const uint32_t a2 = 2u * (uint32_t)(e & 4095);
                if (r0 == cur + 1) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) ha[i] = hb[i];
                    hrow(s + (r0 + 1) * bw, wa, wb, sel, wgt, hb);
                } else if (r0 != cur) {
                    hrow(s + r0 * bw, wa, wb, sel, wgt, ha);
                    hrow(s + (r0 + 1) * bw, wa, wb, sel, wgt, hb);
                }
                cur = r0;
                uint32_t v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) v[i] = (4096u - a2) * ha[i] + a2 * hb[i] + (1u << 23);
                const uint32_t packed =
                    __byte_perm(__byte_perm(v[0], v[1], 0x0073), __byte_perm(v[2], v[3], 0x0073), 0x5410);
                uint8_t* dr = d + (size_t)ly * dpitch;
                if (n == 4) {
                    *reinterpret_cast<uint32_t*>(dr) = packed;  // x0 + lx is a multiple of 4, dpitch of 16
                } else {
                    for (int i = 0; i < n; ++i) dr[i] = (uint8_t)(packed >> (8 * i));
                }
            }
        }
        __syncthreads();  // buffer b is free for the tile after next
    }
}

void launch_resize_tma(const Resize* jobs, const uint2* items, int n_tiles, const CUtensorMap* maps,
                       const Call* call, int buf_bytes, int grid, void* stream) {
    if (n_tiles <= 0) return;
    grid = grid < n_tiles ? grid : n_tiles;
    k_resize_tma<<<grid, RT_THREADS, 2 * buf_bytes + 128, (cudaStream_t)stream>>>(jobs, items, n_tiles, maps, call,
                                                                                   buf_bytes);
}

// The kernel's dynamic shared-memory limit is raised once to the largest
// size any plan may use (two buffers of RT_MAX_BUF), so graphs captured for
// different plans never depend on which plan set it last.
int resize_tma_blocks_per_sm(int buf_bytes) {
    if (buf_bytes <= 0 || buf_bytes > RT_MAX_BUF) return 0;
    if (cudaFuncSetAttribute(k_resize_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * RT_MAX_BUF + 128) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_resize_tma, RT_THREADS, 2 * buf_bytes + 128) !=
        cudaSuccess)
        return 0;
    return n;
}

}  // namespace ofk
