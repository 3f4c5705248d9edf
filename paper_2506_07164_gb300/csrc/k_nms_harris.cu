// Candidate selection, strict 3x3 non-maximum suppression and the Harris key
// of every survivor, fused per 128 x TH tile, TH = 32, 64 or 128 rows (the
// FAST -> Harris fusion of Sec. 5.2: the survivors' Harris sums are computed
// from the same shared-memory tile, with no round trip of points through
// global memory).  The score maps hold offset scores s - (t_lo - 1) (0 where
// s < t_lo); NMS compares them as they are (the shift keeps the order).
//
// Persistent launch; per tile, one thread fetches the TMA boxes into the next
// buffer pair while the block works on the current one: the score rows
// (160 x 34 boxes at a 32-row step, +1 row/col halo) and the image rows
// (160 x 40 boxes, +4 halo), stacked.
// 1. (APPLY variant: the maps hold s(p) where s(p) >= t_lo and the cell
//    flags are set; the final-score variants get maps that already hold S(p)
//    and mask the detect region in registers.)  S(p) in place on the staged
//    score rows: s(p) when p is a candidate at its cell's threshold, else 0;
//    0 outside the detect region and outside proposed tiles.  Each thread
//    keeps one staged word column, whose in-region bytes lie in at most two
//    cells, and a run of rows (one flag lookup per cell row it enters).
// 2. NMS, two pixels per register in 16-bit lanes: p survives when S(p) > the
//    three-input maximum of its 8 neighbours.  Survivors go to a queue (one
//    shared atomic per warp).
// 3. Harris (Eqs. 2-4, Alg. 3): one thread per survivor slides down the 9 x 9
//    footprint keeping three rows of the horizontal Sobel passes (difference
//    [-1 0 1] and smoothing [1 2 1], one byte dot product each from a 4-byte
//    window) in registers -- the circular buffer of Alg. 3 -- and combines
//    them vertically into gx, gy, accumulating the exact int32 sums
//    A = sum gx^2, B = sum gy^2, C = sum gx gy over 7 x 7.
//    key = kden (AB - C^2) - knum (A+B)^2 (int64, exact for k = knum/kden).
// 4. One atomicAdd per warp of the Harris phase reserves its survivors' slots
//    in the image's list.
#include <cuda_runtime.h>

#include <type_traits>

#include "of_internal.h"
#include "of_tile.cuh"
#include "of_tma.cuh"

namespace ofk {

constexpr int S_BOX = SCORE_BOX_ROWS * SROW;     // 5440
constexpr int I_BOX = IMG_BOX_ROWS * SROW;       // 6400
constexpr int S_W0 = HALO_X / 4 - 1;             // first staged word the 3x3 test reads (X0-4)
constexpr int S_WORDS = TILE_W / 4 + 2;          // words X0-4 .. X0+TILE_W+3
constexpr int S_GROUPS = DET_THREADS / S_WORDS;  // row groups of the S(p) pass

// Unsigned bytes of a times signed bytes of b, summed, plus c.
__device__ __forceinline__ int dp4a_us(uint32_t a, uint32_t b, int c) {
    int d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

constexpr uint32_t W_DIFF = 0x000100FFu;  // byte weights (-1, 0, 1, 0): p[u+2] - p[u]
constexpr uint32_t W_SMOOTH = 0x00010201u;  // byte weights (1, 2, 1, 0): p[u] + 2 p[u+1] + p[u+2]

__device__ __forceinline__ void harris_sums(const uint8_t* __restrict__ s, int lx, int ly,
                                            int32_t& A, int32_t& B, int32_t& C) {
    // s: image tile, row 0 = tile row -4, column HALO_X = tile column 0.  A
    // window row is bytes lx-4 .. lx+4: three aligned words, realigned by two
    // funnel shifts; the seven 4-byte windows give both horizontal passes as
    // byte dot products.
    const int start = HALO_X + lx - 4;
    const int w0 = start >> 2, sh = 8 * (start & 3);
    int hd[3][7], hsm[3][7];
    int a = 0, bb = 0, c = 0;
#pragma unroll
    for (int v = -4; v <= 4; ++v) {
        const uint32_t* rp = reinterpret_cast<const uint32_t*>(s + (ly + 4 + v) * SROW) + w0;
        const uint32_t x0 = rp[0], x1 = rp[1], x2 = rp[2];
        const uint32_t r0 = __funnelshift_r(x0, x1, sh), r1 = __funnelshift_r(x1, x2, sh), r2 = x2 >> sh;
        const uint32_t win[7] = {r0, __byte_perm(r0, r1, 0x4321), __byte_perm(r0, r1, 0x5432),
                                 __byte_perm(r0, r1, 0x6543), r1, __byte_perm(r1, r2, 0x4321),
                                 __byte_perm(r1, r2, 0x5432)};
        const int slot = (v + 4) % 3;
#pragma unroll
        for (int u = 0; u < 7; ++u) {
            hd[slot][u] = dp4a_us(win[u], W_DIFF, 0);
            hsm[slot][u] = (int)__dp4a(win[u], W_SMOOTH, 0u);
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

struct NmsTile {
    int32_t img, x0, y0;
};

// Geometry of TH-row NMS tiles: the score box (34 rows) and the image box (40
// rows) are loaded as many times as the tile's rows need, stacked in shared
// memory on 128-byte boundaries (a 64-row tile takes two of each, a 128-row
// tile four): score box k lands at staged row 32k (its first two rows repeat
// the previous box's last two, same bytes), image box k at staged row 40k.
template <int TH>
struct NmsGeom {
    static constexpr int RPT_N = TH / 8;                                    // rows per thread
    static constexpr int S_ROWS_N = TH + 2;                                 // score rows Y0-1 .. Y0+TH
    static constexpr int S_STEP = 32;                                       // staged rows between score boxes
    static constexpr int S_LOADS = (S_ROWS_N - SCORE_BOX_ROWS + S_STEP - 1) / S_STEP + 1;
    static constexpr int I_LOADS = (TH + 8 + IMG_BOX_ROWS - 1) / IMG_BOX_ROWS;  // image rows Y0-4 .. Y0+TH+3
    static constexpr int S_BUF_N = (((S_LOADS - 1) * S_STEP + SCORE_BOX_ROWS) * SROW + 127) / 128 * 128;
    static constexpr int I_BUF_N = (I_LOADS * I_BOX + 127) / 128 * 128;
    static constexpr int QCAP_N = TILE_W * TH / 4;                          // strict maxima are never adjacent
    static constexpr int QBYTES = (2 * QCAP_N + 127) / 128 * 128;             // 16-bit entries
    static constexpr int DYN_BYTES = 2 * I_BUF_N + 2 * S_BUF_N + QBYTES + 128;  // + alignment slack
    static_assert((S_STEP * SROW) % 128 == 0 && I_BOX % 128 == 0, "TMA destinations on 128-byte boundaries");
};

// Queue entries: (tile row << 7) | tile column (rows and columns below 128).
__device__ __forceinline__ uint16_t q_entry(int row, int col) { return (uint16_t)((row << 7) | col); }

// Step 2 for one thread: strict 3x3 maxima of its 4 columns x RPT rows of the
// staged score rows sS (staged row 0 = tile row -1), appended to queue with
// one shared atomic per warp (count in *nq; with nq null the queue is the
// warp's own and the count is returned).  MASK: the staged scores are the
// raw maps, so bytes outside [lox, hix) x [ry0, ry1) are masked here.  Rows
// below the detect region hold no survivor; a warp entirely below it only
// takes part in the queue.
template <bool MASK, int RPT>
__device__ __forceinline__ int nms_queue(const uint8_t* __restrict__ sS, int X0, int Y0, int lox, int hix, int ry0,
                                         int ry1, int lane, int ty, uint16_t* __restrict__ queue, int* nq) {
    const int nrows = min(RPT, ry1 - (Y0 + ty * RPT));
    // Survivor bits (2 * row + pair) * 2 + lane: 4 per row, 64-bit beyond 8 rows.
    using SMask = typename std::conditional<(RPT > 8), unsigned long long, uint32_t>::type;
    SMask smask = 0u;
    if (nrows > 0) {
        // Interleaved pixel pairs: lanes (x, x+2) and (x+1, x+3).  Per staged
        // row the words e0 = (x-1, x+1), e1 = (x, x+2), e2 = (x+1, x+3),
        // e3 = (x+2, x+4) hold every horizontal neighbour of both pairs.
        uint32_t hw[RPT + 2][4];
        // MASK: the in-region bytes of the three words this thread reads.
        uint32_t cm_m = 0xFFFFFFFFu, cm_c = 0xFFFFFFFFu, cm_q = 0xFFFFFFFFu;
        if (MASK) {
            const int xc = X0 + 4 * lane;
            cm_m = range_mask4(xc - 4, lox, hix);
            cm_c = range_mask4(xc, lox, hix);
            cm_q = range_mask4(xc + 4, lox, hix);
        }
#pragma unroll
        for (int k = 0; k < RPT + 2; ++k) {
            const uint8_t* row = sS + (ty * RPT + k) * SROW + HALO_X + 4 * lane;
            uint32_t wm = *reinterpret_cast<const uint32_t*>(row - 4);
            uint32_t wc = *reinterpret_cast<const uint32_t*>(row);
            uint32_t wq = *reinterpret_cast<const uint32_t*>(row + 4);
            if (MASK) {
                const int iy = Y0 - 1 + ty * RPT + k;
                const uint32_t rm = (iy >= ry0 && iy < ry1) ? 0xFFFFFFFFu : 0u;
                wm &= cm_m & rm;
                wc &= cm_c & rm;
                wq &= cm_q & rm;
            }
            hw[k][0] = __byte_perm(wm, wc, 0x0503) & 0x00FF00FFu;  // (x-1, x+1)
            hw[k][1] = __byte_perm(wc, 0u, 0x4240);                 // (x, x+2)
            hw[k][2] = __byte_perm(wc, 0u, 0x4341);                 // (x+1, x+3)
            hw[k][3] = __byte_perm(wc, wq, 0x0402) & 0x00FF00FFu;  // (x+2, x+4)
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) {
                // Pair pr: centre hw[.][1 + pr], left neighbour hw[.][pr], right hw[.][2 + pr].
                const uint32_t* a = hw[r];
                const uint32_t* c = hw[r + 1];
                const uint32_t* d = hw[r + 2];
                const uint32_t nb = __vimax3_u16x2(__vimax3_u16x2(a[pr], a[1 + pr], a[2 + pr]),
                                                   __vimax3_u16x2(c[pr], c[2 + pr], d[pr]),
                                                   __vimax3_u16x2(d[1 + pr], d[2 + pr], d[2 + pr]));
                // Lane bit 15 set when centre > neighbours (values <= 255).
                const uint32_t keep = (c[1 + pr] + 0x7FFF7FFFu - nb) & 0x80008000u;
                const int bit = 2 * (2 * r + pr);
                smask |= (SMask)((keep >> 15) & 1u) << bit | (SMask)(keep >> 31) << (bit + 1);
            }
        }
    }
    // A warp scan of the per-thread counts and one shared atomic per warp.
    const int mine = RPT > 8 ? __popcll((unsigned long long)smask) : __popc((uint32_t)smask);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    // nq null: the queue is the warp's own (entries from 0; the count is returned).
    int wbase = 0;
    if (nq != nullptr && lane == 31 && incl) wbase = atomicAdd(nq, incl);
    int slot = __shfl_sync(0xFFFFFFFFu, wbase, 31) + incl - mine;
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    while (smask) {
        const int bit = (RPT > 8 ? __ffsll((long long)smask) : __ffs((int)smask)) - 1;
        smask &= smask - 1u;
        // bit = 2 (2 row + pair) + lane: column 4 lane + pair + 2 lane
        queue[slot++] = q_entry(ty * RPT + (bit >> 2), 4 * lane + ((bit >> 1) & 1) + 2 * (bit & 1));
    }
    return total;
}

// Step 3-4 for the block: Harris sums and key of every queued survivor of the
// tile at (X0, Y0) of image I, from its staged image rows sI; each warp
// reserves its entries' slots in the image's candidate list with one atomic
// (its latency hides behind the sums).  Block-uniform loop.
template <int NT>
__device__ __forceinline__ void harris_phase(const uint8_t* __restrict__ sI, const uint16_t* __restrict__ queue,
                                             int count, const Img& I, int X0, int Y0, int64_t knum, int64_t kden,
                                             int tid) {
    const int lane = tid & 31, ty = tid >> 5;
    for (int i0 = 0; i0 < count; i0 += NT) {
        const int i = i0 + tid;
        const int n_w = min(max(count - (i0 + 32 * ty), 0), 32);
        int wb = 0;
        if (lane == 0 && n_w > 0) wb = atomicAdd(&I.ctr[0], n_w);
        int32_t A = 0, B = 0, C = 0;
        int lx = 0, ly = 0;
        if (i < count) {
            const uint32_t e = queue[i];
            lx = (int)(e & 127u);
            ly = (int)(e >> 7);
            harris_sums(sI, lx, ly, A, B, C);
        }
        const int slot = __shfl_sync(0xFFFFFFFFu, wb, 0) + lane;
        if (i < count) {
            const int64_t det = (int64_t)A * B - (int64_t)C * C;
            const int64_t tr = (int64_t)A + B;
            const int64_t key = kden * det - knum * tr * tr;
            if (slot < I.cand_cap) {
                I.ckey[slot] = (uint64_t)key ^ 0x8000000000000000ull;
                I.cyx[slot] = ((uint32_t)(Y0 + ly) << 16) | (uint32_t)(X0 + lx);
            } else {
                I.ctr[2] = 1;  // cannot happen: survivors are an independent set
            }
        }
    }
}

// FINAL: the score maps already hold S(p) inside the detect region (a FAST
// kernel or the threshold pass applied the cell thresholds); the kernel masks
// the region in registers.  Otherwise (APPLY) it turns the staged score rows
// into S(p) first.  TH: tile rows (32, 64 or 128 -- fewer barriers per pixel
// and more survivors per Harris phase).  Buffers live in dynamic shared
// memory (NmsGeom<TH>::DYN_BYTES, from a 128-byte boundary).
template <bool FINAL, int TH>
__global__ void __launch_bounds__(DET_THREADS, TH == 32 ? 5 : 4)
k_nms_harris(const Img* __restrict__ imgs, const int32_t* __restrict__ list,
             const int32_t* __restrict__ prefix, int n_list, int n_tiles,
             const CUtensorMap* __restrict__ img_maps, const CUtensorMap* __restrict__ score_maps,
             const Call* __restrict__ call, int t_hi, int t_lo, int border, int cell, uint32_t cell_magic,
             int order) {
    // cell_magic = 2^32 / cell rounded up: n / cell == umulhi(n, cell_magic) for 0 <= n < 2^16.
    using G = NmsGeom<TH>;
    constexpr int RPT = G::RPT_N, S_ROWS = G::S_ROWS_N, S_BUF = G::S_BUF_N, I_BUF = G::I_BUF_N;
    extern __shared__ __align__(128) uint8_t nms_dyn_raw[];
    uint8_t* nms_dyn = nms_dyn_raw + ((128u - (smem_u32(nms_dyn_raw) & 127u)) & 127u);
    uint8_t* ibuf = nms_dyn;
    uint8_t* sbuf = nms_dyn + 2 * I_BUF;
    uint16_t* queue = reinterpret_cast<uint16_t*>(nms_dyn + 2 * I_BUF + 2 * S_BUF);
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ NmsTile tinfo[2];
    __shared__ int nq;

    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](int t, int b) {
        const int j = find_tile_job(prefix, n_list, t);
        const int ii = __ldg(list + j);
        const Img& I = imgs[ii];
        const int tt = t - __ldg(prefix + j);
        const int x0 = I.tile_x0 + (tt % I.tiles_x) * TILE_W, y0 = border + (tt / I.tiles_x) * TH;
        tinfo[b] = NmsTile{ii, x0, y0};
        tensormap_acquire(score_maps + ii);
        tensormap_acquire(img_maps + ii);
        mbar_arrive_expect_tx(&mbar[b], G::S_LOADS * S_BOX + G::I_LOADS * I_BOX);
#pragma unroll
        for (int k = 0; k < G::S_LOADS; ++k)
            tma_load_2d(sbuf + b * S_BUF + k * G::S_STEP * SROW, score_maps + ii, x0 - HALO_X,
                        y0 - 1 + k * G::S_STEP, &mbar[b]);
#pragma unroll
        for (int k = 0; k < G::I_LOADS; ++k)
            tma_load_2d(ibuf + b * I_BUF + k * I_BOX, img_maps + ii, x0 - HALO_X, y0 - 4 + k * IMG_BOX_ROWS,
                        &mbar[b]);
    };
    const int g = gridDim.x;
    if (tid == 0 && tile_of(order, blockIdx.x, g, n_tiles, 0) < n_tiles) issue(tile_of(order, blockIdx.x, g, n_tiles, 0), 0);

    const int lane = tid & 31, ty = tid >> 5;
    const int64_t knum = call->knum, kden = call->kden;
    for (int it = 0;; ++it) {
        const int t = tile_of(order, blockIdx.x, g, n_tiles, it);
        if (t >= n_tiles) break;
        const int tn = tile_of(order, blockIdx.x, g, n_tiles, it + 1);
        const int b = it & 1;
        if (tid == 0) {
            nq = 0;
            if (tn < n_tiles) {
                fence_proxy_async_smem();
                issue(tn, b ^ 1);
            }
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
        const NmsTile ti = tinfo[b];
        const Img& I = imgs[ti.img];
        uint8_t* sS = sbuf + b * S_BUF;
        const uint8_t* sI = ibuf + b * I_BUF;
        const int X0 = ti.x0, Y0 = ti.y0;
        // Learned path: no survivor can lie in a work tile whose proposal tiles are all off.
        if (I.pmask) {
            const int tx = (X0 - I.tile_x0) / TILE_W, tyt = (Y0 - border) / TILE_H;
            uint32_t on = 0u;
            for (int k = 0; k < TH / TILE_H && tyt + k < I.tiles_y; ++k)
                on |= *reinterpret_cast<const uint32_t*>(I.pmask + (size_t)(tyt + k) * 4 * I.tiles_x + 4 * tx);
            if (on == 0u) {
                fence_proxy_async_smem();
                __syncthreads();
                continue;
            }
        }
        const int rx0 = border, rx1 = I.w - border, ry0 = border, ry1 = I.h - border;
        // Only columns X0-1 .. X0+TILE_W feed the 3x3 test; the rest become 0.
        const int lox = max(rx0, X0 - 1), hix = min(rx1, X0 + TILE_W + 1);

        // 1. S(p) in place for rows Y0-1 .. Y0+TH, on the staged words the 3x3
        //    test reads (X0-4 .. X0+TILE_W+3).  A thread keeps one word column
        //    (its in-region byte mask and the at most two cells of its bytes are
        //    fixed for the tile) and a run of consecutive rows.
        if (!FINAL) {
            const int k = S_W0 + tid % S_WORDS, rg = tid / S_WORDS;
            if (rg < S_GROUPS) {
                const int ix = X0 - HALO_X + 4 * k;
                const uint32_t cmask = range_mask4(ix, lox, hix);
                const uint32_t th = (uint32_t)(t_hi - t_lo + 1);  // t_hi in the maps' offset scores
                const bool cells = t_hi != t_lo;
                int ca = 0;
                uint32_t ma = 0u, mb = 0u;
                if (cells && cmask) {
                    ca = (int)__umulhi((uint32_t)(max(ix, lox) - rx0), cell_magic);
                    ma = cmask & range_mask4(ix, 0, rx0 + (ca + 1) * cell);
                    mb = cmask & ~ma;
                }
                int px = 0;
                bool col_on = cmask != 0u;
                if (I.pmask) {
                    px = (ix - I.tile_x0) >> 5;
                    col_on = col_on && ix >= I.tile_x0 && px < 4 * I.tiles_x;
                }
                constexpr int RUN = (S_ROWS + S_GROUPS - 1) / S_GROUPS;
                const int r0 = rg * RUN, r1 = min(r0 + RUN, S_ROWS);
                int y_next = -1;  // first row of the next cell row (none entered yet)
                uint32_t fm = 0u;
                for (int r = r0; r < r1; ++r) {
                    const int iy = Y0 - 1 + r;
                    uint32_t* wp = reinterpret_cast<uint32_t*>(sS + r * SROW) + k;
                    uint32_t val = 0u;
                    bool on = col_on && iy >= ry0 && iy < ry1;
                    if (on && I.pmask) {
                        // Outside the proposed tiles S is 0 (each staged word lies in one proposal tile).
                        const int py = (iy - ry0) >> 5;
                        on = py < I.tiles_y && I.pmask[(size_t)py * 4 * I.tiles_x + px] != 0;
                    }
                    if (on) {
                        val = *wp & cmask;
                        if (cells && val) {
                            if (iy >= y_next) {  // entering a cell row: its flags for this word's bytes
                                const int cy = (int)__umulhi((uint32_t)(iy - ry0), cell_magic);
                                y_next = ry0 + (cy + 1) * cell;
                                const uint32_t* fr = I.cell + (size_t)cy * I.ncx + ca;
                                fm = (ma && fr[0] ? ma : 0u) | (mb && fr[1] ? mb : 0u);
                            }
                            val = apply_cell_threshold(val, fm, th);
                        }
                    }
                    *wp = val;
                }
            }
            __syncthreads();
        }

        // 2. Strict 3x3 maxima, two pixels per register, into the queue.
        nms_queue<FINAL, RPT>(sS, X0, Y0, lox, hix, ry0, ry1, lane, ty, queue, &nq);
        __syncthreads();
        // 3-4. Harris sums and keys of the survivors.
        harris_phase<DET_THREADS>(sI, queue, nq, I, X0, Y0, knum, kden, tid);
        fence_proxy_async_smem();  // this thread's buffer accesses before the next TMA into them
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Per-warp pipelines on the 128 x 32 detect tiles.  Each warp walks its own
// tiles with two shared-memory buffers of its own, one per box -- the tile's
// 34 score rows (160 x 34 from (X0-16, Y0-1)) and its 40 image rows (160 x 40
// from (X0-16, Y0-4)) -- each with its own mbarrier.  Per tile: wait for the
// score box, run the 3x3 test into the warp's queue and refill the score
// buffer with the next tile's box; wait for the image box, compute the Harris
// keys of the queued survivors (rounds of 32, one survivor per lane; a 32-row
// tile holds ~90 at t = 20, so lanes are ~90 % busy) and refill the image
// buffer.  No block barrier: a warp never waits for another warp.
//
// APPLY: the maps hold s(p) - (t_lo - 1) where s(p) >= t_lo (FAST's output)
// and the cell flags are set.  Each staged score word becomes S(p) in
// registers as it is read (bytes below t_hi cleared in flagged cells), so
// the maps need no threshold pass.  A lane thresholds its own word and the
// halo word of the warp's edge (lane 0: columns X0-4..X0-1, lane 31:
// X0+128..X0+131); the 3x3 test's outer neighbours come from lanes +-1.
// A chunk of NW_CHUNK output rows reads 8 new staged rows, which lie in at
// most two cell rows for cells of 8 or more rows.  Otherwise the maps hold
// S(p).  Bytes outside the detect region, and outside the proposed tiles of
// an image that has them, are zeroed in the staged score box first (in the
// words of lanes whose word is not wholly inside).

constexpr int NW_QCAP = TILE_W * TILE_H / 4;             // strict maxima are never adjacent
constexpr int NW_SBUF = (S_BOX + 127) / 128 * 128;       // 5504
constexpr int NW_BYTES = NW_SBUF + I_BOX + 2 * NW_QCAP;  // per warp: score box, image box, queue
constexpr int NW_WARPS = DET_THREADS / 32;
constexpr int NW_DYN = NW_WARPS * NW_BYTES + 128;        // + alignment slack
constexpr int NW_CHUNK = 8;                              // output rows per unrolled chunk (one bit each per byte)
static_assert(NW_BYTES % 128 == 0 && NW_SBUF % 128 == 0, "TMA destinations on 128-byte boundaries");
static_assert(TILE_H % NW_CHUNK == 0, "whole chunks per tile");

// Bytes of a staged word in the detect region, split by cell: ma in cell ca,
// mb in cell ca + 1 (a word's 4 bytes span at most two cells).
struct WordCells {
    uint32_t ma, mb;
    int ca;
};

__device__ __forceinline__ WordCells word_cells(int xw, uint32_t cm, int lox, int rx0, int cell, uint32_t magic) {
    WordCells c{0u, 0u, 0};
    if (cm) {
        c.ca = (int)__umulhi((uint32_t)(max(xw, lox) - rx0), magic);
        c.ma = cm & range_mask4(xw, 0, rx0 + (c.ca + 1) * cell);
        c.mb = cm & ~c.ma;
    }
    return c;
}

// 0xFF over the bytes of a word whose cell in cell row `crow` is flagged.
__device__ __forceinline__ uint32_t word_flags(const WordCells& c, const uint32_t* __restrict__ crow) {
    return (c.ma && crow[c.ca] ? c.ma : 0u) | (c.mb && crow[c.ca + 1] ? c.mb : 0u);
}

// Each byte of the result: the sign (bit 7) of the same byte of g, replicated
// (prmt's sign-extending byte selectors 8..11).
__device__ __forceinline__ uint32_t sign_bytes(uint32_t g) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(g), "r"(0u), "r"(0xBA98u));
    return r;
}

// The bytes of v below th cleared where fm is 0xFF (flagged cells).  For
// th <= 128, bit 7 of ((b | 0x80) - th) | b is set exactly when b >= th (no
// borrow leaves a byte), as in bytes_ge, and its sign replicated is the mask.
template <bool SMALL_T>
__device__ __forceinline__ uint32_t threshold_word(uint32_t v, uint32_t fm, uint32_t th) {
    const uint32_t ge = SMALL_T ? sign_bytes(((v | 0x80808080u) - th * 0x01010101u) | v) : bytes_ge_any(v, th);
    return v & (ge | ~fm);
}

template <bool APPLY, bool SMALL_T>
__global__ void __launch_bounds__(DET_THREADS, 2)
k_nms_warp(const Img* __restrict__ imgs, const uint2* __restrict__ items, int n_tiles,
           const CUtensorMap* __restrict__ img_maps, const CUtensorMap* __restrict__ score_maps,
           const Call* __restrict__ call, int t_hi, int t_lo, int border, int cell, uint32_t cell_magic, int order) {
    extern __shared__ __align__(128) uint8_t nw_raw[];
    uint8_t* const dyn = nw_raw + ((128u - (smem_u32(nw_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t mbar[NW_WARPS][2];  // [0] score box, [1] image box
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint8_t* const sS = dyn + w * NW_BYTES;
    uint8_t* const sI = sS + NW_SBUF;
    uint16_t* const queue = reinterpret_cast<uint16_t*>(sI + I_BOX);
    if (lane == 0) {
        mbar_init(&mbar[w][0], 1);
        mbar_init(&mbar[w][1], 1);
        fence_barrier_init();
    }
    __syncwarp();
    const int nw = gridDim.x * NW_WARPS, gw = blockIdx.x * NW_WARPS + w;
    auto locate = [&](int t) {  // the plan's item table: (image, (y0 << 16) | x0)
        const uint2 e = __ldg(items + t);
        return NmsTile{(int)e.x, (int)(e.y & 0xFFFFu), (int)(e.y >> 16)};
    };
    auto issue_s = [&](const NmsTile& ti) {  // lane 0
        tensormap_acquire(score_maps + ti.img);
        mbar_arrive_expect_tx(&mbar[w][0], S_BOX);
        tma_load_2d(sS, score_maps + ti.img, ti.x0 - HALO_X, ti.y0 - 1, &mbar[w][0]);
    };
    auto issue_i = [&](const NmsTile& ti) {  // lane 0
        tensormap_acquire(img_maps + ti.img);
        mbar_arrive_expect_tx(&mbar[w][1], I_BOX);
        tma_load_2d(sI, img_maps + ti.img, ti.x0 - HALO_X, ti.y0 - 4, &mbar[w][1]);
    };
    int t = tile_of(order, gw, nw, n_tiles, 0);
    NmsTile cur{0, 0, 0};
    if (t < n_tiles) {
        cur = locate(t);
        if (lane == 0) {
            issue_s(cur);
            issue_i(cur);
        }
    }
    const int64_t knum = call->knum, kden = call->kden;
    const uint32_t th = (uint32_t)(t_hi - t_lo + 1);  // t_hi in the maps' offset scores
    for (int it = 0; t < n_tiles; ++it) {
        const int tn = tile_of(order, gw, nw, n_tiles, it + 1);
        const NmsTile nxt = tn < n_tiles ? locate(tn) : cur;
        const uint32_t par = (uint32_t)(it & 1);
        bool ok = mbar_wait(&mbar[w][0], par);
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            if (lane == 0) {
                atomicOr(call->status, OF_DEV_TIMEOUT);
                // Let this warp's copies in flight land before the block's shared memory can go away.
                mbar_wait(&mbar[w][0], par, OF_WAIT_LIMIT_NS / 8);
                mbar_wait(&mbar[w][1], par, OF_WAIT_LIMIT_NS / 8);
            }
            __syncwarp();
            return;
        }
        const Img& I = imgs[cur.img];
        const int X0 = cur.x0, Y0 = cur.y0;
        int n = 0;
        // Learned path: a tile whose four proposal tiles are off holds no survivor.
        bool skip = false;
        if (I.pmask) {
            const int py = (Y0 - border) / TILE_H, px = (X0 - I.tile_x0) / TILE_W;
            skip = *reinterpret_cast<const uint32_t*>(I.pmask + (size_t)py * 4 * I.tiles_x + 4 * px) == 0u;
        }
        if (!skip) {
            const int rx0 = border, rx1 = I.w - border, ry0 = border, ry1 = I.h - border;
            const int xc = X0 + 4 * lane;
            const int xh = lane == 0 ? X0 - 4 : X0 + TILE_W;  // the halo word (used by lanes 0 and 31)
            const int nrows = min(TILE_H, ry1 - Y0);
            const uint8_t* const srow = sS + HALO_X + 4 * lane;
            const int hoff = xh - xc;
            // Zero the staged bytes outside the detect region, and outside the
            // proposed tiles of an image that has them, in the words the 3x3 test
            // reads (staged rows 0 .. nrows + 1; a lane's word, and the halo word of
            // lanes 0 and 31), so that the row loop needs no masks.  Staged row 0 is
            // image row Y0 - 1, rows 1 .. nrows lie in the region, row nrows + 1 is
            // Y0 + nrows.  A word lies in one proposal tile (tile_x0, X0: multiples of 16).
            {
                const uint8_t* const pmask = I.pmask;
                const bool top_in = Y0 - 1 >= ry0, bot_in = Y0 + nrows < ry1;
                auto sanitize = [&](int x, int off) {
                    const uint32_t m = range_mask4(x, rx0, rx1);
                    uint32_t m0 = top_in ? m : 0u, m1 = m, m2 = bot_in ? m : 0u;
                    if (pmask && m) {
                        const int px = (x - I.tile_x0) >> 5, py = (Y0 - ry0) >> 5;
                        auto on = [&](int yy) {
                            return yy >= 0 && yy < I.tiles_y && px >= 0 && px < 4 * I.tiles_x &&
                                   pmask[(size_t)yy * 4 * I.tiles_x + px] != 0;
                        };
                        if (!on(top_in ? (Y0 - 1 - ry0) >> 5 : -1)) m0 = 0u;
                        if (!on(py)) m1 = 0u;
                        if (!on(bot_in ? (Y0 + nrows - ry0) >> 5 : -1)) m2 = 0u;
                    }
                    uint32_t* p = reinterpret_cast<uint32_t*>(sS + HALO_X + off);
                    if (m0 != 0xFFFFFFFFu) p[0] &= m0;
                    if (m1 != 0xFFFFFFFFu)
                        for (int k = 1; k <= nrows; ++k) p[k * (SROW / 4)] &= m1;
                    if (m2 != 0xFFFFFFFFu) p[(nrows + 1) * (SROW / 4)] &= m2;
                };
                sanitize(xc, 4 * lane);
                if (lane == 0 || lane == 31) sanitize(xh, xh - X0);
                __syncwarp();
            }
            WordCells wc_c{0u, 0u, 0}, wc_h{0u, 0u, 0};
            const uint32_t* cellp = I.cell;
            const int ncx = I.ncx;
            if (APPLY) {
                wc_c = word_cells(xc, range_mask4(xc, rx0, rx1), rx0, rx0, cell, cell_magic);
                wc_h = word_cells(xh, range_mask4(xh, rx0, rx1), rx0, rx0, cell, cell_magic);
            }
            // Flag masks of staged row iy (APPLY): cell row of iy (rows outside the region hold zeros).
            auto flags_of = [&](int iy, uint32_t& fc, uint32_t& fh) {
                const int cy = (int)__umulhi((uint32_t)max(iy - ry0, 0), cell_magic);
                const uint32_t* crow = cellp + (size_t)min(cy, I.ncy - 1) * ncx;
                fc = word_flags(wc_c, crow);
                fh = word_flags(wc_h, crow);
            };
            // Staged row k (image row Y0 - 1 + k) reduced to what the 3x3 test takes
            // from it for the pixel pairs (x, x+2) and (x+1, x+3) in 16-bit lanes: the
            // centres, the maxima of the left and right neighbours (the centre row's
            // part) and the maxima of all three (an adjacent row's part).
            struct Row3 {
                uint32_t ctr[2], side[2], all[2];
            };
            auto load_row = [&](int k, uint32_t fc, uint32_t fh) {
                const uint8_t* row = srow + k * SROW;
                uint32_t vc = *reinterpret_cast<const uint32_t*>(row);
                uint32_t vh = *reinterpret_cast<const uint32_t*>(row + hoff);
                if (APPLY) {
                    vc = threshold_word<SMALL_T>(vc, fc, th);
                    vh = threshold_word<SMALL_T>(vh, fh, th);
                }
                uint32_t vm = __shfl_up_sync(0xFFFFFFFFu, vc, 1);
                uint32_t vq = __shfl_down_sync(0xFFFFFFFFu, vc, 1);
                if (lane == 0) vm = vh;
                if (lane == 31) vq = vh;
                const uint32_t h0 = __byte_perm(vm, vc, 0x0503) & 0x00FF00FFu;  // (x-1, x+1)
                const uint32_t h1 = __byte_perm(vc, 0u, 0x4240);                 // (x, x+2)
                const uint32_t h2 = __byte_perm(vc, 0u, 0x4341);                 // (x+1, x+3)
                const uint32_t h3 = __byte_perm(vc, vq, 0x0402) & 0x00FF00FFu;  // (x+2, x+4)
                Row3 o;
                o.ctr[0] = h1;
                o.ctr[1] = h2;
                o.side[0] = __vimax3_u16x2(h0, h2, h2);
                o.side[1] = __vimax3_u16x2(h1, h3, h3);
                o.all[0] = __vimax3_u16x2(h0, h1, h2);
                o.all[1] = __vimax3_u16x2(h1, h2, h3);
                return o;
            };
            Row3 ra, rb;  // staged rows of the output row's upper neighbours and of the row itself
            {
                uint32_t fc = 0u, fh = 0u;
                if (APPLY) flags_of(Y0 - 1, fc, fh);
                ra = load_row(0, fc, fh);
                if (APPLY) flags_of(Y0, fc, fh);
                rb = load_row(1, fc, fh);
            }
#pragma unroll 1
            for (int r0 = 0; r0 < nrows; r0 += NW_CHUNK) {
                // Staged rows r0+2 .. r0+9: cell rows A and (from row yb on) B.
                uint32_t fa_c = 0u, fa_h = 0u, fb_c = 0u, fb_h = 0u;
                int yb = 0;
                if (APPLY) {
                    const int iy0 = Y0 + 1 + r0;
                    flags_of(iy0, fa_c, fa_h);
                    const int cya = (int)__umulhi((uint32_t)max(iy0 - ry0, 0), cell_magic);
                    yb = ry0 + (cya + 1) * cell;
                    if (yb <= iy0 + NW_CHUNK - 1) flags_of(yb, fb_c, fb_h);
                }
                // Survivor bits: byte j (pair j >> 1, lane half j & 1) bit r (chunk row r).
                uint32_t smask = 0u;
#pragma unroll
                for (int r = 0; r < NW_CHUNK; ++r) {
                    if (r0 + r >= nrows) break;
                    const bool b_row = APPLY && Y0 + 1 + r0 + r >= yb;
                    const Row3 rc = load_row(r0 + r + 2, b_row ? fb_c : fa_c, b_row ? fb_h : fa_h);
                    // Lane bit 15 set when the centre > its 8 neighbours (values <= 255).
                    const uint32_t k0 = rb.ctr[0] + 0x7FFF7FFFu - __vimax3_u16x2(ra.all[0], rb.side[0], rc.all[0]);
                    const uint32_t k1 = rb.ctr[1] + 0x7FFF7FFFu - __vimax3_u16x2(ra.all[1], rb.side[1], rc.all[1]);
                    smask |= (__byte_perm(k0, k1, 0x7531) & 0x80808080u) >> (7 - r);
                    ra = rb;
                    rb = rc;
                }
                // Append the chunk's survivors: a warp scan of the per-lane counts.
                const int mine = __popc(smask);
                int incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o) incl += v;
                }
                int slot = n + incl - mine;
                n += __shfl_sync(0xFFFFFFFFu, incl, 31);
                while (smask) {
                    const int bit = __ffs((int)smask) - 1;
                    smask &= smask - 1u;
                    const int j = bit >> 3;  // column 4 lane + pair + 2 half
                    queue[slot++] = q_entry(r0 + (bit & 7), 4 * lane + (j >> 1) + 2 * (j & 1));
                }
            }
        }
        // The score buffer is free: fetch the next tile's score box.
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0 && tn < n_tiles) issue_s(nxt);
        ok = mbar_wait(&mbar[w][1], par);
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            if (lane == 0) {
                atomicOr(call->status, OF_DEV_TIMEOUT);
                mbar_wait(&mbar[w][1], par, OF_WAIT_LIMIT_NS / 8);
                if (tn < n_tiles) mbar_wait(&mbar[w][0], par ^ 1u, OF_WAIT_LIMIT_NS / 8);
            }
            __syncwarp();
            return;
        }
        if (n > 0) harris_phase<32>(sI, queue, n, I, X0, Y0, knum, kden, lane);
        fence_proxy_async_smem();
        __syncwarp();  // every lane is done with the image box and the queue
        if (lane == 0 && tn < n_tiles) issue_i(nxt);
        cur = nxt;
        t = tn;
    }
}

template <bool APPLY, bool SMALL_T>
static void launch_nms_warp_t(const Img* imgs, const uint2* items, int n_tiles, const CUtensorMap* img_maps,
                              const CUtensorMap* score_maps, const Call* call, int t_hi, int t_lo, int border,
                              int cell, int grid, int order, void* stream) {
    const uint32_t magic = 0xFFFFFFFFu / (uint32_t)cell + 1u;
    k_nms_warp<APPLY, SMALL_T><<<grid, DET_THREADS, NW_DYN, (cudaStream_t)stream>>>(
        imgs, items, n_tiles, img_maps, score_maps, call, t_hi, t_lo, border, cell, magic, order);
}

void launch_nms_warp(const Img* imgs, const uint2* items, int n_tiles, const CUtensorMap* img_maps,
                     const CUtensorMap* score_maps, const Call* call, int t_hi, int t_lo, int border, int cell,
                     int grid, int order, void* stream, bool apply) {
    if (n_tiles <= 0) return;
    const int warps = (n_tiles + NW_WARPS - 1) / NW_WARPS;
    grid = grid < warps ? grid : warps;
    apply = apply && t_hi != t_lo;
    if (!apply)
        launch_nms_warp_t<false, true>(imgs, items, n_tiles, img_maps, score_maps, call, t_hi, t_lo, border, cell,
                                       grid, order, stream);
    else if (t_hi - t_lo + 1 <= 128)
        launch_nms_warp_t<true, true>(imgs, items, n_tiles, img_maps, score_maps, call, t_hi, t_lo, border, cell,
                                      grid, order, stream);
    else
        launch_nms_warp_t<true, false>(imgs, items, n_tiles, img_maps, score_maps, call, t_hi, t_lo, border, cell,
                                       grid, order, stream);
}

// Resident blocks per SM of the per-warp NMS kernel (also raises its dynamic shared-memory limit).
int nms_warp_blocks_per_sm() {
    int n = 0, m = 0;
    const cudaError_t e0 = cudaFuncSetAttribute(k_nms_warp<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, NW_DYN);
    const cudaError_t e1 = cudaFuncSetAttribute(k_nms_warp<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, NW_DYN);
    const cudaError_t e2 = cudaFuncSetAttribute(k_nms_warp<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, NW_DYN);
    if (e0 != cudaSuccess || e1 != cudaSuccess || e2 != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_nms_warp<true, true>, DET_THREADS, NW_DYN) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_nms_warp<false, true>, DET_THREADS, NW_DYN) != cudaSuccess)
        return 1;
    n = n < m ? n : m;
    return n < 1 ? 1 : n;
}

template <bool FINAL, int TH>
void launch_nms_t(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix, int n_list, int n_tiles,
                  const CUtensorMap* img_maps, const CUtensorMap* score_maps, const Call* call, int t_hi, int t_lo,
                  int border, int cell, int grid, int order, void* stream) {
    const uint32_t magic = 0xFFFFFFFFu / (uint32_t)cell + 1u;
    k_nms_harris<FINAL, TH><<<grid, DET_THREADS, NmsGeom<TH>::DYN_BYTES, (cudaStream_t)stream>>>(
        imgs, img_list, tile_prefix, n_list, n_tiles, img_maps, score_maps, call, t_hi, t_lo, border, cell, magic,
        order);
}

void launch_nms_harris(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix,
                       int n_list, int n_tiles, const CUtensorMap* img_maps, const CUtensorMap* score_maps,
                       const Call* call, int t_hi, int t_lo, int border, int cell, int grid, int order,
                       void* stream, bool final_scores, int tile_h) {
    if (n_tiles <= 0) return;
    grid = grid < n_tiles ? grid : n_tiles;
#define OF_NMS_LAUNCH(FI, TH)                                                                                  \
    launch_nms_t<FI, TH>(imgs, img_list, tile_prefix, n_list, n_tiles, img_maps, score_maps, call, t_hi, t_lo, \
                         border, cell, grid, order, stream)
    if (final_scores) {
        if (tile_h == 64) OF_NMS_LAUNCH(true, 64);
        else if (tile_h == 128) OF_NMS_LAUNCH(true, 128);
        else OF_NMS_LAUNCH(true, 32);
    } else {
        if (tile_h == 64) OF_NMS_LAUNCH(false, 64);
        else if (tile_h == 128) OF_NMS_LAUNCH(false, 128);
        else OF_NMS_LAUNCH(false, 32);
    }
#undef OF_NMS_LAUNCH
}

// Resident blocks per SM of the NMS kernel with TH-row tiles.  Raises the
// dynamic shared-memory limit where the buffers need it.
template <bool FI, int TH>
static cudaError_t nms_occupancy(int* n) {
    cudaError_t e = cudaFuncSetAttribute(k_nms_harris<FI, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         NmsGeom<TH>::DYN_BYTES);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_nms_harris<FI, TH>, DET_THREADS,
                                                          NmsGeom<TH>::DYN_BYTES);
    return e;
}

int nms_blocks_per_sm(int tile_h, bool final_scores) {
    if (tile_h == 32 && final_scores) return nms_warp_blocks_per_sm();
    int n = 0;
    cudaError_t e;
    if (final_scores)
        e = tile_h == 64 ? nms_occupancy<true, 64>(&n) : tile_h == 128 ? nms_occupancy<true, 128>(&n)
                                                                        : nms_occupancy<true, 32>(&n);
    else
        e = tile_h == 64 ? nms_occupancy<false, 64>(&n) : tile_h == 128 ? nms_occupancy<false, 128>(&n)
                                                                         : nms_occupancy<false, 32>(&n);
    return (e != cudaSuccess || n < 1) ? 1 : n;
}

int nms_blocks_per_sm() { return nms_blocks_per_sm(32, false); }

}  // namespace ofk
