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
// no branches.  The map stores the offset score s(p) - (t_lo - 1) where
// s(p) >= t_lo (the lowest threshold in use), else 0: an order-preserving
// shift that costs nothing (both terms of the final maximum carry a bias of
// 512 - (t_lo - 1) per lane and its floor is 512, so each lane's low byte is
// the offset score) and replaces a clip below t_lo; readers of the map shift
// their thresholds (t_hi -> t_hi - t_lo + 1) and the reported score back.
//
// Data movement.  A thread owns 4 adjacent pixels x..x+3 over RPT rows.  Each
// staged row gives it three 32-bit words (bytes x-4..x+7); one byte permute
// per pair turns them into six 16-bit-lane words (pixel pairs x-4.., x-2..,
// x.., x+2.., x+4.., x+6..).  A ring pixel at an even column offset is one of
// those words; at an odd offset one more permute joins two of them.
//
// Per-cell fallback: a cell with any pixel scoring >= t_hi is flagged.  The
// general kernel sets the flags itself: a thread keeps the running maximum of
// its pixels' scores per cell row (one packed maximum per pixel pair and
// row), compares it with t_hi once per cell row, and ORs its (at most two)
// cells' flags into a per-tile table in shared memory; the tile's flagged
// cells reach the global flags with one atomicOr each, in the next iteration
// after its first barrier.  The threshold pass then only applies them.  The
// cell-tile kernels further down, whose tiles hold whole cells, apply the
// thresholds directly.
//
// Persistent launch: a grid of a few blocks per SM walks all tiles of the
// batch; a 128 x TH tile (TH = 32, 64, 128 or 256 rows) arrives by TMA as
// 1, 2, 4 or 7 stacked 160 x 40 boxes (zero-filled outside the image) into
// one of two shared-memory buffers, so the next tile's load overlaps the
// current tile's arithmetic.  Warps below the detect region skip their rows.
#include <cuda_runtime.h>

#include "of_internal.h"
#include "of_tile.cuh"
#include "of_tma.cuh"

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

// One side of the score for the two pixels in the lanes of q[]: MIN = true
// gives the largest arc minimum max_j min_{k<9} q[j+k], MIN = false the
// smallest arc maximum.  Minima of 3 contiguous ring pixels, then of three
// 3-runs 3 apart (9 pixels), then the extremum over the 16 starts.
template <bool MIN>
__device__ __forceinline__ uint32_t arc_side(const uint32_t (&q)[16]) {
    auto f = [](uint32_t a, uint32_t b, uint32_t c) {
        if constexpr (MIN) return __vimin3_u16x2(a, b, c);
        else return __vimax3_u16x2(a, b, c);
    };
    auto g = [](uint32_t a, uint32_t b, uint32_t c) {
        if constexpr (MIN) return __vimax3_u16x2(a, b, c);
        else return __vimin3_u16x2(a, b, c);
    };
    uint32_t m3[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) m3[i] = f(q[i], q[(i + 1) & 15], q[(i + 2) & 15]);
    uint32_t m9[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) m9[i] = f(m3[i], m3[(i + 3) & 15], m3[(i + 6) & 15]);
    const uint32_t a0 = g(m9[0], m9[1], m9[2]), a1 = g(m9[3], m9[4], m9[5]), a2 = g(m9[6], m9[7], m9[8]);
    const uint32_t a3 = g(m9[9], m9[10], m9[11]), a4 = g(m9[12], m9[13], m9[14]);
    return g(g(a0, a1, a2), a3, g(a4, m9[15], m9[15]));
}

constexpr uint32_t PAIR_BIAS = 0x02000200u;  // 512 per lane: every biased difference stays positive

// For the two pixels of a pair, lanes of 512 + max(amax - c - off, c - amin - off, 0)
// with kb = PAIR_BIAS - off per lane (0 <= off <= 254): the low byte of each
// lane is the offset score max(s(p) - off, 0) (s(p) itself for off = 0).
__device__ __forceinline__ uint32_t pair_score(const uint32_t (&q)[16], uint32_t c, uint32_t kb) {
    const uint32_t amax = arc_side<true>(q);
    const uint32_t amin = arc_side<false>(q);
    return __vimax3_u16x2(amax + kb - c, c + kb - amin, PAIR_BIAS);
}

// 0xFFFF in each 16-bit lane whose value is >= t (values and t below 2^15).
__device__ __forceinline__ uint32_t lanes_ge(uint32_t v, uint32_t t) {
    const uint32_t d = v + (0x8000u - t) * 0x00010001u;
    return ((d >> 15) & 0x00010001u) * 0xFFFFu;
}

// Biased offset score (pair_score) of pixel pair E (pixels x+2E, x+2E+1) of
// an output row from the pair words of staged rows y-3 .. y+3 (hw[0..6]).
template <int E>
__device__ __forceinline__ uint32_t ring_pair_score(const uint32_t (*hw)[6], uint32_t kb) {
    uint32_t q[16];
#define OF_LOAD_RING(i, dx, dy) q[i] = pair_at<(dx) + 2 * E>(hw[3 + (dy)]);
    OF_RING(OF_LOAD_RING)
#undef OF_LOAD_RING
    return pair_score(q, hw[3][2 + E], kb);
}

// s(p) itself, in 16-bit lanes.
template <int E>
__device__ __forceinline__ uint32_t ring_pair_raw(const uint32_t (*hw)[6]) {
    return ring_pair_score<E>(hw, PAIR_BIAS) - PAIR_BIAS;
}

// Interleaved pixel pairs (general kernel): a thread's pixels x..x+3 as the
// pairs (x, x+2) and (x+1, x+3).  Then every ring pixel of either pair, at
// any column offset, is one word of its staged row: e[o + 3] = (c_o, c_{o+2})
// for o = -3..4, c_j the byte at column x + j -- ten instructions per staged
// row (six byte picks and four cross-word joins) and none per output row.
__device__ __forceinline__ void staged_row_words(const uint8_t* row, uint32_t (&e)[8]) {
    const uint32_t w0 = *reinterpret_cast<const uint32_t*>(row - 4);
    const uint32_t w1 = *reinterpret_cast<const uint32_t*>(row);
    const uint32_t w2 = *reinterpret_cast<const uint32_t*>(row + 4);
    const uint32_t w0e = __byte_perm(w0, 0u, 0x4240), w0o = __byte_perm(w0, 0u, 0x4341);  // (c-4, c-2), (c-3, c-1)
    const uint32_t w1e = __byte_perm(w1, 0u, 0x4240), w1o = __byte_perm(w1, 0u, 0x4341);  // (c0, c2), (c1, c3)
    const uint32_t w2e = __byte_perm(w2, 0u, 0x4240), w2o = __byte_perm(w2, 0u, 0x4341);  // (c4, c6), (c5, c7)
    e[0] = w0o;
    e[1] = __byte_perm(w0e, w1e, 0x5432);  // (c-2, c0): high lane of one, low lane of the next
    e[2] = __byte_perm(w0o, w1o, 0x5432);  // (c-1, c1)
    e[3] = w1e;
    e[4] = w1o;
    e[5] = __byte_perm(w1e, w2e, 0x5432);  // (c2, c4)
    e[6] = __byte_perm(w1o, w2o, 0x5432);  // (c3, c5)
    e[7] = w2e;
}

// Biased offset score (pair_score) of interleaved pair C (0: pixels x, x+2;
// 1: x+1, x+3) of an output row from the words of staged rows y-3 .. y+3.
template <int C>
__device__ __forceinline__ uint32_t ring_ipair_score(const uint32_t (*e)[8], uint32_t kb) {
    uint32_t q[16];
#define OF_LOAD_IRING(i, dx, dy) q[i] = e[3 + (dy)][(dx) + C + 3];
    OF_RING(OF_LOAD_IRING)
#undef OF_LOAD_IRING
    return pair_score(q, e[3][C + 3], kb);
}

// The same score with the 7 staged rows held in a rotating window: row k of
// the ring (dy = k - 3) is slot (r + k) % 7.  r is a compile-time constant
// once the caller's row loop is unrolled.
template <int C>
__device__ __forceinline__ uint32_t ring_ipair_score_rot(const uint32_t (*hw)[8], int r, uint32_t kb) {
    uint32_t q[16];
#define OF_LOAD_RRING(i, dx, dy) q[i] = hw[(r + 3 + (dy)) % 7][(dx) + C + 3];
    OF_RING(OF_LOAD_RRING)
#undef OF_LOAD_RRING
    return pair_score(q, hw[(r + 3) % 7][C + 3], kb);
}

// Store the bytes of v selected by mask (0xFF per byte) at d: one word store
// when all four are selected, else byte stores (the other bytes may belong
// to a tile another block writes at the same time).
__device__ __forceinline__ void store_bytes(uint8_t* d, uint32_t v, uint32_t mask) {
    if (mask == 0xFFFFFFFFu) {
        *reinterpret_cast<uint32_t*>(d) = v;
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if ((mask >> (8 * i)) & 1u) d[i] = (uint8_t)(v >> (8 * i));
    }
}

struct CellTile {
    int32_t img, x_lo, y0, box_x;
};

// Tile t of the launch: its image and origin.
struct TileInfo {
    int32_t img, x0, y0;
};

__device__ __forceinline__ TileInfo tile_info(const Img* __restrict__ imgs, const int32_t* __restrict__ list,
                                              const int32_t* __restrict__ prefix, int n_list, int t,
                                              int border, int tile_h) {
    const int j = find_tile_job(prefix, n_list, t);
    const int ii = __ldg(list + j);
    const Img& I = imgs[ii];
    const int tt = t - __ldg(prefix + j);
    const int tx = tt % I.tiles_x, ty = tt / I.tiles_x;
    return TileInfo{ii, I.tile_x0 + tx * TILE_W, border + ty * tile_h};
}

// Work item t of a per-warp kernel from the plan's item table: (image,
// (y0 << 16) | x0), written on the host (no search over the image list).
__device__ __forceinline__ TileInfo item_info(const uint2* __restrict__ items, int t) {
    const uint2 e = __ldg(items + t);
    return TileInfo{(int)e.x, (int)(e.y & 0xFFFFu), (int)(e.y >> 16)};
}

constexpr int FAST_BOX = IMG_BOX_ROWS * SROW;           // bytes per TMA box (160 x 40)
constexpr int FAST_BUF = (FAST_BOX + 127) / 128 * 128;  // buffer stride in shared memory
// Dynamic shared memory of the TH-row kernel: two buffers of stacked boxes + alignment slack.
constexpr int fast_dyn_bytes(int th) { return 2 * ((th + 8 + IMG_BOX_ROWS - 1) / IMG_BOX_ROWS) * FAST_BUF + 128; }

// Cells a 128 x TH tile can overlap (cells of at least 8 pixels).
template <int TH>
struct FastCells {
    static constexpr int LCW = TILE_W / 8 + 2, LCH = TH / 8 + 2, N = LCW * LCH;
};

// The per-tile cell-flag table of one tile, for its flush in the next iteration.
struct FlagTile {
    uint32_t* cell;  // the image's global flags
    int32_t ncx, ncy, cx0, cy0, lcw, n;
};

// Persistent: each block walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// Thread 0 fetches the next tile by TMA into the other buffer while the
// block scores the current one, and the block sets the per-cell "a pixel
// scores >= t_hi" flags.  TH: tile rows, 32, 64, 128 or 256 -- a taller tile
// stacks more image boxes and divides the barriers per pixel and the staged
// rows per output row; 128- and 256-row tiles keep their buffers in dynamic
// shared memory (over the 48 KB static limit).
template <bool FLAGS, int TH>
__global__ void __launch_bounds__(DET_THREADS, TH == 32 ? 3 : 2)
k_fast(const Img* __restrict__ imgs, const int32_t* __restrict__ list,
       const int32_t* __restrict__ prefix, int n_list, int n_tiles, const CUtensorMap* __restrict__ maps,
       const Call* __restrict__ call, int t_hi, int t_lo, int border, int cell, uint32_t cell_magic, int order) {
    // cell_magic = 2^32 / cell rounded up: n / cell == umulhi(n, cell_magic) for 0 <= n < 2^16.
    constexpr int RPT = TH / 8;                                    // rows per thread
    constexpr int LOADS = (TH + 8 + IMG_BOX_ROWS - 1) / IMG_BOX_ROWS;  // image boxes per tile
    constexpr int BUF = LOADS * FAST_BUF;
    constexpr bool DYN = TH > 64;
    __shared__ __align__(128) uint8_t sbuf_static[DYN ? 128 : 2 * BUF];
    extern __shared__ __align__(128) uint8_t fast_dyn[];  // DYN: 2 * BUF bytes from a 128-byte boundary
    uint8_t* const sbuf = DYN ? fast_dyn + ((128u - (smem_u32(fast_dyn) & 127u)) & 127u) : sbuf_static;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ TileInfo tinfo[2];
    __shared__ uint32_t sflag[2][FLAGS ? FastCells<TH>::N : 1];  // per-tile cell flags, by tile parity
    __shared__ FlagTile finfo[2];

    const int tid = threadIdx.x;
    const bool cells = FLAGS && t_hi != t_lo;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_barrier_init();
        finfo[0].n = finfo[1].n = 0;
    }
    for (int i = tid; i < (FLAGS ? 2 * FastCells<TH>::N : 2); i += blockDim.x) (&sflag[0][0])[i] = 0u;
    __syncthreads();
    // The flagged cells of a finished tile (table b) go to the global flags; the table is cleared.
    auto flush_flags = [&](int b) {
        const FlagTile f = finfo[b];
        for (int i = tid; i < f.n; i += blockDim.x) {
            if (sflag[b][i]) {
                const int cx = f.cx0 + i % f.lcw, cy = f.cy0 + i / f.lcw;
                if (cx < f.ncx && cy < f.ncy) atomicOr(&f.cell[cy * f.ncx + cx], 1u);
                sflag[b][i] = 0u;
            }
        }
    };
    auto issue = [&](int t, int b) {
        const TileInfo ti = tile_info(imgs, list, prefix, n_list, t, border, TH);
        tinfo[b] = ti;
        tensormap_acquire(maps + ti.img);
        mbar_arrive_expect_tx(&mbar[b], LOADS * FAST_BOX);
#pragma unroll
        for (int k = 0; k < LOADS; ++k)
            tma_load_2d(sbuf + b * BUF + k * FAST_BOX, maps + ti.img, ti.x0 - HALO_X, ti.y0 - 4 + k * IMG_BOX_ROWS,
                        &mbar[b]);
    };
    const int g = gridDim.x;
    if (tid == 0 && tile_of(order, blockIdx.x, g, n_tiles, 0) < n_tiles) issue(tile_of(order, blockIdx.x, g, n_tiles, 0), 0);

    const int lane = tid & 31, ty = tid >> 5;
    int it = 0;
    for (;; ++it) {
        const int t = tile_of(order, blockIdx.x, g, n_tiles, it);
        if (t >= n_tiles) break;
        const int tn = tile_of(order, blockIdx.x, g, n_tiles, it + 1);
        const int b = it & 1;
        if (tid == 0 && tn < n_tiles) {
            fence_proxy_async_smem();
            issue(tn, b ^ 1);
        }
        const bool ok = mbar_wait(&mbar[b], (it >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(call->status, OF_DEV_TIMEOUT);
                // Let this block's copies in flight land before its shared memory goes away.
                mbar_wait(&mbar[b], (it >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
                if (tn < n_tiles) mbar_wait(&mbar[b ^ 1], ((it + 1) >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
            }
            return;
        }
        if (cells && it > 0) flush_flags(b ^ 1);  // the previous tile's table (its writers passed the barrier)
        const TileInfo ti = tinfo[b];
        const Img& I = imgs[ti.img];
        const uint8_t* s = sbuf + b * BUF;
        const int X0 = ti.x0, Y0 = ti.y0;
        // Learned path: the 4 proposal tiles of each 32-row band of this work
        // tile; skip the tile when all are off.  A warp's rows lie in one band.
        uint32_t pm = 0xFFFFFFFFu, pm_any = 0xFFFFFFFFu;
        if (I.pmask) {
            const int tx = (X0 - I.tile_x0) / TILE_W, tyt = (Y0 - border) / TILE_H;
            const int band = tyt + (ty * RPT) / TILE_H;
            pm = band < I.tiles_y ? *reinterpret_cast<const uint32_t*>(I.pmask + (size_t)band * 4 * I.tiles_x + 4 * tx)
                                  : 0u;
            pm_any = 0u;
            for (int k = 0; k < TH / TILE_H && tyt + k < I.tiles_y; ++k)
                pm_any |= *reinterpret_cast<const uint32_t*>(I.pmask + (size_t)(tyt + k) * 4 * I.tiles_x + 4 * tx);
        }
        if (pm_any == 0u) {
            if (tid == 0) finfo[b].n = 0;
            __syncthreads();
            continue;
        }
        const uint32_t lane_on = ((pm >> (8 * (lane >> 3))) & 0xFFu) ? 0xFFFFFFFFu : 0u;
        const int rx0 = border, rx1 = I.w - border, ry1 = I.h - border;
        const int cx0 = (max(X0, rx0) - rx0) / cell;
        const int cy0 = (Y0 - border) / cell;
        const int lcw = TILE_W / cell + 2;
        const int x = X0 + 4 * lane;
        if (tid == 0) finfo[b] = FlagTile{I.cell, I.ncx, I.ncy, cx0, cy0, lcw, cells ? lcw * (TH / cell + 2) : 0};

        // Eight interleaved pair words per staged row: rows y-3 .. y+RPT+2
        // (staged row 0 is Y0-4), each built just before the first output row
        // that needs it.
        uint32_t hw[RPT + 6][8];
        auto load_row = [&](int k) {
            staged_row_words(s + (ty * RPT + k + 1) * SROW + HALO_X + 4 * lane, hw[k]);
        };
        // Rows of this warp inside the detect region (warp-uniform): a warp
        // below the region's last row (the last tile row of a level) goes
        // straight to the tile barrier, leaving its issue slots to others.
        const int nrows = min(RPT, ry1 - (Y0 + ty * RPT));
        const uint32_t colmask = range_mask4(x, rx0, rx1) & lane_on;
        // Offset scores: the bias of the score's terms, and t_hi in biased offset units.
        const uint32_t kb = PAIR_BIAS - (uint32_t)(t_lo - 1) * 0x00010001u;
        const uint32_t th = (uint32_t)(t_hi - t_lo + 1) + 512u;
        // The score map's address, read once (the stores below could alias the image's fields).
        uint8_t* const sdst = I.score + x;
        const size_t spitch = (size_t)I.spitch;
        // Cell flags: running maxima of the biased offset scores over the
        // current cell row, per pixel pair (two lanes each); the cell row
        // changes at rows y_next, y_next + cell, ...  The cells of a flush are
        // worked out there (the thread's 4 pixels lie in at most two cell
        // columns, the bytes in mask_a in the first), so that nothing but the
        // maxima and y_next stays live across the rows.
        int y_next = border + ((Y0 + ty * RPT - border) / cell + 1) * cell;
        uint32_t mx0 = 0u, mx1 = 0u;
        auto flag_cells = [&](int yc) {  // yc: a row of the cell row being flushed
            const uint32_t strong = __byte_perm(lanes_ge(mx0, th), lanes_ge(mx1, th), 0x6240) & colmask;
            if (strong) {
                const int ca = (int)__umulhi((uint32_t)(max(x, rx0) - rx0), cell_magic);
                const uint32_t mask_a = range_mask4(x, 0, rx0 + (ca + 1) * cell);
                uint32_t* const f =
                    &sflag[b][((int)__umulhi((uint32_t)(yc - border), cell_magic) - cy0) * lcw + (ca - cx0)];
                if (strong & mask_a) atomicOr(f, 1u);
                if (strong & ~mask_a) atomicOr(f + 1, 1u);
            }
        };

        if (nrows > 0) {
#pragma unroll
            for (int k = 0; k < 7; ++k) load_row(k);
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                if (r >= nrows) break;
                const int y = Y0 + ty * RPT + r;
                if (r > 0) load_row(r + 6);
                if (cells && y == y_next) {  // warp-uniform
                    flag_cells(y - 1);
                    mx0 = mx1 = 0u;
                    y_next += cell;
                }
                // Pixel pairs (x, x+2) and (x+1, x+3), one after the other.
                const uint32_t s0 = ring_ipair_score<0>(hw + r, kb);  // 512 + offset score per lane
                const uint32_t s1 = ring_ipair_score<1>(hw + r, kb);
                const uint32_t m = colmask;  // y < ry1 here
                const uint32_t sc = __byte_perm(s0, s1, 0x6240) & m;
                if (m != 0u) *reinterpret_cast<uint32_t*>(sdst + (size_t)y * spitch) = sc;
                if (FLAGS) {
                    mx0 = __vimax3_u16x2(mx0, s0, s0);
                    mx1 = __vimax3_u16x2(mx1, s1, s1);
                }
            }
            if (cells) flag_cells(y_next - 1);
        }
        __syncthreads();  // buffer b is free for the tile after next; the flag table is complete
    }
    if (cells && it > 0) flush_flags((it - 1) & 1);  // the last tile's table
}

void launch_fast(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix, int n_list,
                 int n_tiles, const CUtensorMap* maps, const Call* call, int t_hi, int t_lo, int border,
                 int cell, int grid, int order, void* stream, bool flags, int tile_h) {
    if (n_tiles <= 0) return;
    grid = grid < n_tiles ? grid : n_tiles;
    const cudaStream_t st = (cudaStream_t)stream;
    const uint32_t magic = 0xFFFFFFFFu / (uint32_t)cell + 1u;
#define OF_FAST_LAUNCH(FL, TH, DYN)                                                                            \
    k_fast<FL, TH><<<grid, DET_THREADS, DYN, st>>>(imgs, img_list, tile_prefix, n_list, n_tiles, maps, call, t_hi, \
                                                   t_lo, border, cell, magic, order)
    if (flags) {
        if (tile_h == 64) OF_FAST_LAUNCH(true, 64, 0);
        else if (tile_h == 128) OF_FAST_LAUNCH(true, 128, fast_dyn_bytes(128));
        else if (tile_h == 256) OF_FAST_LAUNCH(true, 256, fast_dyn_bytes(256));
        else OF_FAST_LAUNCH(true, 32, 0);
    } else {
        if (tile_h == 64) OF_FAST_LAUNCH(false, 64, 0);
        else if (tile_h == 128) OF_FAST_LAUNCH(false, 128, fast_dyn_bytes(128));
        else if (tile_h == 256) OF_FAST_LAUNCH(false, 256, fast_dyn_bytes(256));
        else OF_FAST_LAUNCH(false, 32, 0);
    }
#undef OF_FAST_LAUNCH
}

int fast_blocks_per_sm() { return fast_blocks_per_sm(32, true); }

template <bool FL, int TH>
static cudaError_t fast_occupancy(int* n) {
    const int dyn = TH > 64 ? fast_dyn_bytes(TH) : 0;
    cudaError_t e = cudaSuccess;
    if (dyn) e = cudaFuncSetAttribute(k_fast<FL, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_fast<FL, TH>, DET_THREADS, dyn);
    return e;
}

// Resident blocks per SM of the general kernel with tile_h-row tiles, with or
// without the cell flags (for 128 and 256 rows it also raises the kernel's
// dynamic shared-memory limit, before any launch or capture uses it).
int fast_blocks_per_sm(int tile_h, bool flags) {
    int n = 0;
    cudaError_t e;
    if (flags)
        e = tile_h == 64 ? fast_occupancy<true, 64>(&n) : tile_h == 128 ? fast_occupancy<true, 128>(&n)
          : tile_h == 256 ? fast_occupancy<true, 256>(&n) : fast_occupancy<true, 32>(&n);
    else
        e = tile_h == 64 ? fast_occupancy<false, 64>(&n) : tile_h == 128 ? fast_occupancy<false, 128>(&n)
          : tile_h == 256 ? fast_occupancy<false, 256>(&n) : fast_occupancy<false, 32>(&n);
    return (e != cudaSuccess || n < 1) ? 1 : n;
}

// ---------------------------------------------------------------------------
// General FAST with per-warp pipelines: no block barriers.
//
// Each warp is its own persistent worker over the 128 x 32 detect tiles of
// the launch.  Lane 0 fetches the warp's next tile -- one 160 x 40 TMA box,
// rows Y0-4 .. Y0+35, the box the 32-row block kernel uses -- into the warp's
// other shared-memory buffer while the lanes score the current one;
// completion on the warp's own mbarrier, so a warp never waits for another
// warp's tile.  A lane scores 4 pixels (two interleaved pairs) of every row,
// in unrolled chunks of FW_CHUNK = 7 rows over a rotating window of 7 staged
// rows (slot (k mod 7) holds staged row k's words, so the slots line up again
// after each chunk and every staged row's words are built once).  The short
// unrolled body fits the instruction cache: 8-row chunks that rebuilt the
// window's 6 shared rows ran 6 % faster than 16-row chunks and a single
// 33-row chunk 24 % slower; the rotating 7-row window is 2 % faster again.  The score map is as the general kernel's; the cell
// flags are left to the threshold pass.

constexpr int FW_WARPS = DET_THREADS / 32;
constexpr int FW_DYN = FW_WARPS * 2 * FAST_BUF + 128;  // two buffers per warp + alignment slack
constexpr int FW_CHUNK = 7;                              // output rows per unrolled chunk (= window rows)
static_assert(FW_CHUNK == 7, "the rotating window holds the 7 staged rows of one output row");

__global__ void __launch_bounds__(DET_THREADS, 2)
k_fast_warp(const Img* __restrict__ imgs, const int32_t* __restrict__ list, const int32_t* __restrict__ prefix,
            int n_list, int n_tiles, const CUtensorMap* __restrict__ maps, const Call* __restrict__ call, int t_lo,
            int border, int order) {
    extern __shared__ __align__(128) uint8_t fw_dyn[];
    uint8_t* const base = fw_dyn + ((128u - (smem_u32(fw_dyn) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t mbar[FW_WARPS][2];
    __shared__ TileInfo tinfo[FW_WARPS][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint8_t* const wbuf = base + w * 2 * FAST_BUF;
    if (lane == 0) {
        mbar_init(&mbar[w][0], 1);
        mbar_init(&mbar[w][1], 1);
        fence_barrier_init();
    }
    __syncwarp();
    const int nw = gridDim.x * FW_WARPS, gw = blockIdx.x * FW_WARPS + w;
    auto issue = [&](int t, int b) {  // lane 0
        const TileInfo ti = tile_info(imgs, list, prefix, n_list, t, border, TILE_H);
        tinfo[w][b] = ti;
        tensormap_acquire(maps + ti.img);
        mbar_arrive_expect_tx(&mbar[w][b], FAST_BOX);
        tma_load_2d(wbuf + b * FAST_BUF, maps + ti.img, ti.x0 - HALO_X, ti.y0 - 4, &mbar[w][b]);
    };
    if (lane == 0 && tile_of(order, gw, nw, n_tiles, 0) < n_tiles) issue(tile_of(order, gw, nw, n_tiles, 0), 0);
    const uint32_t kb = PAIR_BIAS - (uint32_t)(t_lo - 1) * 0x00010001u;
    for (int it = 0;; ++it) {
        const int t = tile_of(order, gw, nw, n_tiles, it);
        if (t >= n_tiles) break;
        const int tn = tile_of(order, gw, nw, n_tiles, it + 1);
        const int b = it & 1;
        if (lane == 0 && tn < n_tiles) {
            fence_proxy_async_smem();
            issue(tn, b ^ 1);
        }
        const bool ok = mbar_wait(&mbar[w][b], (it >> 1) & 1);
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            if (lane == 0) {
                atomicOr(call->status, OF_DEV_TIMEOUT);
                // Let this warp's copies in flight land before the block's shared memory can go away.
                mbar_wait(&mbar[w][b], (it >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
                if (tn < n_tiles) mbar_wait(&mbar[w][b ^ 1], ((it + 1) >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
            }
            __syncwarp();
            return;
        }
        const TileInfo ti = tinfo[w][b];
        const Img& I = imgs[ti.img];
        const uint8_t* const s = wbuf + b * FAST_BUF;
        const int X0 = ti.x0, Y0 = ti.y0;
        // Learned path: the tile's 4 proposal tiles; skip the tile when all are off.
        uint32_t lane_on = 0xFFFFFFFFu;
        if (I.pmask) {
            const int tx = (X0 - I.tile_x0) / TILE_W, band = (Y0 - border) / TILE_H;
            const uint32_t pm =
                band < I.tiles_y ? *reinterpret_cast<const uint32_t*>(I.pmask + (size_t)band * 4 * I.tiles_x + 4 * tx)
                                 : 0u;
            lane_on = ((pm >> (8 * (lane >> 3))) & 0xFFu) ? 0xFFFFFFFFu : 0u;
            if (pm == 0u) {
                __syncwarp();
                continue;
            }
        }
        const int x = X0 + 4 * lane;
        const int nrows = min(TILE_H, I.h - border - Y0);
        const uint32_t colmask = range_mask4(x, border, I.w - border) & lane_on;
        uint8_t* const sdst = I.score + x;
        const size_t spitch = (size_t)I.spitch;
        const uint8_t* const srow = s + SROW + HALO_X + 4 * lane;  // staged row of output row -3
        uint32_t hw[7][8];
#pragma unroll
        for (int k = 0; k < 6; ++k) staged_row_words(srow + k * SROW, hw[k]);
#pragma unroll 1
        for (int r0 = 0; r0 < nrows; r0 += FW_CHUNK) {
#pragma unroll
            for (int r = 0; r < FW_CHUNK; ++r) {
                if (r0 + r >= nrows) break;
                staged_row_words(srow + (r0 + r + 6) * SROW, hw[(r + 6) % FW_CHUNK]);
                const uint32_t s0 = ring_ipair_score_rot<0>(hw, r, kb);  // 512 + offset score per lane
                const uint32_t s1 = ring_ipair_score_rot<1>(hw, r, kb);
                if (colmask != 0u)
                    *reinterpret_cast<uint32_t*>(sdst + (size_t)(Y0 + r0 + r) * spitch) =
                        __byte_perm(s0, s1, 0x6240) & colmask;
            }
        }
        __syncwarp();  // every lane is done with buffer b before lane 0 refills it
    }
}

void launch_fast_warp(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix, int n_list, int n_tiles,
                      const CUtensorMap* maps, const Call* call, int t_lo, int border, int grid, int order,
                      void* stream) {
    if (n_tiles <= 0) return;
    const int warps = (n_tiles + FW_WARPS - 1) / FW_WARPS;
    grid = grid < warps ? grid : warps;
    k_fast_warp<<<grid, DET_THREADS, FW_DYN, (cudaStream_t)stream>>>(imgs, img_list, tile_prefix, n_list, n_tiles,
                                                                     maps, call, t_lo, border, order);
}

// Resident blocks per SM (also raises the kernel's dynamic shared-memory limit).
int fast_warp_blocks_per_sm() {
    int n = 0;
    if (cudaFuncSetAttribute(k_fast_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_DYN) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fast_warp, DET_THREADS, FW_DYN) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

// ---------------------------------------------------------------------------
// Cell-row strips with per-warp pipelines: the general layout, with the cell
// flags set exactly and cheaply (NMS, or the threshold pass, then applies them).
//
// A work item is one cell row (cell <= 33 rows) of one 128-column detect tile
// column of one image: x in [X0, X0 + 128), y in [y0, y0 + cell), y0 =
// border + cy cell, cut to the detect region; one 160 x 40 TMA box from
// (X0 - 16, y0 - 4) covers its rows and halo.  Warps work as the per-warp
// general kernel (own buffers and mbarriers, no block barriers).  Since the
// strip is exactly one cell row, a lane keeps one running maximum per pixel
// pair over all its rows; at the end one warp OR-reduction gives a bit per
// cell the strip touches (at most 128 / 8 + 2 = 18), and one lane per
// flagged cell ORs it into the global flags (cells at the strip's sides are
// shared with the neighbouring strips).  Images with proposal tiles (the
// learned path) get their flags from the threshold pass instead, which sees
// only proposed pixels; nothing in the row loop depends on the proposal.
// Work items come from the plan's item table (image, x0, y0): lane 0 reads
// one entry per item instead of searching the image list, which was a chain
// of dependent loads the rest of the warp waited on (FAST 2.06 -> 1.99 ms).
// An image's last tile column often holds few region columns (18..52 on
// three of the eight 1080p levels): with at most 64 (32) of them the lanes
// form 2 (4) row groups over the first 64 (32) columns, so fewer lanes idle.

__global__ void __launch_bounds__(DET_THREADS, 2)
k_fast_cstrip(const Img* __restrict__ imgs, const uint2* __restrict__ items, int n_tiles,
              const CUtensorMap* __restrict__ maps, const Call* __restrict__ call, int t_hi, int t_lo, int border,
              int cell, uint32_t cell_magic, int order) {
    // cell_magic = 2^32 / cell rounded up: n / cell == umulhi(n, cell_magic) for 0 <= n < 2^16.
    extern __shared__ __align__(128) uint8_t fw_dyn[];
    uint8_t* const base = fw_dyn + ((128u - (smem_u32(fw_dyn) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t mbar[FW_WARPS][2];
    __shared__ TileInfo tinfo[FW_WARPS][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint8_t* const wbuf = base + w * 2 * FAST_BUF;
    if (lane == 0) {
        mbar_init(&mbar[w][0], 1);
        mbar_init(&mbar[w][1], 1);
        fence_barrier_init();
    }
    __syncwarp();
    const int nw = gridDim.x * FW_WARPS, gw = blockIdx.x * FW_WARPS + w;
    auto issue = [&](int t, int b) {  // lane 0
        const TileInfo ti = item_info(items, t);
        const int ii = ti.img;
        tinfo[w][b] = ti;
        tensormap_acquire(maps + ii);
        mbar_arrive_expect_tx(&mbar[w][b], FAST_BOX);
        tma_load_2d(wbuf + b * FAST_BUF, maps + ii, ti.x0 - HALO_X, ti.y0 - 4, &mbar[w][b]);
    };
    if (lane == 0 && tile_of(order, gw, nw, n_tiles, 0) < n_tiles) issue(tile_of(order, gw, nw, n_tiles, 0), 0);
    const bool cells = t_hi != t_lo;
    const uint32_t kb = PAIR_BIAS - (uint32_t)(t_lo - 1) * 0x00010001u;
    const uint32_t th_b = (uint32_t)(t_hi - t_lo + 1) + 512u;  // t_hi in biased offset units
    for (int it = 0;; ++it) {
        const int t = tile_of(order, gw, nw, n_tiles, it);
        if (t >= n_tiles) break;
        const int tn = tile_of(order, gw, nw, n_tiles, it + 1);
        const int b = it & 1;
        if (lane == 0 && tn < n_tiles) {
            fence_proxy_async_smem();
            issue(tn, b ^ 1);
        }
        const bool ok = mbar_wait(&mbar[w][b], (it >> 1) & 1);
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            if (lane == 0) {
                atomicOr(call->status, OF_DEV_TIMEOUT);
                // Let this warp's copies in flight land before the block's shared memory can go away.
                mbar_wait(&mbar[w][b], (it >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
                if (tn < n_tiles) mbar_wait(&mbar[w][b ^ 1], ((it + 1) >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
            }
            __syncwarp();
            return;
        }
        const TileInfo ti = tinfo[w][b];
        const Img& I = imgs[ti.img];
        const uint8_t* const s = wbuf + b * FAST_BUF;
        const int X0 = ti.x0, y0 = ti.y0;
        const int rx0 = border, rx1 = I.w - border;
        const int nrows = min(cell, I.h - border - y0);
        // A tile column with at most 64 (32) columns of the detect region left:
        // the lanes split into 2 (4) row groups that each score columns
        // X0 .. X0+63 (X0+31) over hq = nrows / groups rows (rounded up).  The
        // last group ends at the strip's last row, overlapping its neighbour
        // when the rows do not divide (those rows are scored twice, identically).
        const int lg = rx1 - X0 <= 32 ? 2 : rx1 - X0 <= 64 ? 1 : 0;
        const int cl = lane & (31 >> lg);  // column lane
        const int hq = (nrows + (1 << lg) - 1) >> lg;
        const int ro = min((lane >> (5 - lg)) * hq, nrows - hq);  // the group's first row
        const int x = X0 + 4 * cl;
        const uint32_t colmask = range_mask4(x, rx0, rx1);
        uint8_t* const sdst = I.score + (size_t)(y0 + ro) * I.spitch + x;
        const size_t spitch = (size_t)I.spitch;
        // Learned path: skip a strip with no proposed tile under it (at most 2 x 4
        // proposal tiles; lanes 0..7 look one up each).  The threshold pass zeroes
        // the scores outside proposed tiles and sets the cell flags of such images.
        const uint8_t* const pmask = I.pmask;
        if (pmask) {
            const int py = ((y0 - border) >> 5) + (lane >> 2);
            const int pxl = ((X0 - I.tile_x0) >> 5) + (lane & 3);
            const bool on = lane < 8 && py <= ((y0 + nrows - 1 - border) >> 5) && py < I.tiles_y &&
                            pmask[(size_t)py * 4 * I.tiles_x + pxl] != 0;
            if (!__any_sync(0xFFFFFFFFu, on)) {
                __syncwarp();
                continue;
            }
        }
        uint32_t mx0 = 0u, mx1 = 0u;
        const uint8_t* const srow = s + (ro + 1) * SROW + HALO_X + 4 * cl;  // staged row of group row -3
        // Rotating window of 7 staged rows: each staged row's words are built once.
        uint32_t hw[7][8];
#pragma unroll
        for (int k = 0; k < 6; ++k) staged_row_words(srow + k * SROW, hw[k]);
#pragma unroll 1
        for (int r0 = 0; r0 < hq; r0 += FW_CHUNK) {
#pragma unroll
            for (int r = 0; r < FW_CHUNK; ++r) {
                if (r0 + r >= hq) break;
                staged_row_words(srow + (r0 + r + 6) * SROW, hw[(r + 6) % FW_CHUNK]);
                const uint32_t s0 = ring_ipair_score_rot<0>(hw, r, kb);  // 512 + offset score per lane
                const uint32_t s1 = ring_ipair_score_rot<1>(hw, r, kb);
                mx0 = __vimax3_u16x2(mx0, s0, s0);
                mx1 = __vimax3_u16x2(mx1, s1, s1);
                if (colmask != 0u)
                    *reinterpret_cast<uint32_t*>(sdst + (size_t)(r0 + r) * spitch) =
                        __byte_perm(s0, s1, 0x6240) & colmask;
            }
        }
        if (lg) {  // the row groups' maxima per column (groups: lane bit 4, and bit 3 for four)
            mx0 = __vimax3_u16x2(mx0, __shfl_xor_sync(0xFFFFFFFFu, mx0, 16), mx0);
            mx1 = __vimax3_u16x2(mx1, __shfl_xor_sync(0xFFFFFFFFu, mx1, 16), mx1);
            if (lg == 2) {
                mx0 = __vimax3_u16x2(mx0, __shfl_xor_sync(0xFFFFFFFFu, mx0, 8), mx0);
                mx1 = __vimax3_u16x2(mx1, __shfl_xor_sync(0xFFFFFFFFu, mx1, 8), mx1);
            }
        }
        if (cells && !pmask) {
            // Bit c: cell cx0 + c of this cell row holds a pixel scoring >= t_hi.
            const int cx0 = (int)__umulhi((uint32_t)(max(X0, rx0) - rx0), cell_magic);
            const int ca = (int)__umulhi((uint32_t)(max(x, rx0) - rx0), cell_magic);
            const uint32_t mask_a = colmask & range_mask4(x, 0, rx0 + (ca + 1) * cell);
            const uint32_t strong = __byte_perm(lanes_ge(mx0, th_b), lanes_ge(mx1, th_b), 0x6240) & colmask;
            const uint32_t bits = ((strong & mask_a) ? 1u << (ca - cx0) : 0u) |
                                  ((strong & ~mask_a) ? 2u << (ca - cx0) : 0u);
            const uint32_t flags = __reduce_or_sync(0xFFFFFFFFu, bits);
            if ((flags >> lane) & 1u)
                atomicOr(&I.cell[(size_t)__umulhi((uint32_t)(y0 - border), cell_magic) * I.ncx + cx0 + lane], 1u);
        }
        __syncwarp();  // every lane is done with buffer b before lane 0 refills it
    }
}

void launch_fast_cstrip(const Img* imgs, const uint2* items, int n_strips, const CUtensorMap* maps, const Call* call,
                        int t_hi, int t_lo, int border, int cell, int grid, int order, void* stream) {
    if (n_strips <= 0) return;
    const int warps = (n_strips + FW_WARPS - 1) / FW_WARPS;
    grid = grid < warps ? grid : warps;
    const uint32_t magic = 0xFFFFFFFFu / (uint32_t)cell + 1u;
    k_fast_cstrip<<<grid, DET_THREADS, FW_DYN, (cudaStream_t)stream>>>(imgs, items, n_strips, maps, call, t_hi, t_lo,
                                                                       border, cell, magic, order);
}

int fast_cstrip_blocks_per_sm() {
    int n = 0;
    if (cudaFuncSetAttribute(k_fast_cstrip, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_DYN) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fast_cstrip, DET_THREADS, FW_DYN) != cudaSuccess ||
        n < 1)
        n = 1;
    return n;
}

// ---------------------------------------------------------------------------
// Cell tiles: FAST with the per-cell threshold applied in the same kernel.
//
// A tile is cpt = floor(124 / cell) whole cells wide and cr = ct_cell_rows
// whole cell rows high (4 x 2 cells = 120 x 60 pixels for 30-pixel cells),
// so it sees every pixel of its cells: it scores them, ORs each cell's "a
// pixel scores >= t_hi" flag in shared memory, and writes the candidate score
// S(p) = s(p) if s(p) >= T(cell(p)) else 0 -- what NMS keys on, stored as
// the offset score S(p) - (t_lo - 1) where nonzero -- and the
// cell flags.  Nothing is accumulated across tiles, so no threshold pass runs
// between FAST and NMS.  A tile's writes wait for its flags: they happen in
// the next iteration, right after the one barrier that ends each tile, from
// the scores the threads keep in registers; the flags rotate through three
// shared-memory slots (ORed in iteration i, read in i + 1, cleared in i + 2).
// Lanes own 4-aligned 4-pixel groups (the first and last groups straddle
// the tile edge and store only their in-tile bytes); warp w owns rows
// 5 (w mod nw) .. +4 of cell row w / nw (nw = ct_warps(cell) warps per cell
// row).  The TMA boxes are 160 x 40 image boxes at x = (group origin - 4)
// rounded down to 16 bytes, starting 3 rows above the tile, stacked.


constexpr int CT_BUF = 2 * FAST_BUF;  // two stacked image boxes

__global__ void __launch_bounds__(32 * CT_MAX_WARPS, 2)
k_fast_cells(const Img* __restrict__ imgs, const int32_t* __restrict__ list, const int32_t* __restrict__ prefix,
             int n_list, int n_tiles, const CUtensorMap* __restrict__ maps, const Call* __restrict__ call,
             int t_hi, int t_lo, int border, int cell, int cpt, int order) {
    __shared__ __align__(128) uint8_t sbuf[2 * CT_BUF];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ CellTile tinfo[2];
    __shared__ uint32_t cflag[3][CT_MAX_CR];
    __shared__ int any_on[2];

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const bool cells = t_hi != t_lo;
    const int nw = ct_warps(cell), cr = ct_cell_rows(cell);
    const int wcr = w / nw, wr = w % nw;  // this warp's cell row in the tile, and its 5-row group there
    const int tw = cpt * cell, th = cr * cell;
    const int srow0 = wcr * cell + CT_RPT * wr;  // the warp's first staged row (staged row 0 = tile row -3)
    const int loads = ((cr - 1) * cell + CT_RPT * nw + 6 + IMG_BOX_ROWS - 1) / IMG_BOX_ROWS;  // 1 or 2
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_barrier_init();
    }
    for (int i = tid; i < 3 * CT_MAX_CR; i += blockDim.x) (&cflag[0][0])[i] = 0u;
    __syncthreads();
    auto issue = [&](int t, int b) {
        const int j = find_tile_job(prefix, n_list, t);
        const int ii = __ldg(list + j);
        const Img& I = imgs[ii];
        const int tt = t - __ldg(prefix + j);
        const int ftx = tt % I.ftiles_x, fty = tt / I.ftiles_x;
        const int x_lo = border + ftx * tw, y0 = border + fty * th;
        const int box_x = ((x_lo & ~3) - 4) & ~15;
        // Learned path: does any proposal tile under this work tile hold a proposed pixel?
        int on = 1;
        if (I.pmask) {
            on = 0;
            const int x_hi = min(x_lo + tw, I.w - border) - 1, y_hi = min(y0 + th, I.h - border) - 1;
            for (int py = (y0 - border) >> 5; py <= (y_hi - border) >> 5 && !on; ++py)
                for (int px = (x_lo - I.tile_x0) >> 5; px <= (x_hi - I.tile_x0) >> 5 && !on; ++px)
                    on = I.pmask[(size_t)py * 4 * I.tiles_x + px] != 0;
        }
        tinfo[b] = CellTile{ii, x_lo, y0, box_x};
        any_on[b] = on;
        tensormap_acquire(maps + ii);
        mbar_arrive_expect_tx(&mbar[b], loads * FAST_BOX);
        for (int k = 0; k < loads; ++k)
            tma_load_2d(sbuf + b * CT_BUF + k * FAST_BOX, maps + ii, box_x, y0 - 3 + k * IMG_BOX_ROWS, &mbar[b]);
    };
    const int g = gridDim.x;
    if (tid == 0 && tile_of(order, blockIdx.x, g, n_tiles, 0) < n_tiles)
        issue(tile_of(order, blockIdx.x, g, n_tiles, 0), 0);

    uint32_t sv[CT_RPT][2];  // this thread's scores of the previous tile (16-bit lanes)
    CellTile prev{-1, 0, 0, 0};
    for (int it = 0;; ++it) {
        const int t = tile_of(order, blockIdx.x, g, n_tiles, it);
        const bool have = t < n_tiles;  // block-uniform
        const int b = it & 1;
        if (tid == 0) {
#pragma unroll
            for (int i = 0; i < CT_MAX_CR; ++i) cflag[(it + 1) % 3][i] = 0u;  // slot of tile it - 2, read in it - 1
            const int tn = tile_of(order, blockIdx.x, g, n_tiles, it + 1);
            if (have && tn < n_tiles) {
                fence_proxy_async_smem();
                issue(tn, b ^ 1);
            }
        }
        const bool ok = have ? mbar_wait(&mbar[b], (it >> 1) & 1) : true;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(call->status, OF_DEV_TIMEOUT);
                // Let this block's copies in flight land before its shared memory goes away.
                mbar_wait(&mbar[b], (it >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
                if (tile_of(order, blockIdx.x, g, n_tiles, it + 1) < n_tiles)
                    mbar_wait(&mbar[b ^ 1], ((it + 1) >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
            }
            return;
        }

        // The previous tile: its flags are complete (the barrier that ended its
        // iteration); write its cell flags and S(p) from the kept scores.
        if (prev.img >= 0) {
            const Img& I = imgs[prev.img];
            const int rx1 = I.w - border, ry1 = I.h - border;
            const int x_hi = min(prev.x_lo + tw, rx1);
            const int x = (prev.x_lo & ~3) + 4 * lane;
            const int row0 = prev.y0 + srow0;
            const int y1 = min(prev.y0 + (wcr + 1) * cell, ry1);
            const uint32_t* fl = cflag[(it - 1) % 3];
            if (tid < cpt * cr) {
                const int cx = (prev.x_lo - border) / cell + tid % cpt, cy = (prev.y0 - border) / cell + tid / cpt;
                if (cx < I.ncx && cy < I.ncy) I.cell[cy * I.ncx + cx] = (fl[tid / cpt] >> (tid % cpt)) & 1u;
            }
            const uint32_t colmask = range_mask4(x, prev.x_lo, x_hi);
            if (row0 < y1 && colmask != 0u) {
                // Cells of this lane's bytes: ca for the bytes in mask_a, ca + 1 for the rest.
                const int ca = (max(x, prev.x_lo) - prev.x_lo) / cell;
                const uint32_t mask_a = colmask & range_mask4(x, 0, prev.x_lo + (ca + 1) * cell);
                const uint32_t flags = fl[wcr];
                const bool fa = (flags >> ca) & 1u, fb = (flags >> (ca + 1)) & 1u;
                uint32_t kk[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const bool flagged = ((mask_a >> (8 * i)) & 1u) ? fa : fb;
                    kk[i] = 0x8000u - (uint32_t)(flagged ? t_hi : t_lo);
                }
                const uint32_t K0 = kk[0] | (kk[1] << 16), K1 = kk[2] | (kk[3] << 16);
                const uint32_t off = (uint32_t)(t_lo - 1) * 0x00010001u;
#pragma unroll
                for (int r = 0; r < CT_RPT; ++r) {
                    const int y = row0 + r;
                    if (y >= y1) break;
                    // Kept lanes (s >= T >= t_lo) store the offset score s - (t_lo - 1).
                    const uint32_t k0 = (((sv[r][0] + K0) >> 15) & 0x00010001u) * 0xFFFFu;
                    const uint32_t k1 = (((sv[r][1] + K1) >> 15) & 0x00010001u) * 0xFFFFu;
                    const uint32_t s0 = (sv[r][0] & k0) - (off & k0);
                    const uint32_t s1 = (sv[r][1] & k1) - (off & k1);
                    store_bytes(I.score + (size_t)y * I.spitch + x, __byte_perm(s0, s1, 0x6420), colmask);
                }
            }
        }
        if (!have) break;

        // This tile: scores into sv, each cell's strong flag into slot it % 3.
        const CellTile ti = tinfo[b];
        prev = ti;
        const Img& I = imgs[ti.img];
        const uint8_t* s = sbuf + b * CT_BUF;
        const int rx1 = I.w - border, ry1 = I.h - border;
        const int x_hi = min(ti.x_lo + tw, rx1);
        const int gx0 = ti.x_lo & ~3;
        const int x = gx0 + 4 * lane;
        const int row0 = ti.y0 + srow0;
        const int y1 = min(ti.y0 + (wcr + 1) * cell, ry1);
        const uint32_t colmask = range_mask4(x, ti.x_lo, x_hi);
#pragma unroll
        for (int r = 0; r < CT_RPT; ++r) sv[r][0] = sv[r][1] = 0u;
        if (any_on[b] && row0 < y1) {  // warp-uniform
            // Six pair words per staged row, loaded just in time.
            uint32_t hw[CT_RPT + 6][6];
            const int xoff = gx0 - ti.box_x + 4 * lane;  // >= 4, multiple of 4
            auto load_row = [&](int k) {
                const uint8_t* row = s + (srow0 + k) * SROW + xoff;
                const uint32_t wm = *reinterpret_cast<const uint32_t*>(row - 4);
                const uint32_t wc = *reinterpret_cast<const uint32_t*>(row);
                const uint32_t wp = *reinterpret_cast<const uint32_t*>(row + 4);
                hw[k][0] = __byte_perm(wm, 0u, 0x4140);
                hw[k][1] = __byte_perm(wm, 0u, 0x4342);
                hw[k][2] = __byte_perm(wc, 0u, 0x4140);
                hw[k][3] = __byte_perm(wc, 0u, 0x4342);
                hw[k][4] = __byte_perm(wp, 0u, 0x4140);
                hw[k][5] = __byte_perm(wp, 0u, 0x4342);
            };
            uint32_t u0 = 0u, u1 = 0u;  // running maxima of the in-tile scores (16-bit lanes)
#pragma unroll
            for (int k = 0; k < 7; ++k) load_row(k);
#pragma unroll
            for (int r = 0; r < CT_RPT; ++r) {
                if (r > 0) load_row(r + 6);
                const int y = row0 + r;
                uint32_t s0 = ring_pair_raw<0>(hw + r);
                uint32_t s1 = ring_pair_raw<1>(hw + r);
                uint32_t m = (y < y1) ? colmask : 0u;
                if (I.pmask && m) {
                    const int px = (x - I.tile_x0) >> 5, py = (y - border) >> 5;
                    if (I.pmask[(size_t)py * 4 * I.tiles_x + px] == 0) m = 0u;
                }
                const uint32_t m0 = __byte_perm(m, 0u, 0x4140), m1 = __byte_perm(m, 0u, 0x4342);
                s0 &= m0;
                s1 &= m1;
                sv[r][0] = s0;
                sv[r][1] = s1;
                u0 = __vimax3_u16x2(u0, s0, s0);
                u1 = __vimax3_u16x2(u1, s1, s1);
            }
            if (cells) {
                const int ca = (max(x, ti.x_lo) - ti.x_lo) / cell;
                const uint32_t mask_a = colmask & range_mask4(x, 0, ti.x_lo + (ca + 1) * cell);
                const uint32_t mask_b = colmask & ~mask_a;
                const uint32_t su = __byte_perm(lanes_ge(u0, (uint32_t)t_hi), lanes_ge(u1, (uint32_t)t_hi), 0x6420);
                uint32_t bits = ((su & mask_a) ? 1u << ca : 0u) | ((su & mask_b) ? 2u << ca : 0u);
                bits = __reduce_or_sync(0xFFFFFFFFu, bits);
                if (lane == 0 && bits) atomicOr(&cflag[it % 3][wcr], bits);
            }
        }
        __syncthreads();  // this tile's flags are complete; buffer b is free for the tile after next
    }
}

void launch_fast_cells(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix, int n_list,
                       int n_tiles, const CUtensorMap* maps, const Call* call, int t_hi, int t_lo, int border,
                       int cell, int grid, int order, void* stream) {
    if (n_tiles <= 0) return;
    grid = grid < n_tiles ? grid : n_tiles;
    const int threads = 32 * ct_warps(cell) * ct_cell_rows(cell), cpt = CT_MAX_W / cell;
    k_fast_cells<<<grid, threads, 0, (cudaStream_t)stream>>>(imgs, img_list, tile_prefix, n_list, n_tiles, maps,
                                                              call, t_hi, t_lo, border, cell, cpt, order);
}

int fast_cells_blocks_per_sm(int cell) {
    const int threads = 32 * ct_warps(cell) * ct_cell_rows(cell);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fast_cells, threads, 0) != cudaSuccess || n < 1) n = 1;
    return n;
}

// ---------------------------------------------------------------------------
// Cell-aligned tiles (cells of 15 or 30 pixels): the general kernel's
// arithmetic on 120 x 120 tiles that hold whole cells, so the per-cell
// threshold is applied here and no threshold pass runs before NMS.
//
// A tile is AL_T x AL_T pixels from (border + 120 i, border + 120 j); warp w
// scores rows 15w .. 15w+14 (one cell row's part: 15 divides the cell), a
// lane the 4-aligned 4-pixel group gx0 + 4 lane (gx0 = x_lo rounded down to
// 4; the first and last groups straddle the tile edge and store only their
// in-tile bytes).  The tile's packed offset scores go to shared memory while
// each warp ORs, per cell, whether a pixel scores >= t_hi; after a barrier
// every thread clears the bytes below t_hi in flagged cells and stores its
// rows, and the tile's cell flags are written.  Image rows y0-3 .. y0+122
// arrive as four stacked 160 x 40 TMA boxes from x = (gx0 - 4) rounded down
// to 16 bytes.
constexpr int AL_T = FAST_AL_T;                                         // tile side
constexpr int AL_RPT = AL_T / (DET_THREADS / 32);                        // rows per warp: 15
constexpr int AL_LOADS = (AL_T + 6 + IMG_BOX_ROWS - 1) / IMG_BOX_ROWS;  // image boxes per tile: 4
constexpr int AL_BUF = AL_LOADS * FAST_BUF;
constexpr int AL_SCO = AL_T * 32 * 4;                                   // packed scores of one tile
constexpr int AL_DYN = 2 * AL_BUF + AL_SCO + 128;                       // + alignment slack
static_assert(AL_RPT * (DET_THREADS / 32) == AL_T, "warps cover the tile's rows");

// 0xFF in each byte of v that is below t (t <= 255).
__device__ __forceinline__ uint32_t bytes_lt(uint32_t v, uint32_t t) {
    const uint32_t tt = (0x8000u - t) * 0x00010001u;
    const uint32_t lo = __byte_perm(v, 0u, 0x4140) + tt, hi = __byte_perm(v, 0u, 0x4342) + tt;
    return ~__byte_perm((lo >> 15 & 0x00010001u) * 0xFFu, (hi >> 15 & 0x00010001u) * 0xFFu, 0x6420);
}

__global__ void __launch_bounds__(DET_THREADS, 2)
k_fast_aligned(const Img* __restrict__ imgs, const int32_t* __restrict__ list, const int32_t* __restrict__ prefix,
               int n_list, int n_tiles, const CUtensorMap* __restrict__ maps, const Call* __restrict__ call,
               int t_hi, int t_lo, int border, int cell, int order) {
    extern __shared__ __align__(128) uint8_t al_dyn[];
    uint8_t* const sbuf = al_dyn + ((128u - (smem_u32(al_dyn) & 127u)) & 127u);
    uint32_t* const sco = reinterpret_cast<uint32_t*>(sbuf + 2 * AL_BUF);  // [row][lane]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ CellTile tinfo[2];
    __shared__ int any_on[2];
    __shared__ uint32_t cflag[AL_T / 15];  // per cell row of the tile: one bit per cell

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const bool cells = t_hi != t_lo;
    const int cpt = AL_T / cell;                // cells per tile row and per tile column
    const int wcr = (AL_RPT * w) / cell;        // this warp's cell row in the tile
    const uint32_t kb = PAIR_BIAS - (uint32_t)(t_lo - 1) * 0x00010001u;
    const uint32_t th = (uint32_t)(t_hi - t_lo + 1);  // t_hi in offset units
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_barrier_init();
    }
    if (tid < AL_T / 15) cflag[tid] = 0u;
    __syncthreads();
    auto issue = [&](int t, int b) {
        const int j = find_tile_job(prefix, n_list, t);
        const int ii = __ldg(list + j);
        const Img& I = imgs[ii];
        const int tt = t - __ldg(prefix + j);
        const int x_lo = border + (tt % I.ftiles_x) * AL_T, y0 = border + (tt / I.ftiles_x) * AL_T;
        const int box_x = ((x_lo & ~3) - 4) & ~15;
        // Learned path: does any proposal tile under this work tile hold a proposed pixel?
        int on = 1;
        if (I.pmask) {
            on = 0;
            const int x_hi = min(x_lo + AL_T, I.w - border) - 1, y_hi = min(y0 + AL_T, I.h - border) - 1;
            for (int py = (y0 - border) >> 5; py <= (y_hi - border) >> 5 && !on; ++py)
                for (int px = (x_lo - I.tile_x0) >> 5; px <= (x_hi - I.tile_x0) >> 5 && !on; ++px)
                    on = I.pmask[(size_t)py * 4 * I.tiles_x + px] != 0;
        }
        tinfo[b] = CellTile{ii, x_lo, y0, box_x};
        any_on[b] = on;
        tensormap_acquire(maps + ii);
        mbar_arrive_expect_tx(&mbar[b], AL_LOADS * FAST_BOX);
#pragma unroll
        for (int k = 0; k < AL_LOADS; ++k)
            tma_load_2d(sbuf + b * AL_BUF + k * FAST_BOX, maps + ii, box_x, y0 - 3 + k * IMG_BOX_ROWS, &mbar[b]);
    };
    const int g = gridDim.x;
    if (tid == 0 && tile_of(order, blockIdx.x, g, n_tiles, 0) < n_tiles)
        issue(tile_of(order, blockIdx.x, g, n_tiles, 0), 0);

    for (int it = 0;; ++it) {
        const int t = tile_of(order, blockIdx.x, g, n_tiles, it);
        if (t >= n_tiles) break;
        const int tn = tile_of(order, blockIdx.x, g, n_tiles, it + 1);
        const int b = it & 1;
        if (tid == 0) {
#pragma unroll
            for (int i = 0; i < AL_T / 15; ++i) cflag[i] = 0u;  // last read before the previous tile's final barrier
            if (tn < n_tiles) {
                fence_proxy_async_smem();
                issue(tn, b ^ 1);
            }
        }
        const bool ok = mbar_wait(&mbar[b], (it >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(call->status, OF_DEV_TIMEOUT);
                // Let this block's copies in flight land before its shared memory goes away.
                mbar_wait(&mbar[b], (it >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
                if (tn < n_tiles) mbar_wait(&mbar[b ^ 1], ((it + 1) >> 1) & 1, OF_WAIT_LIMIT_NS / 8);
            }
            return;
        }
        // Only what the scoring loop needs stays live across it; the masks of
        // the flag and store passes are derived again after it.
        uint32_t* const srow = sco + (size_t)(AL_RPT * w) * 32 + lane;
        int nrows;
        {
            const CellTile ti = tinfo[b];
            const Img& I = imgs[ti.img];
            nrows = min(AL_RPT, min(ti.y0 + AL_T, I.h - border) - (ti.y0 + AL_RPT * w));  // warp-uniform
            if (any_on[b] && nrows > 0) {
                const uint8_t* const s = sbuf + b * AL_BUF;
                const int xoff = (ti.x_lo & ~3) - ti.box_x + 4 * lane;  // >= 4, multiple of 4
                // Six pair words per staged row (staged row 0 = tile row -3), loaded just in time.
                uint32_t hw[AL_RPT + 6][6];
                auto load_row = [&](int k) {
                    const uint8_t* row = s + (AL_RPT * w + k) * SROW + xoff;
                    const uint32_t wm = *reinterpret_cast<const uint32_t*>(row - 4);
                    const uint32_t wc = *reinterpret_cast<const uint32_t*>(row);
                    const uint32_t wp = *reinterpret_cast<const uint32_t*>(row + 4);
                    hw[k][0] = __byte_perm(wm, 0u, 0x4140);
                    hw[k][1] = __byte_perm(wm, 0u, 0x4342);
                    hw[k][2] = __byte_perm(wc, 0u, 0x4140);
                    hw[k][3] = __byte_perm(wc, 0u, 0x4342);
                    hw[k][4] = __byte_perm(wp, 0u, 0x4140);
                    hw[k][5] = __byte_perm(wp, 0u, 0x4342);
                };
#pragma unroll
                for (int k = 0; k < 7; ++k) load_row(k);
#pragma unroll
                for (int r = 0; r < AL_RPT; ++r) {
                    if (r >= nrows) break;
                    if (r > 0) load_row(r + 6);
                    const uint32_t s0 = ring_pair_score<0>(hw + r, kb);  // 512 + offset score per lane
                    const uint32_t s1 = ring_pair_score<1>(hw + r, kb);
                    srow[r * 32] = __byte_perm(s0, s1, 0x6420);          // packed offset scores
                }
            }
        }
        const CellTile ti = tinfo[b];
        const Img& I = imgs[ti.img];
        const int rx1 = I.w - border;
        const int x_hi = min(ti.x_lo + AL_T, rx1);
        const int x = (ti.x_lo & ~3) + 4 * lane;
        const int row0 = ti.y0 + AL_RPT * w;
        const uint32_t colmask = range_mask4(x, ti.x_lo, x_hi);
        // Cells of this lane's bytes: ca for the bytes in mask_a, ca + 1 for the rest.
        const int ca = (max(x, ti.x_lo) - ti.x_lo) / cell;
        const uint32_t mask_a = colmask & range_mask4(x, 0, ti.x_lo + (ca + 1) * cell);
        const uint32_t mask_b = colmask & ~mask_a;
        const bool on = any_on[b];
        if (on && nrows > 0) {
            // Flags: bytes >= t_hi of the in-region, proposed pixels.  Scores
            // outside the proposed tiles (learned path) become 0 here.
            const uint8_t* const pmask = I.pmask;
            uint32_t acc = 0u;
            for (int r = 0; r < nrows; ++r) {
                uint32_t v = srow[r * 32] & colmask;
                if (pmask && colmask) {
                    const int px = (x - I.tile_x0) >> 5, py = (row0 + r - border) >> 5;
                    if (pmask[(size_t)py * 4 * I.tiles_x + px] == 0) {
                        v = 0u;
                        srow[r * 32] = 0u;
                    }
                }
                acc |= ~bytes_lt(v, th);
            }
            if (cells) {
                uint32_t bits = ((acc & mask_a) ? 1u << ca : 0u) | ((acc & mask_b) ? 2u << ca : 0u);
                bits = __reduce_or_sync(0xFFFFFFFFu, bits);
                if (lane == 0 && bits) atomicOr(&cflag[wcr], bits);
            }
        }
        __syncthreads();  // the tile's flags are complete
        if (tid < cpt * cpt) {
            const int cx = (ti.x_lo - border) / cell + tid % cpt, cy = (ti.y0 - border) / cell + tid / cpt;
            if (cx < I.ncx && cy < I.ncy) I.cell[cy * I.ncx + cx] = (cflag[tid / cpt] >> (tid % cpt)) & 1u;
        }
        if (nrows > 0 && colmask != 0u) {
            const uint32_t flags = cflag[wcr];
            const uint32_t fm = (((flags >> ca) & 1u) ? mask_a : 0u) | (((flags >> (ca + 1)) & 1u) ? mask_b : 0u);
            uint8_t* const dst = I.score + x;
            const size_t spitch = (size_t)I.spitch;
#pragma unroll 5
            for (int r = 0; r < AL_RPT; ++r) {
                if (r >= nrows) break;
                const uint32_t v = on ? srow[r * 32] : 0u;
                store_bytes(dst + (size_t)(row0 + r) * spitch, v & ~(fm & bytes_lt(v, th)), colmask);
            }
        }
        fence_proxy_async_smem();  // this thread's buffer accesses before the next TMA into them
        __syncthreads();           // buffer b, the packed scores and cflag are free
    }
}

void launch_fast_aligned(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix, int n_list,
                         int n_tiles, const CUtensorMap* maps, const Call* call, int t_hi, int t_lo, int border,
                         int cell, int grid, int order, void* stream) {
    if (n_tiles <= 0) return;
    grid = grid < n_tiles ? grid : n_tiles;
    k_fast_aligned<<<grid, DET_THREADS, AL_DYN, (cudaStream_t)stream>>>(imgs, img_list, tile_prefix, n_list,
                                                                         n_tiles, maps, call, t_hi, t_lo, border,
                                                                         cell, order);
}

// Resident blocks per SM of the cell-aligned kernel (raises its dynamic
// shared-memory limit first).
int fast_aligned_blocks_per_sm() {
    int n = 0;
    cudaError_t e = cudaFuncSetAttribute(k_fast_aligned, cudaFuncAttributeMaxDynamicSharedMemorySize, AL_DYN);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fast_aligned, DET_THREADS, AL_DYN);
    return (e != cudaSuccess || n < 1) ? 1 : n;
}

// A block that waits, with the same bounded wait as the tile loads, on a flag
// nothing sets; exercises the timeout path without any copy in flight.
__global__ void k_wait_test(const int32_t* flag, int32_t* status, uint64_t limit_ns) {
    if (threadIdx.x == 0 && !flag_wait(flag, limit_ns)) atomicOr(status, OF_DEV_TIMEOUT);
}

void launch_wait_test(const int32_t* flag, int32_t* status, uint64_t limit_ns, void* stream) {
    k_wait_test<<<1, 32, 0, (cudaStream_t)stream>>>(flag, status, limit_ns);
}

}  // namespace ofk
