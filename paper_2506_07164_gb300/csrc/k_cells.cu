// Per-cell threshold applied to FAST score maps in place.
//
// After the general FAST kernel the maps hold s(p) where s(p) >= t_lo, as
// the offset score s(p) - (t_lo - 1) (0 elsewhere), and the cell flags are
// set (a cell is flagged when some pixel in it scores >= t_hi).  This pass
// turns the maps into the candidate scores NMS keys on,
// S(p) = s(p) if s(p) >= T(cell(p)) else 0 with T = t_hi in flagged cells:
// in a flagged cell the bytes below t_hi (t_hi - t_lo + 1 in offset units)
// are cleared.  On the learned path it also clears the scores outside the
// proposed 32 x 32 tiles.
//
// One block per band of cell rows (one cell high) of one image.  With FLAGS
// (when the FAST kernel did not set the flags) the block first ORs, per lane
// and 16-byte chunk, a "byte >= t_hi" bit over the band's rows (three
// instructions per word), maps the set bits to cells in shared memory and
// stores the band's flags.  Then it writes, for up to 4096 columns at a time,
// a byte 0xFF where the column's cell in this band is flagged (all rows of a
// band share their cells' flags), and its warps stream the band's rows in
// 16-byte chunks against that mask, four chunks in flight per lane, writing a
// chunk back only when it changes (the second read of a band mostly hits
// L2).  The byte test "b >= t" takes five instructions per word (bytes_ge).
#include <cuda_runtime.h>
#include <stdint.h>

#include "of_internal.h"
#include "of_tile.cuh"

namespace ofk {

constexpr int CA_THREADS = 256;
constexpr int CA_SEG = 256;  // 16-byte chunks per column-mask segment (4096 columns)

// Bit 7 of each byte of the result is set when that byte of v is >= t
// (1 <= t <= 128; the other bits are garbage): ORed over many words, then
// masked with 0x80808080 once.
__device__ __forceinline__ uint32_t ge_bits(uint32_t v, uint32_t t) { return ((v | 0x80808080u) - t * 0x01010101u) | v; }

// Clear the bytes of v below t where fm is 0xFF (flagged cells).
template <bool SMALL_T>
__device__ __forceinline__ uint32_t apply_word(uint32_t v, uint32_t fm, uint32_t t) {
    return v & ((SMALL_T ? bytes_ge(v, t) : bytes_ge_any(v, t)) | ~fm);
}

template <bool FLAGS, bool APPLY, bool SMALL_T>
__global__ void __launch_bounds__(CA_THREADS)
k_cell_apply(const Img* __restrict__ imgs, const int32_t* __restrict__ list, const int32_t* __restrict__ band_prefix,
             int n_list, int n_bands, int t_hi, int t_lo, int border, int cell, int pmask_only) {
    // FLAGS: set the cell flags (only for images with proposal tiles when pmask_only).
    __shared__ __align__(16) uint8_t colmask[16 * CA_SEG];
    __shared__ uint32_t bflag[FLAGS ? CA_MAX_CELLS : 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool cells = t_hi != t_lo;
    const uint32_t th = (uint32_t)(t_hi - t_lo + 1);  // t_hi in the maps' offset scores (s - (t_lo - 1))
    const uint32_t magic = 0xFFFFFFFFu / (uint32_t)cell + 1u;  // n / cell == umulhi(n, magic) for n < 2^16
    for (int band = blockIdx.x; band < n_bands; band += gridDim.x) {
        const int j = find_tile_job(band_prefix, n_list, band);
        const Img& I = imgs[__ldg(list + j)];
        // The image's fields, read once (the stores below could alias them).
        const uint8_t* const pmask = I.pmask;
        uint8_t* const score = I.score;
        const int spitch = I.spitch, ncx = I.ncx, tiles_x = I.tiles_x, tile_x0 = I.tile_x0;
        if (!cells && !pmask) continue;  // block-uniform
        const int cy = band - __ldg(band_prefix + j);
        const int rx1 = I.w - border, ry1 = I.h - border;
        const int xb0 = border & ~15;  // first chunk column
        const int n_chunks = (rx1 - xb0 + 15) >> 4;
        uint32_t* const crow = I.cell + (size_t)cy * ncx;
        const uint32_t* fl = crow;
        const int y0 = border + cy * cell, y1 = min(y0 + cell, ry1);
        if (FLAGS && cells && (pmask || !pmask_only)) {
            __syncthreads();  // the previous band's readers are done with bflag and colmask
            for (int i = tid; i < ncx; i += CA_THREADS) bflag[i] = 0u;
            __syncthreads();
            for (int c0 = 0; c0 < n_chunks; c0 += 128) {
                uint4 acc[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[k] = make_uint4(0u, 0u, 0u, 0u);
                for (int y = y0 + warp; y < y1; y += CA_THREADS / 32) {
                    const uint8_t* srow = score + (size_t)y * spitch;
                    const int py = (y - border) >> 5;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int c = c0 + lane + 32 * k;
                        if (c >= n_chunks) continue;
                        const int x = xb0 + 16 * c;
                        // Scores outside proposed tiles are stale: they do not count.
                        if (pmask && pmask[(size_t)py * 4 * tiles_x + ((x - tile_x0) >> 5)] == 0) continue;
                        const uint4 v = *reinterpret_cast<const uint4*>(srow + x);
                        if (SMALL_T) {
                            acc[k].x |= ge_bits(v.x, th);
                            acc[k].y |= ge_bits(v.y, th);
                            acc[k].z |= ge_bits(v.z, th);
                            acc[k].w |= ge_bits(v.w, th);
                        } else {
                            acc[k].x |= bytes_ge_any(v.x, th);
                            acc[k].y |= bytes_ge_any(v.y, th);
                            acc[k].z |= bytes_ge_any(v.z, th);
                            acc[k].w |= bytes_ge_any(v.w, th);
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c = c0 + lane + 32 * k;
                    if (c >= n_chunks) continue;
                    const int x = xb0 + 16 * c;
                    const uint32_t wd[4] = {acc[k].x & 0x80808080u, acc[k].y & 0x80808080u,
                                            acc[k].z & 0x80808080u, acc[k].w & 0x80808080u};
                    if ((wd[0] | wd[1] | wd[2] | wd[3]) == 0u) continue;
                    int last = -1;  // last cell flagged by this chunk (adjacent bytes share cells)
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int xx = x + i;
                        if (((wd[i >> 2] >> (8 * (i & 3) + 7)) & 1u) && xx >= border && xx < rx1) {
                            const int cx = (int)__umulhi((uint32_t)(xx - border), magic);
                            if (cx != last) {
                                atomicOr(&bflag[cx], 1u);
                                last = cx;
                            }
                        }
                    }
                }
            }
            __syncthreads();
            for (int i = tid; i < ncx; i += CA_THREADS) crow[i] = bflag[i];
            fl = bflag;
        }
        if constexpr (APPLY) {  // else flags only: NMS applies them on its staged tiles
            for (int s0 = 0; s0 < n_chunks; s0 += CA_SEG) {
                const int s1 = min(s0 + CA_SEG, n_chunks);
                __syncthreads();  // earlier readers of colmask are done
                // Column mask of the segment: 0xFF where the column is in the region and its cell is flagged.
                int any = 0;
                for (int c = s0 + tid; c < s1; c += CA_THREADS) {
                    const int x = xb0 + 16 * c;
                    uint32_t w[4];
    #pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t m = 0u;
                        if (cells) {
    #pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int xx = x + 4 * q + i;
                                if (xx >= border && xx < rx1 && fl[(int)__umulhi((uint32_t)(xx - border), magic)])
                                    m |= 0xFFu << (8 * i);
                            }
                        }
                        w[q] = m;
                        any |= m != 0u;
                    }
                    *reinterpret_cast<uint4*>(colmask + 16 * (c - s0)) = make_uint4(w[0], w[1], w[2], w[3]);
                }
                // A segment with no flagged cell keeps its bytes (unless proposal tiles clear some).
                if (!__syncthreads_or(any) && !pmask) continue;
                for (int y = y0 + warp; y < y1; y += CA_THREADS / 32) {
                    uint8_t* srow = score + (size_t)y * spitch;
                    const int py = (y - border) >> 5;
                    for (int c0 = s0; c0 < s1; c0 += 128) {
                        uint4 v[4];
    #pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int c = c0 + lane + 32 * k;
                            if (c < s1) v[k] = *reinterpret_cast<const uint4*>(srow + xb0 + 16 * c);
                        }
    #pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int c = c0 + lane + 32 * k;
                            if (c >= s1) continue;
                            const int x = xb0 + 16 * c;
                            uint4 nv;
                            if (pmask && pmask[(size_t)py * 4 * tiles_x + ((x - tile_x0) >> 5)] == 0) {
                                // Outside the proposed tiles the region's bytes become 0.
                                nv.x = v[k].x & ~range_mask4(x, border, rx1);
                                nv.y = v[k].y & ~range_mask4(x + 4, border, rx1);
                                nv.z = v[k].z & ~range_mask4(x + 8, border, rx1);
                                nv.w = v[k].w & ~range_mask4(x + 12, border, rx1);
                            } else {
                                const uint4 fm = *reinterpret_cast<const uint4*>(colmask + 16 * (c - s0));
                                nv.x = apply_word<SMALL_T>(v[k].x, fm.x, th);
                                nv.y = apply_word<SMALL_T>(v[k].y, fm.y, th);
                                nv.z = apply_word<SMALL_T>(v[k].z, fm.z, th);
                                nv.w = apply_word<SMALL_T>(v[k].w, fm.w, th);
                            }
                            if (nv.x != v[k].x || nv.y != v[k].y || nv.z != v[k].z || nv.w != v[k].w)
                                *reinterpret_cast<uint4*>(srow + x) = nv;
                        }
                    }
                }
            }
        }
    }
}

void launch_cell_apply(const Img* imgs, const int32_t* img_list, const int32_t* band_prefix, int n_list, int n_bands,
                       int t_hi, int t_lo, int border, int cell, int grid, void* stream, int flags, bool apply) {
    if (n_bands <= 0) return;
    grid = grid < n_bands ? grid : n_bands;
    const cudaStream_t st = (cudaStream_t)stream;
    const bool small_t = t_hi - t_lo + 1 <= 128;
#define OF_CA_LAUNCH(FL, AP, SM)                                                                              \
    k_cell_apply<FL, AP, SM><<<grid, CA_THREADS, 0, st>>>(imgs, img_list, band_prefix, n_list, n_bands, t_hi, t_lo, \
                                                          border, cell, flags == 2)
    if (flags && !apply) {
        if (small_t) OF_CA_LAUNCH(true, false, true);
        else OF_CA_LAUNCH(true, false, false);
    } else if (flags) {
        if (small_t) OF_CA_LAUNCH(true, true, true);
        else OF_CA_LAUNCH(true, true, false);
    } else {
        if (small_t) OF_CA_LAUNCH(false, true, true);
        else OF_CA_LAUNCH(false, true, false);
    }
#undef OF_CA_LAUNCH
}

}  // namespace ofk
