// Internal descriptors shared by the host runtime and the sm_103a kernels.
// Not part of the public ABI (include/ofast.h).
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "ofast.h"

namespace ofk {

// Tile geometry of the detect-stage kernels (FAST score, NMS + Harris).
// A tile is TILE_W x TILE_H pixels; its x origin is a multiple of 16 so that
// 16-byte vector loads stay aligned.  256 threads: 32 columns of 4 pixels
// x 8 rows of RPT pixels.
constexpr int TILE_W = 128;
constexpr int TILE_H = 32;
constexpr int DET_THREADS = 256;
constexpr int RPT = TILE_H / 8;        // rows per thread
constexpr int HALO_X = 16;             // left/right staging margin (bytes), keeps alignment
constexpr int SROW = TILE_W + 2 * HALO_X;  // staged row length (bytes)
constexpr int MAX_CELLS_LOCAL = 128;   // cells overlapping one tile (+halo); needs cell >= 8
constexpr int IMG_BOX_ROWS = TILE_H + 8;   // image TMA box: rows Y0-4 .. Y0+TILE_H+3, SROW bytes wide
constexpr int SCORE_BOX_ROWS = TILE_H + 2; // score TMA box: rows Y0-1 .. Y0+TILE_H

// Cell tiles of the FAST kernel that applies the per-cell threshold itself:
// floor(CT_MAX_W / cell) whole cells wide and ct_cell_rows(cell) cell rows
// high (at most CT_MAX_TILE_ROWS rows); used for cells of CT_MIN_CELL ..
// CT_MAX_CELL pixels.  A warp scores CT_RPT rows of one cell row, so a cell
// row takes ct_warps(cell) warps; a tile's staged rows fit two stacked
// 40-row image boxes.
// Tall tiles of the flag-free FAST kernel (dynamic shared memory).
constexpr int FT_HS[2] = {128, 256};
constexpr int CT_MAX_W = 124;
constexpr int CT_MIN_CELL = 8;
constexpr int CT_MAX_CELL = 30;
constexpr int CT_RPT = 5;             // rows per warp
constexpr int CT_MAX_WARPS = 12;      // warps per block
constexpr int CT_MAX_TILE_ROWS = 64;  // rows per tile
constexpr int CT_MAX_CR = 8;          // cell rows per tile
__host__ __device__ constexpr int ct_warps(int cell) { return (cell + CT_RPT - 1) / CT_RPT; }
__host__ __device__ constexpr int ct_cell_rows(int cell) {
    return CT_MAX_TILE_ROWS / cell < CT_MAX_WARPS / ct_warps(cell) ? CT_MAX_TILE_ROWS / cell
                                                                   : CT_MAX_WARPS / ct_warps(cell);
}
static_assert(ct_cell_rows(CT_MIN_CELL) <= CT_MAX_CR && ct_cell_rows(CT_MAX_CELL) >= 1, "cell rows per tile");

// Resize tile: 128 x (32 or 64) output pixels; each thread writes 4 consecutive pixels
// in 2 or 4 rows.  The autotuner picks the height.
constexpr int RS_TILE_W = 128;
constexpr int RS_TILE_HS[2] = {32, 64};
constexpr int RS_THREADS = 512;

constexpr int SELECT_THREADS = 512;
constexpr int ORIENT_WARPS = 8;        // warps per block in the orientation kernel

// One (frame, level) image of a batch.
struct Img {
    const uint8_t* img;  // level pixels (level 0: caller's frame or its aligned copy)
    uint8_t* score;      // FAST score map, spitch bytes per row
    uint32_t* cell;      // per-cell "has a strong pixel" flags, ncx * ncy
    uint64_t* ckey;      // candidates: order-preserving key (signed key ^ 2^63)
    uint32_t* cyx;       // candidates: (y << 16) | x
    uint64_t* kkey;      // kept (ranked) keys
    uint32_t* kyx;       // kept positions
    int32_t* ctr;        // [0] candidate count, [1] kept count, [2] overflow flag
    int32_t w, h, pitch, spitch;
    int32_t ncx, ncy;
    int32_t cand_cap, quota;
    int32_t frame, level;
    int32_t tiles_x, tiles_y;  // detect-stage tiling (0 when the detect region is empty)
    int32_t tile_x0;           // x origin of tile 0 (multiple of 16)
    int32_t ftiles_x;          // cell tiles per row of the cell-tile FAST kernel (0: not used)
    int32_t slot0;             // first output slot of this image (sum of earlier quotas)
    double lscale;             // scale^level
    // Level-0 coordinates of the level's pixel columns and rows: fx[x] =
    // (float)(x * scale^level), the product taken in float64 and rounded once
    // (on the host).  Null only for a level-0 image (the allocation-free entry
    // point), whose coordinates are x and y themselves.
    const float* fx;
    const float* fy;
    // Learned path: one byte per 32 x 32 proposal tile on the detect-tile grid
    // (4 * tiles_x columns, tiles_y rows, tile (px, py) covers x in
    // [tile_x0 + 32 px, +32), y in [border + 32 py, +32)); 0 = skip.  Null: all on.
    const uint8_t* pmask;
};

// One resize job: dst = bilinear(src).  Tables hold (i0 << 12) | a per
// destination column / row, i0 the first source index and a in [0, 2048].
struct Resize {
    const uint8_t* src;
    uint8_t* dst;
    const int32_t* xtab;
    const int32_t* ytab;
    int32_t sw, sh, spitch;
    int32_t dw, dh, dpitch;
    int32_t tiles_x, tiles_y;
    // Source box of the persistent TMA kernel (box_w a multiple of 16, both
    // <= 256): the largest source window of one RS_TILE_W x RT_TILE_H output
    // tile.  0 when the job is not eligible (scale too large).
    int32_t box_w, box_h;
};

// Persistent TMA resize: 128 x 64 output tiles, 8 warps of 8 output rows.
constexpr int RT_TILE_H = 64;
constexpr int RT_THREADS = 256;
constexpr int RT_MAX_BUF = 100 * 1024;  // largest source buffer (two per block)

// Per-call constants.
struct Call {
    of_keypoint* out;     // n_frames * n_features records
    int32_t* counts;      // n_frames
    int32_t* status;      // device status word (OF_DEV_* bits), cleared before each call
    int64_t knum, kden;   // Harris k = knum / kden
    int32_t n_frames, levels, n_features;
    int32_t t_hi, t_lo;   // t_lo == t_hi: no per-cell fallback
    int32_t border, cell, radius;
    int32_t n_img;        // n_frames * levels
    int32_t total_slots;  // sum of quotas
    float resp_scale;     // (1 / (4*7*255))^4 / kden, rounded to float: response = key * resp_scale
};

// Order in which a persistent block walks the tiles of a launch:
// 0 round-robin (t = block + i * grid), 1 contiguous chunks (t = block * per + i).
__host__ __device__ __forceinline__ int tile_of(int order, int block, int grid, int n_tiles, int i) {
    if (order == 0) return block + i * grid;
    const int per = (n_tiles + grid - 1) / grid;
    return i < per ? block * per + i : n_tiles;
}

}  // namespace ofk

// Kernel launchers (implemented in the .cu files).  All take device pointers
// to the plan's descriptor arrays and launch on `stream`.
namespace ofk {
void launch_resize(const Resize* jobs, const int32_t* tile_prefix, int n_jobs, int n_tiles,
                   int tile_h, void* stream);
void launch_resize_tma(const Resize* jobs, const uint2* items, int n_tiles, const CUtensorMap* maps,
                       const Call* call, int buf_bytes, int grid, void* stream);
int resize_tma_blocks_per_sm(int buf_bytes);  // also raises the kernel's shared-memory limit
// General FAST on 128 x tile_h tiles (32, 64, 128 or 256 rows); flags: also
// set the cell flags (else the threshold pass sets them).
void launch_fast(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix,
                 int n_list, int n_tiles, const CUtensorMap* maps, const Call* call, int t_hi,
                 int t_lo, int border, int cell, int grid, int order, void* stream, bool flags = true,
                 int tile_h = 32);
void launch_fast_cells(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix, int n_list,
                       int n_tiles, const CUtensorMap* maps, const Call* call, int t_hi, int t_lo, int border,
                       int cell, int grid, int order, void* stream);
int fast_cells_blocks_per_sm(int cell);
// Cell-aligned general FAST (120 x 120 tiles of whole cells; cells of 15 or 30 pixels).
constexpr int FAST_AL_T = 120;
inline bool fast_aligned_ok(int cell) { return cell == 15 || cell == 30; }
void launch_fast_aligned(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix, int n_list,
                         int n_tiles, const CUtensorMap* maps, const Call* call, int t_hi, int t_lo, int border,
                         int cell, int grid, int order, void* stream);
int fast_aligned_blocks_per_sm();
int fast_blocks_per_sm(int tile_h, bool flags);  // the general kernel
// General FAST with per-warp pipelines over the 128 x 32 detect tiles (no cell flags).
void launch_fast_warp(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix, int n_list, int n_tiles,
                      const CUtensorMap* maps, const Call* call, int t_lo, int border, int grid, int order,
                      void* stream);
int fast_warp_blocks_per_sm();
// Cell-row strips (one cell row of one 128-column tile per warp item; cells
// of 8..33 pixels): general FAST that also sets the cell flags exactly.
constexpr int CS_MAX_CELL = 33;
void launch_fast_cstrip(const Img* imgs, const uint2* items, int n_strips, const CUtensorMap* maps, const Call* call,
                        int t_hi, int t_lo, int border, int cell, int grid, int order, void* stream);
int fast_cstrip_blocks_per_sm();
// Threshold pass: flags 1: sets the cell flags (when the FAST kernel did
// not), 2: only for images with proposal tiles, 0: never; apply: applies them
// to the maps (else NMS applies them on its staged tiles).
void launch_cell_apply(const Img* imgs, const int32_t* img_list, const int32_t* band_prefix, int n_list, int n_bands,
                       int t_hi, int t_lo, int border, int cell, int grid, void* stream, int flags, bool apply = true);
constexpr int CA_MAX_CELLS = 1024;  // cells per band row the threshold pass can flag itself
void launch_nms_harris(const Img* imgs, const int32_t* img_list, const int32_t* tile_prefix,
                       int n_list, int n_tiles, const CUtensorMap* img_maps,
                       const CUtensorMap* score_maps, const Call* call, int t_hi, int t_lo,
                       int border, int cell, int grid, int order, void* stream,
                       bool final_scores = false, int tile_h = 32);
// Resident blocks per SM of the NMS kernel a plan launches for tile_h (32 with
// final scores: the per-warp kernel).
int nms_blocks_per_sm(int tile_h, bool final_scores);
// Per-warp NMS + Harris on the 128 x 32 detect tiles.  apply: the maps hold
// FAST's offset scores and the cell flags are set (cells of 8 or more rows);
// the kernel applies the per-cell thresholds to the staged words itself.
// Otherwise the maps hold S(p).  Scores outside proposed tiles count as 0.
void launch_nms_warp(const Img* imgs, const uint2* items, int n_tiles, const CUtensorMap* img_maps,
                     const CUtensorMap* score_maps, const Call* call, int t_hi, int t_lo, int border, int cell,
                     int grid, int order, void* stream, bool apply);
int nms_warp_blocks_per_sm();
void launch_select(const Img* imgs, int n_img, const Call* call, int max_quota, void* stream);
void launch_orient(const Img* imgs, int n_img, const Call* call, int total_slots, void* stream);
// Slots [slot_begin, slot_end) of images [img_begin, img_begin + n_img) (one frame group).
void launch_orient_range(const Img* imgs, int img_begin, int n_img, int slot_begin, int slot_end, const Call* call,
                         void* stream, const uint16_t* slot_img = nullptr);
// S(p) of image `img` from a dense w x h copy of its map (offset scores):
// the per-cell thresholds and proposal tiles applied, t_lo - 1 added back.
void launch_inspect_score_final(const Img* imgs, int img, uint8_t* d, int w, int h, int t_hi, int t_lo, int border,
                                int cell, void* stream);
void launch_inspect_cells(const Img* imgs, int img, int t_hi, int t_lo, uint8_t* dst,
                          void* stream);
void launch_inspect_cands(const Img* imgs, int img, int n, uint8_t* dst, void* stream);
int select_smem_bytes(int max_quota);
// Paper ablation variants (k_ablation.cu); returns the number of launches.
int launch_variant(int fast_v, int harris_v, const uint8_t* img, int w, int h, int pitch, int t, int border,
                   int64_t knum, int64_t kden, of_var_point* out, int32_t* count, int cap, int n_sms, void* stream);
}  // namespace ofk
