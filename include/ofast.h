/*
 * ofast.h — C ABI of the GB300 (sm_103a) Oriented FAST detector.
 *
 * Method: "Faster than Fast: Accelerating Oriented FAST Feature Detection on
 * Low-end Embedded GPUs" (arXiv 2506.07164).  One call runs, on the GPU, the
 * whole detection chain of an ORB front end:
 *
 *   1. pyramid: level l is a bilinear resize of level l-1, sizes
 *      w_l = floor(W / scale^l + 0.5) (Sec. 1; Sec. 6.1 "decrease exponentially");
 *   2. FAST-9 segment test with a score (Eq. 1, Sec. 3.1, Alg. 2, Fig. 3);
 *   3. per-cell threshold fallback and strict 3x3 non-maximum suppression
 *      (Fig. 1 "NMS");
 *   4. Harris response from separable Sobel gradients and 7x7 window sums
 *      (Eqs. 2-4, Alg. 3, Fig. 4);
 *   5. top-N per level by Harris response (Sec. 1: Harris "screens" the FAST
 *      points; Sec. 3.2);
 *   6. intensity-centroid orientation (Fig. 1 "Centroid").
 *
 * Conventions for every entry point:
 *   - Pointers marked [device] are CUDA device pointers (e.g. torch tensors'
 *     data_ptr()); [host] pointers are ordinary host memory.
 *   - Images are uint8, row-major, `pitch` bytes between rows; the caller
 *     guarantees `h * pitch` readable bytes.  Level 0 is read in place when
 *     its address and pitch are multiples of 16, otherwise it is first copied
 *     into the handle's scratch (same results, one extra copy).
 *   - The caller owns every buffer it passes; the handle owns all scratch
 *     (pyramid, score maps, candidate lists), allocated once by of_create.
 *   - Work is ordered on the handle's stream (of_params.stream; NULL means the
 *     CUDA default stream).  Nothing traps the GPU: errors are
 *     negative return codes, with a message from of_last_error().
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef OFAST_H
#define OFAST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OF_VERSION 1

/* Return codes (negative = error). */
#define OF_OK 0
#define OF_ERR_ARG (-1)           /* invalid argument (null pointer, size, range) */
#define OF_ERR_TOO_LARGE (-2)     /* request exceeds what the handle was created for */
#define OF_ERR_CUDA (-3)          /* a CUDA runtime call failed (message in of_last_error) */
#define OF_ERR_TIMEOUT (-4)       /* a bounded device-side wait expired */
#define OF_ERR_UNSUPPORTED (-5)   /* valid but not implemented (e.g. harris_block != 7) */

typedef struct of_handle of_handle;

/* Creation parameters.  Zero fields take the default shown. */
typedef struct of_params {
    int32_t max_w, max_h;     /* largest level-0 frame accepted (required, > 0) */
    int32_t max_levels;       /* pyramid levels per frame, 1..16 (default 8) */
    int32_t max_features;     /* largest n_features per frame (default 1000, <= 8192) */
    int32_t max_batch;        /* largest number of frames per call (default 1) */
    float min_scale;          /* smallest pyramid scale accepted, > 1 (default 1.2);
                                 scratch is sized for pyramids of this scale */
    int32_t fast_t_lo;        /* per-cell fallback FAST threshold: a 30x30 cell with no
                                 pixel scoring >= fast_t uses fast_t_lo instead.
                                 0 (default) disables the fallback. */
    int32_t cell;             /* fallback cell side in pixels (default 30) */
    int32_t border;           /* pixels excluded at each level edge (default 19; >= orient_radius, >= 4) */
    int32_t harris_block;     /* Harris window side (default 7; only 7 is implemented) */
    int32_t orient_radius;    /* centroid disc radius (default 15; 1..15) */
    void* stream;             /* cudaStream_t to order work on; NULL = the CUDA default stream */
    int32_t autotune;         /* 1: run of_autotune's search when a new batch shape is first seen */
    int64_t arena_bytes;      /* > 0: scratch size in bytes instead of the worst case for max_batch
                                 frames of max_w x max_h; a batch that needs more is rejected with
                                 OF_ERR_TOO_LARGE (see of_batch_bytes) */
} of_params;

/* Launch configuration of one batch shape, as chosen by of_autotune (or the
 * defaults before tuning). */
typedef struct of_tuning {
    int32_t resize_tile_h;        /* pyramid output tile height: 32 or 64 rows */
    int32_t fast_blocks_per_sm;   /* persistent FAST grid = SMs x this */
    int32_t nms_blocks_per_sm;    /* persistent NMS + Harris grid = SMs x this */
    int32_t fast_order;           /* tile walk: 0 round-robin, 1 contiguous chunks */
    int32_t nms_order;
    int32_t resize_tma;           /* 1: persistent TMA resize on the levels whose source box fits */
    int32_t stream_groups;        /* k > 1: the frames run as k groups on k forked graph branches (1..8) */
    int32_t fast_cell_tiles;      /* FAST form.  1: FAST on whole-cell tiles applies the cell threshold
                                     itself (cells of 8..30 pixels); 2: the same on 120 x 120 cell-aligned
                                     tiles with the general kernel's layout (cells of 15 or 30 pixels);
                                     0: general FAST (fast_tile_h rows), then a threshold pass; 3: general
                                     FAST on 128 x 32 tiles with per-warp pipelines, then the pass; 4: the
                                     same on strips one cell row high, which also set the cell flags, then
                                     the pass applies them (cells of 8..33 pixels).  With nms_tile_h 32 the
                                     NMS kernel applies the cell flags itself: the pass then only sets
                                     flags where FAST does not */
    int32_t nms_tile_h;           /* NMS + Harris tile height: 32 (per-warp kernel on the 128 x 32 detect
                                     tiles), 64 or 128 rows (block kernels) */
    int32_t fast_tile_h;          /* general FAST tile height: 32, 64, 128 or 256 rows */
    int32_t candidates_tried;     /* configurations timed */
    float resize_ms, fast_ms, nms_ms;  /* best measured time of each tuned stage (all levels);
                                          fast_ms covers FAST + NMS (the FAST forms differ in both) */
} of_tuning;

/* One detected keypoint, 64 bytes.  Level-major, rank order within a level
 * (Harris key descending, then y ascending, then x ascending). */
typedef struct of_keypoint {
    float x, y;           /* level-0 coordinates: (x_l, y_l) * scale^l */
    int32_t x_l, y_l;     /* pixel position in its level */
    int32_t level;
    int32_t fast_score;   /* s(p): largest FAST threshold at which p passes */
    float response;       /* Harris score det(M) - k trace(M)^2 times (1/(4*7*255))^4 */
    float angle;          /* atan2(m01, m10), radians in (-pi, pi]; 0 when both are 0 */
    int32_t A, B, C;      /* exact window sums of gx^2, gy^2, gx*gy */
    int32_t m10, m01;     /* exact centroid moments over the disc */
    int32_t reserved;
    int64_t key;          /* exact integer Harris key: den*det(M) - num*trace(M)^2, k = num/den */
} of_keypoint;

/* One input frame for of_detect_batch. */
typedef struct of_frame {
    const uint8_t* img;   /* [device] uint8 image */
    int32_t w, h, pitch;
} of_frame;

/* Create a handle; allocates all device scratch for max_batch frames of
 * max_w x max_h with max_levels levels at min_scale.  Returns NULL on failure
 * (message in of_last_error()). */
of_handle* of_create(const of_params* p);

/* Free the handle and its scratch.  NULL is ignored. */
void of_destroy(of_handle* h);

/* Detect keypoints in one frame.
 *   img [device]          uint8 frame, w x h_px, `pitch` bytes per row (pitch >= w)
 *   levels                pyramid levels, 1..max_levels
 *   scale                 pyramid scale between levels, min_scale <= scale <= 4
 *   fast_t                FAST threshold t of Eq. 1, 1..255
 *   harris_k              Harris k of Eq. 3, 0 <= k <= 0.25, rounded to a multiple of 1e-6
 *                         whose reduced denominator must be <= 3000 (e.g. 0.04 = 1/25)
 *   n_features            keypoints per frame, split over levels by area, 0..max_features
 *   out_kpts [device]     room for n_features records
 * Returns the number of keypoints written (>= 0) or a negative OF_ERR_*.
 * Synchronises the handle's stream to read the count back. */
int of_detect(of_handle* h, const uint8_t* img, int w, int h_px, int pitch, int levels,
              float scale, int fast_t, float harris_k, int n_features, of_keypoint* out_kpts);

/* Detect keypoints in n_frames frames of any sizes in one batched launch
 * sequence (replayed from a cached CUDA graph for a repeated batch shape).
 *   frames [host]         n_frames descriptors, 1 <= n_frames <= max_batch
 *   out_kpts [device]     n_frames * n_features records; frame i starts at i * n_features
 *   out_counts [device]   n_frames int32: keypoints written per frame
 * Other arguments as of_detect.  Asynchronous: returns OF_OK once the work is
 * queued on the handle's stream; results are valid after that stream syncs. */
int of_detect_batch(of_handle* h, const of_frame* frames, int n_frames, int levels,
                    float scale, int fast_t, float harris_k, int n_features,
                    of_keypoint* out_kpts, int32_t* out_counts);

/* Copy an intermediate buffer of the most recent detect call into `dst`, for
 * inspection and parity checks.  what:
 *   OF_BUF_LEVEL  pyramid level image, w x h bytes, packed rows (pitch = w)
 *   OF_BUF_SCORE  candidate score map, w x h bytes: S(p) = s(p) where s(p)
 *                 >= the threshold of p's cell (fast_t, or fast_t_lo in a cell
 *                 with no pixel scoring >= fast_t), else 0; 0 outside the
 *                 detect region -- what NMS keys on
 *   OF_BUF_CELLT  per-cell threshold, ncx x ncy bytes (fast_t or fast_t_lo)
 *   OF_BUF_CAND   NMS survivors, count x 16 bytes {int64 key; int32 x; int32 y},
 *                 in no particular order
 *   OF_BUF_PMASK  (after of_detect_learned only) the tile mask the exact path
 *                 ran on, gx x gy bytes, 1 = tile kept (proposed, a dilated
 *                 neighbour, or every tile of a fallback image)
 *   OF_BUF_LOGIT  (after of_detect_learned only) the network's logit of each
 *                 proposal tile, gx x gy float32
 * dst [device] may be NULL to query the size.  dims [host] receives
 * {w, h, count_or_ncx, ncy}, or {gx, gy, 0, 0} for the two tile buffers
 * (tile (i, j) covers x in [tile_x0 + 32 i, +32), y in [border + 32 j, +32),
 * tile_x0 = border rounded down to a multiple of 16).  Returns the byte
 * size, or a negative OF_ERR_*.  Synchronises the handle's stream. */
#define OF_BUF_LEVEL 0
#define OF_BUF_SCORE 1
#define OF_BUF_CELLT 2
#define OF_BUF_CAND 3
#define OF_BUF_PMASK 4
#define OF_BUF_LOGIT 5
int64_t of_inspect(of_handle* h, int what, int frame, int level, void* dst, int64_t dst_bytes,
                   int32_t* dims);

/* Autotuner (batched path): for this batch shape, time each candidate
 * launch configuration -- pyramid kernel (staged tiles of 32 or 64 rows, or
 * the persistent TMA kernel), persistent grid size and tile order of the FAST
 * and NMS kernels, the FAST tile height (32..256 rows) and NMS tile height
 * (32..128 rows), the FAST form (0..4, see of_tuning), and whether the frames
 * run as one group or as 2..8 groups
 * on forked graph branches -- with CUDA events on these frames (reps
 * timed repetitions each, 1..100), keep the fastest for every later call with
 * the same shape, and run the batch once with it.  Arguments
 * as of_detect_batch; result [host, may be NULL] receives the choice.
 * Synchronises the handle's stream.  The paper has no counterpart: its kernels
 * use fixed launch shapes (Sec. 6). */
int of_autotune(of_handle* h, const of_frame* frames, int n_frames, int levels, float scale,
                int fast_t, float harris_k, int n_features, of_keypoint* out_kpts,
                int32_t* out_counts, int reps, of_tuning* result);

/* Fix the launch configuration of a batch shape (for instance one saved from
 * an earlier of_autotune) instead of searching: the shape's plan is built if
 * needed and its graphs re-captured with *tuning [host].  Fields checked:
 * resize_tile_h 32 or 64, resize_tma 0 or 1, fast/nms_blocks_per_sm in
 * 1..the kernel's occupancy, fast/nms_order 0 or 1, stream_groups 1..8
 * (capped at the number of frames), fast_cell_tiles 0..4 (1 and 2 become 0
 * for cells outside 8..30 pixels, 4 for cells over 33; 2 becomes 1 for cells
 * other than 15 and 30),
 * nms_tile_h 32, 64 or 128, fast_tile_h 32, 64, 128 or 256 (else
 * OF_ERR_ARG); the
 * remaining fields are ignored.  Launches nothing.  Arguments as
 * of_detect_batch.  No paper counterpart. */
int of_set_tuning(of_handle* h, const of_frame* frames, int n_frames, int levels, float scale,
                  int fast_t, float harris_k, int n_features, of_keypoint* out_kpts,
                  int32_t* out_counts, const of_tuning* tuning);

/* Wait for the handle's queued work and report device-side failures: returns
 * OF_ERR_TIMEOUT when a bounded device wait (a tile load that never arrived)
 * expired since the last check -- the affected calls' out_counts entries are
 * then OF_ERR_TIMEOUT too -- else OF_OK.  Clears the condition. */
int of_sync(of_handle* h);

/* Failure-path self test: runs a kernel that waits, with the detector's
 * bounded wait, on a device flag that nothing sets, for limit_us
 * microseconds (1..1e7), then reports through of_sync.  Returns
 * OF_ERR_TIMEOUT when the timeout path works; the handle stays usable. */
int of_test_timeout(of_handle* h, int64_t limit_us);

/* Stage timing: the next detect call on this handle runs its stages as
 * separate launches and records events[i] (cudaEvent_t, created by the
 * caller with timing enabled) on the handle's stream before stage i and
 * events[5] after the last one:
 *   0 pyramid (clear + resize)  1 FAST score  2 cell thresholds (when FAST
 *   did not apply them) + NMS + Harris  3 top-N  4 orientation.
 * Results are identical to an untimed call.  Returns OF_OK or OF_ERR_ARG. */
#define OF_N_STAGES 5
int of_time_stages(of_handle* h, void* const* events);

/* Single-level detection that allocates nothing.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code running inside a CUDA graph capture, real-time loops
 * that must not touch the allocator after start-up, and plug-in hosts that
 * own every device allocation.
 *   img [device]        uint8 frame, w x h, pitch bytes per row (one level, no pyramid)
 *   fast_t, fast_t_lo   threshold and per-30x30-cell fallback (0 = none), as of_create/of_detect
 *   harris_k, n_features as of_detect (n_features <= 8192); border 19, cell 30, radius 15
 *   out_kpts [device]   room for n_features records (rank order)
 *   out_count [device]  one int32: keypoints written
 *   stream              cudaStream_t (NULL = default stream); the call is asynchronous
 * Intermediate buffers live in one static device array of
 * OF_NOALLOC_SCRATCH_BYTES inside the library, held by every GPU that loads
 * it until the process exits.  A frame whose buffers do not fit returns
 * OF_ERR_TOO_LARGE (a 1920x1080 frame fits).  The first call on each device
 * looks the array's address up with cudaGetSymbolAddress, with that device
 * current; make that first call before any stream capture.  The address is
 * kept for the life of the process, so a device reset (cudaDeviceReset or
 * any teardown of the primary context) is not supported afterwards.  Calls
 * share the array: each call clears what must start at zero, and calls whose
 * work overlaps on the GPU race -- serialise them.  Returns OF_OK or OF_ERR_*. */
#define OF_NOALLOC_SCRATCH_BYTES (16u << 20)
int of_detect_level_noalloc(const uint8_t* img, int w, int h, int pitch, int fast_t,
                            int fast_t_lo, float harris_k, int n_features,
                            of_keypoint* out_kpts, int32_t* out_count, void* stream);

/* Host-only: scratch bytes a batch of n_frames frames (sizes ws[i] x hs[i])
 * needs on a handle created with *p (border and cell taken from p, zero
 * fields defaulted as in of_create), counting unaligned level-0 copies.
 * Returns the byte count or OF_ERR_ARG. */
int64_t of_batch_bytes(const of_params* p, const int32_t* ws, const int32_t* hs, int n_frames,
                       int levels, float scale, int n_features);

/* ------------------------------------------------------------------------
 * Serving loop with continuous batching.  The paper measures single images
 * and videos (Sec. 6, Fig. 14); this loop serves streams of mixed-resolution
 * frames from many clients.
 *
 * The server owns `slots` engines, each a handle with its own stream and a
 * 1/slots share of memory_budget (scratch arena, device input frames,
 * outputs).  of_server_submit copies a host frame into the queue and returns
 * at once.  A dispatcher thread admits queued requests into any free slot --
 * the oldest request and later ones of the same resolution, in arrival
 * order, while the batch fits the slot's scratch and input bytes and
 * max_batch -- and launches the batch asynchronously; batches on different
 * slots overlap on the device, and requests that arrive meanwhile are
 * admitted as soon as a slot and its memory free up.  Each batch's pyramids
 * stay resident in its slot until the slot takes its next batch.  Results are
 * identical to of_detect on each frame alone.  All entry points are
 * thread-safe. */
typedef struct of_server of_server;

typedef struct of_server_params {
    int32_t max_w, max_h;   /* largest frame (required) */
    int32_t levels;         /* default 8 */
    float scale;            /* default 1.2 */
    int32_t fast_t;         /* default 20 */
    int32_t fast_t_lo;      /* per-cell fallback threshold, 0 = none */
    float harris_k;         /* default 0.04 */
    int32_t n_features;     /* per frame, default 1000 */
    int32_t slots;          /* concurrent batches, default 3 (1..16) */
    int32_t max_batch;      /* frames per batch, default 8 */
    int64_t memory_budget;  /* device bytes for all slots (required) */
    int32_t border, cell, orient_radius;  /* 0 = defaults of of_create */
} of_server_params;

typedef struct of_server_result {
    int64_t id, tag;        /* id from of_server_submit, caller's tag */
    int32_t w, h;
    int32_t count;          /* keypoints written (>= 0) or a negative OF_ERR_* */
    int32_t batch_frames;   /* frames in the batch that carried this request */
    double t_submit, t_launch, t_done;  /* steady-clock seconds */
} of_server_result;

typedef struct of_server_stats {
    int64_t submitted, completed, queued, batches, frames_launched, in_flight_batches;
    int64_t slot_arena_bytes, slot_input_bytes;
} of_server_stats;

/* NULL on failure (e.g. OF_ERR_TOO_LARGE when a max-size frame does not fit one slot's share). */
of_server* of_server_create(const of_server_params* p);
/* Stops the dispatcher after the batches in flight; queued requests are dropped. */
void of_server_destroy(of_server* s);
/* img [host] w x h, pitch bytes per row; copied before return.  Returns the request id (>= 0). */
int64_t of_server_submit(of_server* s, const uint8_t* img, int w, int h, int pitch, int64_t tag);
/* Moves up to max_results finished requests into results [host]; their keypoints go to
 * kpts [host, may be NULL] + i * n_features.  Waits up to wait_ms for the first.  Returns the number moved. */
int of_server_poll(of_server* s, of_server_result* results, of_keypoint* kpts, int max_results,
                   int wait_ms);
int of_server_stats_get(of_server* s, of_server_stats* out);

/* ------------------------------------------------------------------------
 * Learned tile proposal.  The paper has no counterpart; this is a learned
 * front end to its exact detector.  A tiny network scores every 32 x 32 tile
 * of every pyramid level (on the detect-tile grid) from the tile and a
 * 16-pixel halo: 3 x 3 convolutions with stride 2 and ReLU, 1 -> 8 -> 16 ->
 * 16 channels, global average pool, linear -> 1 logit; bf16 weights, fp32
 * accumulation; trained with the library's own forward / backward / Adam
 * kernels.  The exact path then runs only on proposed tiles. */
typedef struct of_tcnn of_tcnn;

/* He-uniform initialisation from `seed`, zero biases, Adam state cleared. */
of_tcnn* of_tcnn_create(uint64_t seed);
void of_tcnn_destroy(of_tcnn* net);
int of_tcnn_num_params(void);
/* Flat fp32 parameters [host, of_tcnn_num_params()]: conv1 w[8][1][3][3], b[8],
 * conv2 w[16][8][3][3], b[16], conv3 w[16][16][3][3], b[16], head w[16], b.
 * set: master copy (bf16 compute copy rounded from it; Adam state cleared).
 * get which: 0 master, 1 the bf16 compute copy, 2 the last gradient. */
int of_tcnn_set_params(of_tcnn* net, const float* host);
int of_tcnn_get_params(of_tcnn* net, int which, float* host);
/* tiles [device]: n x 64 x 64 uint8 patches; logits [device]: n floats. */
int of_tcnn_forward(of_tcnn* net, const uint8_t* tiles, int n, float* logits, void* stream);
/* One training step's gradient: weighted BCE with logits over n patches
 * (labels [device] 0/1 floats, positives weighted by pos_weight), mean over n;
 * gradients of the bf16 weights replace the previous ones.  loss_out [host,
 * may be NULL] receives the loss (synchronises the stream). */
int of_tcnn_loss_grad(of_tcnn* net, const uint8_t* tiles, const float* labels, int n, float pos_weight,
                      float* loss_out, void* stream);
/* Adam (bias-corrected, decoupled weight decay) on the master weights. */
int of_tcnn_adam(of_tcnn* net, float lr, float beta1, float beta2, float eps, float weight_decay,
                 void* stream);
/* Checkpoint: "OFTC", version 1, parameter count, step, master weights, Adam
 * moments, CRC-32.  save with buf NULL returns the size; load verifies all. */
int64_t of_tcnn_save(of_tcnn* net, uint8_t* buf, int64_t cap);
int of_tcnn_load(of_tcnn* net, const uint8_t* buf, int64_t n);

/* Detect with tile proposal: the pyramid, then the network on every
 * proposal tile, then FAST / NMS / Harris / top-N / orientation restricted
 * to proposed tiles (scores are 0 outside them).  A tile is proposed when
 * sigmoid(logit) >= threshold, or when a neighbour is and dilate = 1.  An
 * image (frame, level) whose confidence -- mean |2 sigmoid(logit) - 1| over
 * its tiles -- is below min_confidence runs on all its tiles (full-frame
 * fallback).  threshold <= 0 proposes everything (identical to
 * of_detect_batch).  stats [host, may be NULL] receives {tiles, proposed
 * tiles, fallback images} and synchronises.  Other arguments as
 * of_detect_batch. */
int of_detect_learned(of_handle* h, const of_frame* frames, int n_frames, int levels, float scale,
                      int fast_t, float harris_k, int n_features, of_tcnn* net, float threshold,
                      float min_confidence, int dilate, of_keypoint* out_kpts, int32_t* out_counts,
                      int32_t* stats);

/* Copy the 64 x 64 input patches of every proposal tile of (frame, level) of
 * the last detect call into dst [device, may be NULL to query], tile-major in
 * row order of the proposal grid.  grid [host, 2 ints] receives its columns
 * and rows.  Returns the number of tiles, or a negative OF_ERR_*. */
int of_extract_tiles(of_handle* h, int frame, int level, uint8_t* dst, int64_t cap_tiles,
                     int32_t* grid);

/* ---- The paper's ablation variants (Table 2, Sec. 6.2) ------------------
 * For measuring whether the paper's ordering of its FAST and Harris variants
 * holds on GB300; not the detector's path.  One level, FAST points at
 * threshold fast_t (Eq. 1) in the region border <= x < w - border (same for
 * y), border >= 4, and for a Harris variant the exact Sobel sums over the
 * 7 x 7 window (Eqs. 2-4) and key = kden (AB - C^2) - knum (A+B)^2 with
 * harris_k = knum / kden as of_detect.  No NMS, no ranking.
 *   fast_variant    OF_VAR_FAST_*: baseline (branchy run-length test, global
 *                   loads), binary (Alg. 2 bit windows, global), sm, sm_binary
 *                   (the same on a shared-memory tile)
 *   harris_variant  OF_VAR_HARRIS_*: none, baseline (2-D Sobel, second launch,
 *                   global loads; any FAST variant), sep, para_sep, semi_sep
 *                   (fused after sm_binary FAST in one kernel, as the paper
 *                   pairs them; fast_variant must be OF_VAR_FAST_SM_BINARY)
 *   img [device]    uint8 image, w x h, pitch bytes per row
 *   out_points [device] room for capacity records, in no particular order;
 *                   points past capacity are counted but not written
 *   out_count [device]  one int32, set to the number of points
 *   stream          cudaStream_t (NULL = default stream); asynchronous
 * Returns OF_OK or OF_ERR_ARG.  Allocates nothing. */
typedef struct of_var_point {
    int32_t x, y;
    int32_t A, B, C;      /* exact window sums (0 without a Harris variant) */
    int32_t reserved;
    int64_t key;          /* exact Harris key (0 without a Harris variant) */
} of_var_point;
#define OF_VAR_FAST_BASELINE 0
#define OF_VAR_FAST_BINARY 1
#define OF_VAR_FAST_SM 2
#define OF_VAR_FAST_SM_BINARY 3
#define OF_VAR_HARRIS_NONE (-1)
#define OF_VAR_HARRIS_BASELINE 0
#define OF_VAR_HARRIS_SEP 1
#define OF_VAR_HARRIS_PARA_SEP 2
#define OF_VAR_HARRIS_SEMI_SEP 3
int of_variant_detect(int fast_variant, int harris_variant, const uint8_t* img, int w, int h, int pitch,
                      int fast_t, int border, float harris_k, of_var_point* out_points, int32_t* out_count,
                      int64_t capacity, void* stream);

/* Host-only: the pyramid plan the detector uses for a W x H frame (no GPU
 * needed).  ws, hs [host, levels ints] receive level sizes; quota [host,
 * levels ints] receives the per-level feature quota for n_features.
 * Returns OF_OK or OF_ERR_ARG. */
int of_plan_levels(int W, int H, int levels, float scale, int n_features, int32_t* ws,
                   int32_t* hs, int32_t* quota);

/* Bandwidth probe for reporting kernels against a measured peak; the paper
 * has no counterpart and the detector does not use it.  Reads `bytes` of
 * buf [device, 16-byte aligned] `reps` times with 16-byte loads that are
 * cached in L2 only, from 8 blocks of 256 threads per SM; writes a value
 * folded from the data into *sink [device, one uint32] only in a case that
 * practically never occurs (it keeps the loads).  A buffer that fits in L2
 * measures the L2 read bandwidth (bytes * reps / elapsed time on `stream`,
 * timed by the caller), one much larger than L2 the HBM read bandwidth.
 * Asynchronous.  Returns OF_OK, OF_ERR_ARG or OF_ERR_CUDA.  Allocates nothing. */
int of_probe_read(const void* buf, int64_t bytes, int reps, uint32_t* sink, void* stream);

/* Message for the last error on this host thread ("" if none). */
const char* of_last_error(void);

/* OF_VERSION of the loaded library. */
int of_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OFAST_H */
