// Runtime behind the C ABI of include/ofast.h: handle and scratch arena,
// batch plans (level sizes, tiling, resize tables, arena layout), one CUDA
// graph per plan, pointer rebinding between calls, inspection and errors.
//
// A plan is built once per batch shape (frame sizes and pitches, levels,
// scale, thresholds, k, n_features).  Its kernels read every pointer from a
// small device-side descriptor block, so a replay with new frame or output
// pointers only re-uploads that block (from pinned staging memory) before
// launching the same graph.  The arena is allocated once by of_create for the
// largest batch the handle accepts; detect calls never allocate device memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "of_internal.h"
#include "of_plan.h"
#include "ofast.h"

namespace ofk {
void set_select_smem_limit(int bytes);
int fast_blocks_per_sm();
int nms_blocks_per_sm();
void launch_wait_test(const int32_t* flag, int32_t* status, uint64_t limit_ns, void* stream);
int launch_propose(const Img* imgs, const int32_t* list, const int32_t* prefix, int n_list, const float* logits,
                   uint8_t* pos, uint8_t* mask, float threshold, float min_conf, int dilate, int32_t* stats,
                   void* stream);
int launch_extract(const Img* imgs, int img, int border, uint8_t* dst, int n, void* stream);
int tcnn_forward_tiles(of_tcnn* N, const Img* imgs, const int32_t* list, const int32_t* prefix, int n_list,
                       int n_tiles, int border, float* logits, void* stream);
}

using namespace ofk;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define OF_CK(call)                                                                   \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fail(OF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mutex;

// The CUDA driver API's tensor-map encoder, looked up through the runtime (no libcuda link).
int resolve_encoder() {
    std::lock_guard<std::mutex> lock(g_encode_mutex);
    if (g_encode) return OF_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(OF_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return OF_OK;
}

// 2-D uint8 tensor map over a w x h image with `pitch` bytes per row and a
// box of box_w x box_h bytes; reads outside the image return 0.
int encode_u8(CUtensorMap* m, const void* base, int w, int h, int pitch, int box_w, int box_h) {
    std::memset(m, 0, sizeof(*m));
    if (!base || w < 1 || h < 1) return OF_OK;  // unused map
    const cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides,
                                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(OF_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return OF_OK;
}

struct FrameKey {
    int w, h, pitch;
    bool copy;  // level 0 is copied into the arena (unaligned input)
    bool operator==(const FrameKey& o) const {
        return w == o.w && h == o.h && pitch == o.pitch && copy == o.copy;
    }
};

struct Settings {
    int levels;
    float scale;
    int t_hi, t_lo;
    int64_t knum, kden;
    int n_features;
    int border, cell, radius;
};

// Arena layout of one batch.
struct ImgLayout {
    int w = 0, h = 0;
    int pitch = 0, spitch = 0;
    int ncx = 0, ncy = 0, cap = 0, quota = 0;
    int tiles_x = 0, tiles_y = 0, tile_x0 = 0;
    bool det = false;  // detect region not empty
    size_t lev = 0, score = 0, cell = 0, ckey = 0, cyx = 0, kkey = 0, kyx = 0, ctr = 0;
    double lscale = 1.0;
};

struct Layout {
    std::vector<ImgLayout> img;  // frame-major, level-minor
    size_t zero_end = 0;         // [0, zero_end) is cleared before every call
    size_t total = 0;
};

constexpr size_t kAlign = 256;
constexpr int kStages = 5;
constexpr int kMaxGroups = 8;  // frame groups of a forked batched graph

// Lay out one batch.  `quota_each` overrides the per-level quotas (capacity sizing).
Layout make_layout(const std::vector<FrameKey>& frames, const Settings& s, int quota_each) {
    Layout L;
    const int nl = s.levels;
    L.img.resize(frames.size() * nl);
    std::vector<int32_t> ws(nl), hs(nl), q(nl);
    std::vector<double> ls(nl);
    ofh::level_quotas(s.n_features, nl, s.scale, q.data());
    // Pass 1: geometry.
    for (size_t f = 0; f < frames.size(); ++f) {
        ofh::level_sizes(frames[f].w, frames[f].h, nl, s.scale, ws.data(), hs.data(), ls.data());
        bool alive = true;
        for (int l = 0; l < nl; ++l) {
            ImgLayout& I = L.img[f * nl + l];
            if (ws[l] < 1 || hs[l] < 1) alive = false;
            I.quota = quota_each >= 0 ? quota_each : q[l];
            I.lscale = ls[l];
            if (!alive) continue;
            I.w = ws[l];
            I.h = hs[l];
            I.pitch = (l == 0 && !frames[f].copy) ? frames[f].pitch : (int)align_up(I.w, 16);
            const int rw = I.w - 2 * s.border, rh = I.h - 2 * s.border;
            if (rw > 0 && rh > 0) {
                I.det = true;
                I.spitch = (int)align_up(I.w, 16);
                I.ncx = (rw + s.cell - 1) / s.cell;
                I.ncy = (rh + s.cell - 1) / s.cell;
                I.cap = ((rw + 1) / 2) * ((rh + 1) / 2);
                I.tile_x0 = s.border & ~15;
                I.tiles_x = (I.w - s.border - I.tile_x0 + TILE_W - 1) / TILE_W;
                I.tiles_y = (rh + TILE_H - 1) / TILE_H;
            }
        }
    }
    // Pass 2: offsets.  Cleared region first: counters, then cell flags.
    size_t off = 0;
    for (auto& I : L.img) {
        I.ctr = off;
        off += 4 * sizeof(int32_t);
    }
    off = align_up(off, kAlign);
    for (auto& I : L.img) {
        if (!I.det) continue;
        I.cell = off;
        off = align_up(off + sizeof(uint32_t) * I.ncx * I.ncy, 16);
    }
    off = align_up(off, kAlign);
    L.zero_end = off;
    for (size_t f = 0; f < frames.size(); ++f) {
        for (int l = 0; l < nl; ++l) {
            ImgLayout& I = L.img[f * nl + l];
            if (I.w == 0) continue;
            if (l > 0 || frames[f].copy) {
                I.lev = off;
                off = align_up(off + (size_t)I.pitch * I.h, kAlign);
            }
        }
    }
    for (auto& I : L.img) {
        if (!I.det) continue;
        I.score = off;
        off = align_up(off + (size_t)I.spitch * I.h, kAlign);
        I.ckey = off;
        off = align_up(off + sizeof(uint64_t) * I.cap, kAlign);
        I.cyx = off;
        off = align_up(off + sizeof(uint32_t) * I.cap, kAlign);
        I.kkey = off;
        off = align_up(off + sizeof(uint64_t) * std::max(I.quota, 1), kAlign);
        I.kyx = off;
        off = align_up(off + sizeof(uint32_t) * std::max(I.quota, 1), kAlign);
    }
    L.total = off;
    return L;
}

struct Plan {
    std::vector<FrameKey> frames;
    Settings s{};
    Layout lay;
    std::vector<Img> h_img;
    std::vector<Resize> h_rs;
    std::vector<int> rs_begin;      // jobs of level l: [rs_begin[l], rs_begin[l+1])
    std::vector<int32_t> det_list, det_prefix, tables;
    std::vector<float> ftables;  // level-0 coordinates per (level size, scale^level), float
    std::vector<int> rs_frame;      // frame of each resize job
    // Launch ranges of one group of frames: groups[k] splits the batch into k
    // groups (k = 1: everything; k > 1: the forked graph's branches).  Tile
    // prefixes of a group are rebased to 0 and stored in gp_det / gp_rs.
    struct Group {
        int img_begin = 0, n_img = 0;
        int dl_begin = 0, n_list = 0, det_tiles = 0, dp_off = 0;
        int fast_tiles = 0, fp_off = 0;             // cell-tile FAST: tiles and prefix offset in gp_fast
        int cs_strips = 0, cs_off = 0;              // cell-strip FAST: strips and prefix offset in gp_cstrip
        int csi_off = 0, dti_off = 0;               // item tables: cell strips, 128 x 32 detect tiles
        int nms64_tiles = 0, np_off = 0;            // NMS with 64-row tiles: tiles and prefix offset in gp_nms64
        int ftall_tiles[2] = {0, 0}, ftall_off[2] = {0, 0};  // FAST on FT_HS[i]-row tiles: tiles, offset in gp_ftall[i]
        int fal_tiles = 0, fal_off = 0;             // cell-aligned FAST: tiles and prefix offset in gp_fal
        int n_bands = 0, rp_off = 0;                // threshold pass: cell rows and prefix offset in gp_rows
        int slot_begin = 0, slot_end = 0;
        std::vector<int> rs_job, rs_n;              // per level: first resize job, jobs
        std::vector<int> rsp_off[2], rs_tiles[2];   // per level and resize tile height
        std::vector<int> rsi_off;                   // per level: offset of its 64-row tiles in items_rs
    };
    std::vector<Group> groups[kMaxGroups + 1];
    std::vector<int32_t> gp_det, gp_rs, gp_fast, gp_rows, gp_nms64, gp_ftall[2], gp_fal, gp_cstrip;
    // Work-item tables of the per-warp kernels, per group: (image, (y0 << 16) | x0).
    std::vector<uint2> items_cs, items_dt;
    std::vector<uint16_t> slot_img;  // image of every output slot (orientation kernel)
    std::vector<uint2> items_rs;  // TMA resize tiles per group and level: (job in the level's launch, (Y0 << 16) | X0)
    bool cell_tiles = false;     // the cell size allows the cell-tile FAST kernel
    bool apply_flags = false;    // the threshold pass can set the cell flags (else the general FAST kernel does)
    bool strip_ok = false;       // the cell size allows the cell-row strip kernel (cells of 8..33 pixels)
    bool aligned_ok = false;     // ... and the cell-aligned general FAST kernel (cells of 15 or 30 pixels)
    std::vector<int> rt_buf;        // TMA resize buffer bytes of level l (0: staged kernel only)
    std::vector<int> rt_bps;        // TMA resize resident blocks per SM of level l
    int det_tiles = 0, max_quota = 0, total_slots = 0, n_img = 0;
    Call h_call{};
    uint8_t* dbuf = nullptr;
    size_t off_call = 0, off_img = 0, off_rs = 0, off_dl = 0, off_tab = 0, off_ftab = 0;
    size_t off_gdp = 0, off_grs = 0, off_gfp = 0, off_grp = 0, off_gnp = 0, off_gft[2] = {0, 0}, off_gfal = 0,
           off_gcs = 0, off_ics = 0, off_idt = 0, off_irs = 0, off_sli = 0;
    size_t off_maps = 0;
    std::vector<CUtensorMap> h_maps;  // [image maps | score maps] (n_img each) | resize source maps
    of_tuning tun{};  // launch configuration (defaults, or the autotuner's choice)
    bool tuned = false;
    // Learned path: proposal tiles per listed image, device buffers
    // [mask | pos | logits | prefix | stats], allocated on first use.
    std::vector<int32_t> ptile_prefix;  // det_list.size() + 1 entries
    uint8_t* lbuf = nullptr;
    size_t off_mask = 0, off_pos = 0, off_logit = 0, off_pp = 0, off_stats = 0;
    bool pmask_on = false;
    size_t header_bytes = 0;
    uint8_t* stage[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int stage_i = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t stage_exec[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<const uint8_t*> bound_src;
    of_keypoint* bound_out = nullptr;
    int32_t* bound_counts = nullptr;
    bool bound = false;
    uint64_t stamp = 0;

    Img* d_img() const { return reinterpret_cast<Img*>(dbuf + off_img); }
    Resize* d_rs() const { return reinterpret_cast<Resize*>(dbuf + off_rs); }
    Call* d_call() const { return reinterpret_cast<Call*>(dbuf + off_call); }
    const CUtensorMap* d_maps() const { return reinterpret_cast<const CUtensorMap*>(dbuf + off_maps); }
    const int32_t* d_dl() const { return reinterpret_cast<const int32_t*>(dbuf + off_dl); }
    const int32_t* d_gdp() const { return reinterpret_cast<const int32_t*>(dbuf + off_gdp); }
    const int32_t* d_grs() const { return reinterpret_cast<const int32_t*>(dbuf + off_grs); }
    const int32_t* d_gfp() const { return reinterpret_cast<const int32_t*>(dbuf + off_gfp); }
    const int32_t* d_grp() const { return reinterpret_cast<const int32_t*>(dbuf + off_grp); }
    const int32_t* d_gcs() const { return reinterpret_cast<const int32_t*>(dbuf + off_gcs); }
    const uint2* d_ics() const { return reinterpret_cast<const uint2*>(dbuf + off_ics); }
    const uint2* d_idt() const { return reinterpret_cast<const uint2*>(dbuf + off_idt); }
    const uint2* d_irs() const { return reinterpret_cast<const uint2*>(dbuf + off_irs); }
    const uint16_t* d_sli() const { return reinterpret_cast<const uint16_t*>(dbuf + off_sli); }
    const int32_t* d_gnp() const { return reinterpret_cast<const int32_t*>(dbuf + off_gnp); }
    const int32_t* d_gft(int i) const { return reinterpret_cast<const int32_t*>(dbuf + off_gft[i]); }
    const int32_t* d_gfal() const { return reinterpret_cast<const int32_t*>(dbuf + off_gfal); }
};

// Resident blocks per SM of the plan's FAST kernel.
// How the per-cell thresholds reach NMS.  The cell-tile forms (1, 2) write
// final scores themselves.  Otherwise the threshold pass applies the cell
// flags to the maps; it also sets them, unless the FAST kernel did: the
// cell-row strips (form 4) always, the general block kernel when the pass
// cannot flag a band's cells (more than CA_MAX_CELLS cells per row).
bool cell_form(const Plan* P) {
    const int f = P->tun.fast_cell_tiles;
    return P->cell_tiles && (f == 1 || f == 2);
}
bool strip_form(const Plan* P) { return P->strip_ok && P->tun.fast_cell_tiles == 4; }
bool warp_form(const Plan* P) { return P->tun.fast_cell_tiles == 3 && P->apply_flags; }
bool fast_sets_flags(const Plan* P) { return strip_form(P) || (!cell_form(P) && !P->apply_flags); }
// The per-warp NMS kernel (32-row tiles) applies the flags to its staged
// score words itself; the pass then only sets flags where FAST did not (for
// images with proposal tiles at least: FAST skips their flags).
bool nms_applies(const Plan* P) {
    return P->tun.nms_tile_h == 32 && !cell_form(P) && P->s.t_hi != P->s.t_lo;
}

int plan_fast_bps(const Plan* P) {
    if (P->aligned_ok && P->tun.fast_cell_tiles == 2) return fast_aligned_blocks_per_sm();
    if (cell_form(P)) return fast_cells_blocks_per_sm(P->s.cell);
    if (strip_form(P)) return fast_cstrip_blocks_per_sm();
    if (warp_form(P)) return fast_warp_blocks_per_sm();
    return fast_blocks_per_sm(P->tun.fast_tile_h, fast_sets_flags(P));
}

void free_plan(Plan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    for (auto& x : p->stage_exec)
        if (x) cudaGraphExecDestroy(x);
    for (int i = 0; i < 2; ++i) {
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
        if (p->stage[i]) cudaFreeHost(p->stage[i]);
    }
    if (p->dbuf) cudaFree(p->dbuf);
    if (p->lbuf) cudaFree(p->lbuf);
    delete p;
}

}  // namespace

struct of_handle {
    of_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_branch[kMaxGroups - 1] = {};  // further branches of a forked capture
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kMaxGroups - 1] = {};
    uint8_t* arena = nullptr;
    size_t arena_bytes = 0;
    int32_t* d_counts = nullptr;  // [0] of_detect's count, [4] device status word
    int n_sms = 0;
    int32_t* h_count = nullptr;   // pinned
    std::vector<Plan*> plans;
    Plan* last = nullptr;
    uint64_t clock = 0;
    cudaEvent_t stage_ev[6] = {};  // when set: recorded around each stage of the next call
    bool stage_timing = false;
};

namespace {

constexpr int kMaxPlans = 64;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Enqueue stage `stage` of one frame group of a plan on `st` (stage 0 here is
// the resize chain only; the clearing memset is enqueued once per call):
//   0 resize levels 1..L-1 (pyramid)   1 FAST score + cell flags
//   2 (threshold pass,) NMS + Harris keys
//   3 top-N per level                  4 orientation + output records
void enqueue_group_stage(of_handle* H, Plan* P, const Plan::Group& G, int stage, cudaStream_t st) {
    const Settings& s = P->s;
    const int nl = s.levels;
    switch (stage) {
        case 0:
            for (int l = 1; l < nl; ++l) {
                const int nj = G.rs_n[l];
                if (nj <= 0) continue;
                if (P->tun.resize_tma && P->rt_buf[l] > 0) {
                    static_assert(RS_TILE_HS[1] == RT_TILE_H, "TMA resize uses the 64-row tile prefix");
                    launch_resize_tma(P->d_rs() + G.rs_job[l], P->d_irs() + G.rsi_off[l], G.rs_tiles[1][l],
                                      P->d_maps() + 2 * P->n_img + G.rs_job[l], P->d_call(), P->rt_buf[l],
                                      H->n_sms * P->rt_bps[l], st);
                } else {
                    const int v = P->tun.resize_tile_h == RS_TILE_HS[0] ? 0 : 1;
                    launch_resize(P->d_rs() + G.rs_job[l], P->d_grs() + G.rsp_off[v][l], nj, G.rs_tiles[v][l],
                                  RS_TILE_HS[v], st);
                }
            }
            break;
        case 1:
            // The cell-tile kernel writes final candidate scores S(p); the
            // general kernel's maps get the threshold pass at the start of stage 2.
            if (P->aligned_ok && P->tun.fast_cell_tiles == 2)
                launch_fast_aligned(P->d_img(), P->d_dl() + G.dl_begin, P->d_gfal() + G.fal_off, G.n_list,
                                    G.fal_tiles, P->d_maps(), P->d_call(), s.t_hi, s.t_lo, s.border, s.cell,
                                    H->n_sms * P->tun.fast_blocks_per_sm, P->tun.fast_order, st);
            else if (strip_form(P))
                launch_fast_cstrip(P->d_img(), P->d_ics() + G.csi_off, G.cs_strips, P->d_maps(), P->d_call(), s.t_hi,
                                   s.t_lo, s.border, s.cell, H->n_sms * P->tun.fast_blocks_per_sm, P->tun.fast_order, st);
            else if (cell_form(P))
                launch_fast_cells(P->d_img(), P->d_dl() + G.dl_begin, P->d_gfp() + G.fp_off, G.n_list, G.fast_tiles,
                                  P->d_maps(), P->d_call(), s.t_hi, s.t_lo, s.border, s.cell,
                                  H->n_sms * P->tun.fast_blocks_per_sm, P->tun.fast_order, st);
            else if (warp_form(P))
                launch_fast_warp(P->d_img(), P->d_dl() + G.dl_begin, P->d_gdp() + G.dp_off, G.n_list, G.det_tiles,
                                 P->d_maps(), P->d_call(), s.t_lo, s.border, H->n_sms * P->tun.fast_blocks_per_sm,
                                 P->tun.fast_order, st);
            else if (P->tun.fast_tile_h == 64)
                launch_fast(P->d_img(), P->d_dl() + G.dl_begin, P->d_gnp() + G.np_off, G.n_list, G.nms64_tiles,
                            P->d_maps(), P->d_call(), s.t_hi, s.t_lo, s.border, s.cell,
                            H->n_sms * P->tun.fast_blocks_per_sm, P->tun.fast_order, st, fast_sets_flags(P), 64);
            else if (P->tun.fast_tile_h == FT_HS[0] || P->tun.fast_tile_h == FT_HS[1]) {
                const int i = P->tun.fast_tile_h == FT_HS[0] ? 0 : 1;
                launch_fast(P->d_img(), P->d_dl() + G.dl_begin, P->d_gft(i) + G.ftall_off[i], G.n_list,
                            G.ftall_tiles[i], P->d_maps(), P->d_call(), s.t_hi, s.t_lo, s.border, s.cell,
                            H->n_sms * P->tun.fast_blocks_per_sm, P->tun.fast_order, st, fast_sets_flags(P),
                            FT_HS[i]);
            }
            else
                launch_fast(P->d_img(), P->d_dl() + G.dl_begin, P->d_gdp() + G.dp_off, G.n_list, G.det_tiles,
                            P->d_maps(), P->d_call(), s.t_hi, s.t_lo, s.border, s.cell,
                            H->n_sms * P->tun.fast_blocks_per_sm, P->tun.fast_order, st, fast_sets_flags(P), 32);
            break;
        case 2: {
            if (!cell_form(P)) {
                const int flags = strip_form(P) ? 2 : fast_sets_flags(P) ? 0 : 1;
                const bool apply = !nms_applies(P);
                // Flags of images with proposal tiles only (flags 2, no apply): the
                // learned path launches that pass itself (learned_flag_pass).
                if (apply || flags == 1)
                    launch_cell_apply(P->d_img(), P->d_dl() + G.dl_begin, P->d_grp() + G.rp_off, G.n_list,
                                      G.n_bands, s.t_hi, s.t_lo, s.border, s.cell, H->n_sms * 8, st, flags, apply);
            }
            const bool fin = true;
            if (P->tun.nms_tile_h == 32)
                launch_nms_warp(P->d_img(), P->d_idt() + G.dti_off, G.det_tiles, P->d_maps(), P->d_maps() + P->n_img,
                                P->d_call(), s.t_hi, s.t_lo, s.border, s.cell, H->n_sms * P->tun.nms_blocks_per_sm,
                                P->tun.nms_order, st, nms_applies(P));
            else if (P->tun.nms_tile_h == 64)
                launch_nms_harris(P->d_img(), P->d_dl() + G.dl_begin, P->d_gnp() + G.np_off, G.n_list,
                                  G.nms64_tiles, P->d_maps(), P->d_maps() + P->n_img, P->d_call(), s.t_hi, s.t_lo,
                                  s.border, s.cell, H->n_sms * P->tun.nms_blocks_per_sm, P->tun.nms_order, st, fin,
                                  64);
            else  // 128 rows: the tiling of the 128-row FAST tiles
                launch_nms_harris(P->d_img(), P->d_dl() + G.dl_begin, P->d_gft(0) + G.ftall_off[0], G.n_list,
                                  G.ftall_tiles[0], P->d_maps(), P->d_maps() + P->n_img, P->d_call(), s.t_hi,
                                  s.t_lo, s.border, s.cell, H->n_sms * P->tun.nms_blocks_per_sm, P->tun.nms_order, st,
                                  fin, FT_HS[0]);
            break;
        }
        case 3:
            launch_select(P->d_img() + G.img_begin, G.n_img, P->d_call(), P->max_quota, st);
            break;
        case 4:
            launch_orient_range(P->d_img(), G.img_begin, G.n_img, G.slot_begin, G.slot_end, P->d_call(), st,
                                P->n_img <= 65536 ? P->d_sli() : nullptr);
            break;
    }
}

// Enqueue stages [first, last) of a plan on `st`, one launch per stage over
// the whole batch:
//   0 clear counters and cell flags, resize levels 1..L-1 (pyramid)
//   1 FAST score + cell flags      2 NMS + Harris keys
//   3 top-N per level              4 orientation + output records
// Learned path, between FAST and NMS: the cell flags of the images with
// proposal tiles, which the cell-row strip kernel leaves to the threshold
// pass, when the stage-2 graphs run no pass (the per-warp NMS kernel applies
// the thresholds itself).
void learned_flag_pass(of_handle* H, Plan* P, cudaStream_t st) {
    if (cell_form(P) || !strip_form(P) || !nms_applies(P)) return;
    const Plan::Group& G = P->groups[1][0];
    const Settings& s = P->s;
    launch_cell_apply(P->d_img(), P->d_dl() + G.dl_begin, P->d_grp() + G.rp_off, G.n_list, G.n_bands, s.t_hi, s.t_lo,
                      s.border, s.cell, H->n_sms * 8, st, 2, false);
}

void enqueue_stages(of_handle* H, Plan* P, int first, int last, cudaStream_t st) {
    for (int stage = first; stage < last; ++stage) {
        if (stage == 0) cudaMemsetAsync(H->arena, 0, P->lay.zero_end, st);
        enqueue_group_stage(H, P, P->groups[1][0], stage, st);
    }
}

// The whole call with the frames split into k groups whose stage chains run
// on k branches (cs and the handle's further capture streams), forked after
// the clearing memset and joined at the end: one group's latency-bound
// stages overlap another's ALU-bound ones.  Only inside a stream capture.
void enqueue_forked(of_handle* H, Plan* P, int k, cudaStream_t cs) {
    cudaMemsetAsync(H->arena, 0, P->lay.zero_end, cs);
    cudaEventRecord(H->fork_ev, cs);
    for (int g = 1; g < k; ++g) cudaStreamWaitEvent(H->cap_branch[g - 1], H->fork_ev, 0);
    const std::vector<Plan::Group>& gs = P->groups[k];
    for (int stage = 0; stage < kStages; ++stage)
        for (int g = 0; g < k; ++g) enqueue_group_stage(H, P, gs[g], stage, g == 0 ? cs : H->cap_branch[g - 1]);
    for (int g = 1; g < k; ++g) {
        cudaEventRecord(H->join_ev[g - 1], H->cap_branch[g - 1]);
        cudaStreamWaitEvent(cs, H->join_ev[g - 1], 0);
    }
}

cudaError_t capture(of_handle* H, Plan* P, int first, int last, cudaGraph_t* g, int forked = 1) {
    cudaStream_t cs = H->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    if (forked > 1) enqueue_forked(H, P, forked, cs);
    else enqueue_stages(H, P, first, last, cs);
    const cudaError_t le = cudaGetLastError();
    e = cudaStreamEndCapture(cs, g);
    return e != cudaSuccess ? e : le;
}

// Capture the launch sequence once as one graph (forked into two frame
// groups when the tuning says so), and once per stage over the whole batch
// (the per-stage graphs serve calls that time each stage with events).
// Replaces earlier instances.
cudaError_t instantiate_graphs(of_handle* H, Plan* P) {
    if (P->exec) cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
    for (auto& x : P->stage_exec) {
        if (x) cudaGraphExecDestroy(x);
        x = nullptr;
    }
    cudaGraph_t g = nullptr;
    const int k = P->tun.stream_groups;
    cudaError_t e = capture(H, P, 0, kStages, &g, (k > 1 && (int)P->groups[k].size() == k) ? k : 1);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    for (int st = 0; st < kStages && e == cudaSuccess; ++st) {
        g = nullptr;
        e = capture(H, P, st, st + 1, &g);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P->stage_exec[st], g, 0);
        if (g) cudaGraphDestroy(g);
    }
    return e;
}

int build_plan(of_handle* H, const std::vector<FrameKey>& frames, const Settings& s,
               Plan** out) {
    Plan* P = new Plan();
    P->frames = frames;
    P->s = s;
    P->lay = make_layout(frames, s, -1);
    if (P->lay.total > H->arena_bytes) {
        free_plan(P);
        return fail(OF_ERR_TOO_LARGE, "batch needs " + std::to_string(P->lay.total) +
                                          " bytes of scratch; handle has " +
                                          std::to_string(H->arena_bytes));
    }
    const int nl = s.levels;
    const int nf = (int)frames.size();
    P->n_img = nf * nl;
    // Cell tiles: FAST applies the per-cell threshold itself (cells of 8..30 pixels).
    P->cell_tiles = s.cell >= CT_MIN_CELL && s.cell <= CT_MAX_CELL;
    P->aligned_ok = P->cell_tiles && fast_aligned_ok(s.cell);
    P->strip_ok = s.cell <= CS_MAX_CELL;
    // The threshold pass flags the cells itself when a band's cells fit its
    // shared array; otherwise the general FAST kernel sets them.
    P->apply_flags = true;
    for (const auto& L : P->lay.img)
        if (L.ncx > CA_MAX_CELLS) P->apply_flags = false;
    uint8_t* A = H->arena;

    // Image descriptors.
    P->h_img.resize(P->n_img);
    int slot = 0;
    for (int f = 0; f < nf; ++f) {
        for (int l = 0; l < nl; ++l) {
            const ImgLayout& L = P->lay.img[f * nl + l];
            Img& I = P->h_img[f * nl + l];
            std::memset(&I, 0, sizeof(I));
            I.img = (l == 0 && !frames[f].copy) ? nullptr : A + L.lev;  // bound per call
            I.w = L.w;
            I.h = L.h;
            I.pitch = L.pitch;
            I.spitch = L.spitch;
            I.ncx = L.ncx;
            I.ncy = L.ncy;
            I.cand_cap = L.cap;
            I.quota = L.quota;
            I.frame = f;
            I.level = l;
            I.lscale = L.lscale;
            I.ctr = reinterpret_cast<int32_t*>(A + L.ctr);
            if (L.det) {
                I.score = A + L.score;
                I.cell = reinterpret_cast<uint32_t*>(A + L.cell);
                I.ckey = reinterpret_cast<uint64_t*>(A + L.ckey);
                I.cyx = reinterpret_cast<uint32_t*>(A + L.cyx);
                I.kkey = reinterpret_cast<uint64_t*>(A + L.kkey);
                I.kyx = reinterpret_cast<uint32_t*>(A + L.kyx);
                I.tiles_x = L.tiles_x;
                I.tiles_y = L.tiles_y;
                I.tile_x0 = L.tile_x0;
                if (P->cell_tiles) I.ftiles_x = (I.ncx + CT_MAX_W / s.cell - 1) / (CT_MAX_W / s.cell);
            } else {
                I.quota = 0;  // an empty level keeps nothing; its share is not redistributed
            }
            I.slot0 = slot;
            slot += L.quota;
            P->max_quota = std::max(P->max_quota, I.quota);
        }
    }
    P->total_slots = slot;

    // Level-0 coordinate tables of the keypoint records (deduplicated per
    // (length, scale^level)): the orientation kernel then needs no float64.
    std::vector<std::pair<int, int>> ftab_idx(P->n_img);
    {
        std::map<std::pair<int, uint64_t>, int> ftab_of;
        auto ftable = [&](int n, double ls) {
            uint64_t bits = 0;
            std::memcpy(&bits, &ls, sizeof(bits));
            const auto key = std::make_pair(n, bits);
            const auto it = ftab_of.find(key);
            if (it != ftab_of.end()) return it->second;
            const int at = (int)P->ftables.size();
            for (int i = 0; i < n; ++i) P->ftables.push_back((float)((double)i * ls));
            ftab_of[key] = at;
            return at;
        };
        for (int i = 0; i < P->n_img; ++i)
            ftab_idx[i] = std::make_pair(ftable(P->h_img[i].w, P->h_img[i].lscale),
                                         ftable(P->h_img[i].h, P->h_img[i].lscale));
    }

    // Resize jobs and their tables (deduplicated per (n_src, n_dst)).
    std::map<std::pair<int, int>, int> tab_of;
    auto table = [&](int n_src, int n_dst) {
        auto key = std::make_pair(n_src, n_dst);
        auto it = tab_of.find(key);
        if (it != tab_of.end()) return it->second;
        const int at = (int)P->tables.size();
        P->tables.resize(at + n_dst);
        ofh::resize_table(n_src, n_dst, P->tables.data() + at);
        tab_of[key] = at;
        return at;
    };
    std::vector<std::pair<int, int>> tab_idx;  // (xtab, ytab) offsets per job
    P->rs_begin.assign(nl + 1, 0);
    for (int l = 1; l < nl; ++l) {
        P->rs_begin[l] = (int)P->h_rs.size();
        for (int f = 0; f < nf; ++f) {
            const Img& S = P->h_img[f * nl + l - 1];
            const Img& D = P->h_img[f * nl + l];
            if (D.w == 0 || S.w == 0) continue;
            Resize R;
            std::memset(&R, 0, sizeof(R));
            R.src = S.img;  // level 0 bound per call
            R.dst = const_cast<uint8_t*>(D.img);
            R.sw = S.w;
            R.sh = S.h;
            R.spitch = S.pitch;
            R.dw = D.w;
            R.dh = D.h;
            R.dpitch = D.pitch;
            R.tiles_x = (D.w + RS_TILE_W - 1) / RS_TILE_W;
            R.tiles_y = 0;  // depends on the tile height; the groups' prefix arrays carry it
            tab_idx.emplace_back(table(S.w, D.w), table(S.h, D.h));
            P->h_rs.push_back(R);
            P->rs_frame.push_back(f);
        }
    }
    P->rs_begin[nl] = (int)P->h_rs.size();
    // Source boxes of the persistent TMA resize; a level uses it when every
    // job's box fits (<= 256 x 256) and consecutive x0 differ by at most 3.
    P->rt_buf.assign(nl + 1, 0);
    P->rt_bps.assign(nl + 1, 0);
    for (int l = 1; l < nl; ++l) {
        bool ok = P->rs_begin[l + 1] > P->rs_begin[l];
        int buf = 0;
        for (int i = P->rs_begin[l]; i < P->rs_begin[l + 1]; ++i) {
            Resize& R = P->h_rs[i];
            const int32_t* xt = P->tables.data() + tab_idx[i].first;
            const int32_t* yt = P->tables.data() + tab_idx[i].second;
            int bw = 0, bh = 0, step = 0;
            for (int X0 = 0; X0 < R.dw; X0 += RS_TILE_W) {
                const int last = std::min(X0 + RS_TILE_W, R.dw) - 1;
                bw = std::max(bw, (xt[last] >> 12) + 2 - ((xt[X0] >> 12) & ~15));
            }
            for (int Y0 = 0; Y0 < R.dh; Y0 += RT_TILE_H) {
                const int last = std::min(Y0 + RT_TILE_H, R.dh) - 1;
                bh = std::max(bh, (yt[last] >> 12) + 2 - (yt[Y0] >> 12));
            }
            for (int d = 1; d < R.dw; ++d) step = std::max(step, (xt[d] >> 12) - (xt[d - 1] >> 12));
            bw = (bw + 15) & ~15;
            if (bw <= 256 && bh <= 256 && step <= 3) {
                R.box_w = bw;
                R.box_h = bh;
                buf = std::max(buf, (bw * bh + 16 + 127) & ~127);  // +16: a lane's word pair may end past the box
            } else {
                ok = false;
            }
        }
        if (ok && buf <= RT_MAX_BUF) {
            const int bps = resize_tma_blocks_per_sm(buf);
            if (bps > 0) {
                P->rt_buf[l] = buf;
                P->rt_bps[l] = bps;
            }
        }
    }
    for (int i = 0; i < P->n_img; ++i) {
        const Img& I = P->h_img[i];
        if (I.tiles_x > 0) {
            P->det_list.push_back(i);
            P->det_prefix.push_back(P->det_tiles);
            P->det_tiles += I.tiles_x * I.tiles_y;
        }
    }

    // Launch ranges per frame group (k = 1 .. min(kMaxGroups, frames)).
    for (int k = 1; k <= kMaxGroups; ++k) {
        if (k > nf) break;
        for (int g = 0; g < k; ++g) {
            Plan::Group G;
            const int f0 = nf * g / k, f1 = nf * (g + 1) / k;
            G.img_begin = f0 * nl;
            G.n_img = (f1 - f0) * nl;
            const int nd = (int)P->det_list.size();
            int j0 = 0, j1 = 0;
            while (j0 < nd && P->det_list[j0] < G.img_begin) ++j0;
            j1 = j0;
            while (j1 < nd && P->det_list[j1] < G.img_begin + G.n_img) ++j1;
            G.dl_begin = j0;
            G.n_list = j1 - j0;
            G.dp_off = (int)P->gp_det.size();
            const int t0 = j0 < nd ? P->det_prefix[j0] : P->det_tiles;
            for (int j = j0; j < j1; ++j) P->gp_det.push_back(P->det_prefix[j] - t0);
            G.det_tiles = (j1 < nd ? P->det_prefix[j1] : P->det_tiles) - t0;
            G.fp_off = (int)P->gp_fast.size();
            G.rp_off = (int)P->gp_rows.size();
            G.np_off = (int)P->gp_nms64.size();
            for (int i = 0; i < 2; ++i) G.ftall_off[i] = (int)P->gp_ftall[i].size();
            G.fal_off = (int)P->gp_fal.size();
            G.cs_off = (int)P->gp_cstrip.size();
            G.csi_off = (int)P->items_cs.size();
            G.dti_off = (int)P->items_dt.size();
            for (int j = j0; j < j1; ++j) {
                const Img& I = P->h_img[P->det_list[j]];
                const uint32_t ii = (uint32_t)P->det_list[j];
                for (int ty = 0; ty < I.tiles_y; ++ty)  // tile t = ty * tiles_x + tx, as the prefixes count
                    for (int tx = 0; tx < I.tiles_x; ++tx)
                        P->items_dt.push_back(make_uint2(
                            ii, ((uint32_t)(s.border + ty * TILE_H) << 16) | (uint32_t)(I.tile_x0 + tx * TILE_W)));
                if (P->strip_ok)
                    for (int cy = 0; cy < I.ncy; ++cy)
                        for (int tx = 0; tx < I.tiles_x; ++tx)
                            P->items_cs.push_back(make_uint2(
                                ii, ((uint32_t)(s.border + cy * s.cell) << 16) | (uint32_t)(I.tile_x0 + tx * TILE_W)));
                P->gp_nms64.push_back(G.nms64_tiles);
                G.nms64_tiles += I.tiles_x * ((I.h - 2 * s.border + 63) / 64);
                for (int i = 0; i < 2; ++i) {
                    P->gp_ftall[i].push_back(G.ftall_tiles[i]);
                    G.ftall_tiles[i] += I.tiles_x * ((I.h - 2 * s.border + FT_HS[i] - 1) / FT_HS[i]);
                }
                P->gp_fal.push_back(G.fal_tiles);
                if (P->aligned_ok) {
                    const int cr = FAST_AL_T / s.cell;  // cell rows per tile
                    G.fal_tiles += I.ftiles_x * ((I.ncy + cr - 1) / cr);
                }
                P->gp_fast.push_back(G.fast_tiles);
                G.fast_tiles += P->cell_tiles ? I.ftiles_x * ((I.ncy + ct_cell_rows(s.cell) - 1) / ct_cell_rows(s.cell)) : 0;
                P->gp_rows.push_back(G.n_bands);
                G.n_bands += I.ncy;
                P->gp_cstrip.push_back(G.cs_strips);
                G.cs_strips += P->strip_ok ? I.tiles_x * I.ncy : 0;
            }
            G.slot_begin = P->h_img[G.img_begin].slot0;
            G.slot_end = f1 < nf ? P->h_img[f1 * nl].slot0 : P->total_slots;
            G.rs_job.assign(nl + 1, 0);
            G.rs_n.assign(nl + 1, 0);
            G.rsi_off.assign(nl + 1, 0);
            for (int v = 0; v < 2; ++v) {
                G.rsp_off[v].assign(nl + 1, 0);
                G.rs_tiles[v].assign(nl + 1, 0);
            }
            for (int l = 1; l < nl; ++l) {
                int b = P->rs_begin[l];
                while (b < P->rs_begin[l + 1] && P->rs_frame[b] < f0) ++b;
                int e = b;
                while (e < P->rs_begin[l + 1] && P->rs_frame[e] < f1) ++e;
                G.rs_job[l] = b;
                G.rs_n[l] = e - b;
                G.rsi_off[l] = (int)P->items_rs.size();
                for (int i = b; i < e; ++i)  // tile t = ty * tiles_x + tx of job i - b, as the prefixes count
                    for (int ty = 0; ty < (P->h_rs[i].dh + RT_TILE_H - 1) / RT_TILE_H; ++ty)
                        for (int tx = 0; tx < P->h_rs[i].tiles_x; ++tx)
                            P->items_rs.push_back(make_uint2(
                                (uint32_t)(i - b), ((uint32_t)(ty * RT_TILE_H) << 16) | (uint32_t)(tx * RS_TILE_W)));
                for (int v = 0; v < 2; ++v) {
                    G.rsp_off[v][l] = (int)P->gp_rs.size();
                    int tiles = 0;
                    for (int i = b; i < e; ++i) {
                        P->gp_rs.push_back(tiles);
                        tiles += P->h_rs[i].tiles_x * ((P->h_rs[i].dh + RS_TILE_HS[v] - 1) / RS_TILE_HS[v]);
                    }
                    G.rs_tiles[v][l] = tiles;
                }
            }
            P->groups[k].push_back(G);
        }
    }

    Call& C = P->h_call;
    std::memset(&C, 0, sizeof(C));
    C.knum = s.knum;
    C.kden = s.kden;
    C.n_frames = nf;
    C.levels = nl;
    C.n_features = s.n_features;
    C.t_hi = s.t_hi;
    C.t_lo = s.t_lo;
    C.border = s.border;
    C.cell = s.cell;
    C.radius = s.radius;
    C.n_img = P->n_img;
    C.total_slots = P->total_slots;
    C.resp_scale = ofh::response_scale(s.kden);
    C.status = H->d_counts + 4;
    P->tun.resize_tile_h = RS_TILE_HS[1];
    P->tun.resize_tma = 1;
    P->tun.stream_groups = 1;
    // Untuned plans.  Batches of 4 frames or more start from the autotuner's
    // choice on 1080p batches: the cell-row strips (form 4, which set the cell
    // flags) and the per-warp NMS kernel, which applies them (no threshold
    // pass).  Fewer frames per call are launch-bound; there the cell-tile form
    // with the block NMS kernel measured faster (0.144 against 0.150 ms for
    // one 1080p frame per call).
    const bool big = nf >= 4 && P->strip_ok;
    P->tun.fast_cell_tiles = big ? 4 : P->cell_tiles ? 1 : 0;
    P->tun.fast_tile_h = 32;
    P->tun.fast_blocks_per_sm = plan_fast_bps(P);
    P->tun.nms_tile_h = big ? 32 : 64;
    P->tun.nms_blocks_per_sm = nms_blocks_per_sm(P->tun.nms_tile_h, true);
    for (int i = 0; i < 2; ++i)  // raise the tall kernels' shared-memory limits before any capture
        for (int fl = 0; fl < 2; ++fl) fast_blocks_per_sm(FT_HS[i], fl != 0);
    for (int th = 32; th <= 128; th *= 2)
        for (int fin = 0; fin < 2; ++fin) nms_blocks_per_sm(th, fin != 0);
    fast_aligned_blocks_per_sm();  // raises the cell-aligned kernel's shared-memory limit
    fast_warp_blocks_per_sm();     // ... and the per-warp kernels'
    fast_cstrip_blocks_per_sm();
    P->tun.fast_order = 0;
    P->tun.nms_order = 0;

    // Tensor maps: image boxes for FAST and NMS, score boxes for NMS, then
    // the source box of each resize job (TMA resize).
    P->h_maps.assign(2 * P->n_img + P->h_rs.size(), CUtensorMap{});
    for (int i = 0; i < P->n_img; ++i) {
        const Img& I = P->h_img[i];
        int rc = encode_u8(&P->h_maps[i], I.img, I.w, I.h, I.pitch, SROW, IMG_BOX_ROWS);
        if (rc == OF_OK && I.score)
            rc = encode_u8(&P->h_maps[P->n_img + i], I.score, I.w, I.h, I.spitch, SROW, SCORE_BOX_ROWS);
        if (rc != OF_OK) {
            free_plan(P);
            return rc;
        }
    }
    for (size_t i = 0; i < P->h_rs.size(); ++i) {
        const Resize& R = P->h_rs[i];
        if (R.box_w == 0) continue;
        const int rc = encode_u8(&P->h_maps[2 * P->n_img + i], R.src, R.sw, R.sh, R.spitch, R.box_w, R.box_h);
        if (rc != OF_OK) {
            free_plan(P);
            return rc;
        }
    }

    // Device descriptor block: [Call | Img[] | Resize[]] (re-uploaded when
    // pointers change) then [detect list | tables | group tile prefixes
    // (detect, resize)].
    size_t off = 0;
    P->off_call = off;
    off = align_up(off + sizeof(Call), 16);
    P->off_img = off;
    off = align_up(off + sizeof(Img) * P->n_img, 16);
    P->off_rs = off;
    off = align_up(off + sizeof(Resize) * std::max<size_t>(P->h_rs.size(), 1), 128);
    P->off_maps = off;
    off = align_up(off + sizeof(CUtensorMap) * P->h_maps.size(), 16);
    P->header_bytes = off;
    P->off_dl = off;
    off = align_up(off + sizeof(int32_t) * std::max<size_t>(P->det_list.size(), 1), 16);
    P->off_tab = off;
    off = align_up(off + sizeof(int32_t) * std::max<size_t>(P->tables.size(), 1), 16);
    P->off_ftab = off;
    off = align_up(off + sizeof(float) * std::max<size_t>(P->ftables.size(), 1), 16);
    P->off_gdp = off;
    off = align_up(off + sizeof(int32_t) * std::max<size_t>(P->gp_det.size(), 1), 16);
    P->off_grs = off;
    off = align_up(off + sizeof(int32_t) * std::max<size_t>(P->gp_rs.size(), 1), 16);
    P->off_gfp = off;
    off = align_up(off + sizeof(int32_t) * std::max<size_t>(P->gp_fast.size(), 1), 16);
    P->off_grp = off;
    off = align_up(off + sizeof(int32_t) * std::max<size_t>(P->gp_rows.size(), 1), 16);
    P->off_gnp = off;
    off = align_up(off + sizeof(int32_t) * std::max<size_t>(P->gp_nms64.size(), 1), 16);
    for (int i = 0; i < 2; ++i) {
        P->off_gft[i] = off;
        off = align_up(off + sizeof(int32_t) * std::max<size_t>(P->gp_ftall[i].size(), 1), 16);
    }
    P->off_gfal = off;
    off = align_up(off + sizeof(int32_t) * std::max<size_t>(P->gp_fal.size(), 1), 16);
    P->off_gcs = off;
    off = align_up(off + sizeof(int32_t) * std::max<size_t>(P->gp_cstrip.size(), 1), 16);
    P->off_ics = off;
    off = align_up(off + sizeof(uint2) * std::max<size_t>(P->items_cs.size(), 1), 16);
    P->off_idt = off;
    off = align_up(off + sizeof(uint2) * std::max<size_t>(P->items_dt.size(), 1), 16);
    P->off_irs = off;
    off = align_up(off + sizeof(uint2) * std::max<size_t>(P->items_rs.size(), 1), 16);
    // Output slot -> image (slots of image i: [slot0, slot0 + layout quota)).
    P->slot_img.assign(std::max(P->total_slots, 1), 0);
    for (int i = 0; i < P->n_img; ++i) {
        const int e = i + 1 < P->n_img ? P->h_img[i + 1].slot0 : P->total_slots;
        for (int k = P->h_img[i].slot0; k < e; ++k) P->slot_img[k] = (uint16_t)i;
    }
    P->off_sli = off;
    off = align_up(off + sizeof(uint16_t) * P->slot_img.size(), 16);
    cudaError_t e = cudaMalloc(&P->dbuf, off);
    if (e != cudaSuccess) {
        free_plan(P);
        return fail(OF_ERR_CUDA, std::string("cudaMalloc(descriptors): ") + cudaGetErrorString(e));
    }
    const float* d_ftab = reinterpret_cast<const float*>(P->dbuf + P->off_ftab);
    for (int i = 0; i < P->n_img; ++i) {
        P->h_img[i].fx = d_ftab + ftab_idx[i].first;
        P->h_img[i].fy = d_ftab + ftab_idx[i].second;
    }
    const int32_t* d_tab = reinterpret_cast<const int32_t*>(P->dbuf + P->off_tab);
    for (size_t i = 0; i < P->h_rs.size(); ++i) {
        P->h_rs[i].xtab = d_tab + tab_idx[i].first;
        P->h_rs[i].ytab = d_tab + tab_idx[i].second;
    }
    std::vector<uint8_t> blob(off, 0);
    auto put = [&](size_t at, const void* src, size_t n) {
        if (n) std::memcpy(blob.data() + at, src, n);
    };
    put(P->off_call, &C, sizeof(C));
    put(P->off_img, P->h_img.data(), sizeof(Img) * P->h_img.size());
    put(P->off_rs, P->h_rs.data(), sizeof(Resize) * P->h_rs.size());
    put(P->off_maps, P->h_maps.data(), sizeof(CUtensorMap) * P->h_maps.size());
    put(P->off_dl, P->det_list.data(), sizeof(int32_t) * P->det_list.size());
    put(P->off_tab, P->tables.data(), sizeof(int32_t) * P->tables.size());
    put(P->off_ftab, P->ftables.data(), sizeof(float) * P->ftables.size());
    put(P->off_gdp, P->gp_det.data(), sizeof(int32_t) * P->gp_det.size());
    put(P->off_grs, P->gp_rs.data(), sizeof(int32_t) * P->gp_rs.size());
    put(P->off_gfp, P->gp_fast.data(), sizeof(int32_t) * P->gp_fast.size());
    put(P->off_grp, P->gp_rows.data(), sizeof(int32_t) * P->gp_rows.size());
    put(P->off_gnp, P->gp_nms64.data(), sizeof(int32_t) * P->gp_nms64.size());
    for (int i = 0; i < 2; ++i) put(P->off_gft[i], P->gp_ftall[i].data(), sizeof(int32_t) * P->gp_ftall[i].size());
    put(P->off_gfal, P->gp_fal.data(), sizeof(int32_t) * P->gp_fal.size());
    put(P->off_gcs, P->gp_cstrip.data(), sizeof(int32_t) * P->gp_cstrip.size());
    put(P->off_ics, P->items_cs.data(), sizeof(uint2) * P->items_cs.size());
    put(P->off_idt, P->items_dt.data(), sizeof(uint2) * P->items_dt.size());
    put(P->off_irs, P->items_rs.data(), sizeof(uint2) * P->items_rs.size());
    put(P->off_sli, P->slot_img.data(), sizeof(uint16_t) * P->slot_img.size());
    e = cudaMemcpy(P->dbuf, blob.data(), off, cudaMemcpyHostToDevice);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMallocHost(&P->stage[i], P->header_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        free_plan(P);
        return fail(OF_ERR_CUDA, std::string("plan setup: ") + cudaGetErrorString(e));
    }

    e = instantiate_graphs(H, P);
    if (e != cudaSuccess) {
        free_plan(P);
        return fail(OF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    *out = P;
    return OF_OK;
}

// Upload the descriptor header (call constants, images, resize jobs, tensor
// maps) through the plan's pinned staging ring, ordered on the handle's stream.
int upload_header(of_handle* H, Plan* P) {
    const int si = P->stage_i;
    P->stage_i ^= 1;
    OF_CK(cudaEventSynchronize(P->ev[si]));
    uint8_t* st = P->stage[si];
    std::memcpy(st + P->off_call, &P->h_call, sizeof(Call));
    std::memcpy(st + P->off_img, P->h_img.data(), sizeof(Img) * P->h_img.size());
    std::memcpy(st + P->off_rs, P->h_rs.data(), sizeof(Resize) * P->h_rs.size());
    std::memcpy(st + P->off_maps, P->h_maps.data(), sizeof(CUtensorMap) * P->h_maps.size());
    OF_CK(cudaMemcpyAsync(P->dbuf, st, P->header_bytes, cudaMemcpyHostToDevice, H->stream));
    OF_CK(cudaEventRecord(P->ev[si], H->stream));
    return OF_OK;
}

// Turn the proposal masks of a plan on (learned path) or off (plain path).
int set_pmask(of_handle* H, Plan* P, bool on) {
    if (P->pmask_on == on) return OF_OK;
    for (size_t j = 0; j < P->det_list.size(); ++j)
        P->h_img[P->det_list[j]].pmask = on ? P->lbuf + P->off_mask + P->ptile_prefix[j] : nullptr;
    P->pmask_on = on;
    return upload_header(H, P);
}

// Device buffers of the learned path (first use of a plan).
int ensure_learned(Plan* P) {
    if (P->lbuf) return OF_OK;
    const size_t nl = P->det_list.size();
    P->ptile_prefix.assign(nl + 1, 0);
    for (size_t j = 0; j < nl; ++j) {
        const Img& I = P->h_img[P->det_list[j]];
        P->ptile_prefix[j + 1] = P->ptile_prefix[j] + 4 * I.tiles_x * I.tiles_y;  // multiple of 4
    }
    const size_t nt = (size_t)P->ptile_prefix[nl];
    size_t off = 0;
    P->off_mask = off;
    off = align_up(off + std::max<size_t>(nt, 4), 256);
    P->off_pos = off;
    off = align_up(off + std::max<size_t>(nt, 4), 256);
    P->off_logit = off;
    off = align_up(off + sizeof(float) * std::max<size_t>(nt, 1), 256);
    P->off_pp = off;
    off = align_up(off + sizeof(int32_t) * (nl + 1), 256);
    P->off_stats = off;
    off += 4 * sizeof(int32_t);
    cudaError_t e = cudaMalloc(&P->lbuf, off);
    if (e == cudaSuccess)
        e = cudaMemcpy(P->lbuf + P->off_pp, P->ptile_prefix.data(), sizeof(int32_t) * (nl + 1),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(OF_ERR_CUDA, std::string("learned-path buffers: ") + cudaGetErrorString(e));
    return OF_OK;
}

// Point the plan at this call's frames and output, re-uploading the
// descriptor header when anything changed.
int bind_plan(of_handle* H, Plan* P, const of_frame* frames, of_keypoint* out, int32_t* counts) {
    const int nl = P->s.levels;
    const int nf = (int)P->frames.size();
    bool changed = !P->bound || P->bound_out != out || P->bound_counts != counts;
    if (!changed)
        for (int f = 0; f < nf; ++f)
            if (!P->frames[f].copy && P->bound_src[f] != frames[f].img) changed = true;
    if (!changed) return OF_OK;
    P->bound_src.assign(nf, nullptr);
    for (int f = 0; f < nf; ++f) {
        if (P->frames[f].copy) continue;
        P->bound_src[f] = frames[f].img;
        Img& I0 = P->h_img[f * nl];
        I0.img = frames[f].img;
        const int rc = encode_u8(&P->h_maps[f * nl], I0.img, I0.w, I0.h, I0.pitch, SROW, IMG_BOX_ROWS);
        if (rc != OF_OK) return rc;
    }
    // Level-1 resize jobs read level 0.
    if (nl > 1) {
        for (int i = P->rs_begin[1]; i < P->rs_begin[2]; ++i) {
            Resize& R = P->h_rs[i];
            for (int f = 0; f < nf; ++f)
                if (R.dst == P->h_img[f * nl + 1].img) R.src = P->h_img[f * nl].img;
            if (R.box_w > 0) {
                const int rc = encode_u8(&P->h_maps[2 * P->n_img + i], R.src, R.sw, R.sh, R.spitch, R.box_w,
                                         R.box_h);
                if (rc != OF_OK) return rc;
            }
        }
    }
    P->h_call.out = out;
    P->h_call.counts = counts;
    P->bound_out = out;
    P->bound_counts = counts;
    P->bound = true;
    return upload_header(H, P);
}

Plan* find_plan(of_handle* H, const std::vector<FrameKey>& frames, const Settings& s) {
    for (Plan* P : H->plans) {
        if (P->frames.size() != frames.size()) continue;
        const Settings& t = P->s;
        if (t.levels != s.levels || t.scale != s.scale || t.t_hi != s.t_hi || t.t_lo != s.t_lo ||
            t.knum != s.knum || t.kden != s.kden || t.n_features != s.n_features)
            continue;
        bool same = true;
        for (size_t i = 0; i < frames.size() && same; ++i) same = P->frames[i] == frames[i];
        if (same) return P;
    }
    return nullptr;
}

// Validate a batch, find or build its plan, stage unaligned frames and bind
// the call's pointers.  Launches nothing.
int prepare_batch(of_handle* H, const of_frame* frames, int n_frames, int levels, float scale,
                  int fast_t, float harris_k, int n_features, of_keypoint* out, int32_t* counts,
                  Plan** outP) {
    if (!H) return fail(OF_ERR_ARG, "null handle");
    if (!frames || n_frames < 1) return fail(OF_ERR_ARG, "no frames");
    if (n_frames > H->p.max_batch)
        return fail(OF_ERR_TOO_LARGE, "n_frames exceeds max_batch");
    if (levels < 1 || levels > H->p.max_levels) return fail(OF_ERR_ARG, "levels out of range");
    if (!(scale >= H->p.min_scale && scale <= 4.0f))
        return fail(OF_ERR_ARG, "scale must be in [min_scale, 4]");
    if (fast_t < 1 || fast_t > 255) return fail(OF_ERR_ARG, "fast_t must be in 1..255");
    if (n_features < 0 || n_features > H->p.max_features)
        return fail(OF_ERR_ARG, "n_features out of range");
    if (!counts || (n_features > 0 && !out)) return fail(OF_ERR_ARG, "null output pointer");
    Settings s{};
    s.levels = levels;
    s.scale = scale;
    s.t_hi = fast_t;
    s.t_lo = (H->p.fast_t_lo > 0 && H->p.fast_t_lo < fast_t) ? H->p.fast_t_lo : fast_t;
    if (!ofh::k_fraction(harris_k, &s.knum, &s.kden))
        return fail(OF_ERR_ARG, "harris_k must be in [0, 0.25] with a reduced denominator <= 3000");
    s.n_features = n_features;
    s.border = H->p.border;
    s.cell = H->p.cell;
    s.radius = H->p.orient_radius;
    std::vector<FrameKey> keys(n_frames);
    for (int i = 0; i < n_frames; ++i) {
        const of_frame& F = frames[i];
        if (!F.img || F.w < 1 || F.h < 1 || F.pitch < F.w)
            return fail(OF_ERR_ARG, "bad frame " + std::to_string(i));
        if (F.w > H->p.max_w || F.h > H->p.max_h)
            return fail(OF_ERR_TOO_LARGE, "frame larger than max_w x max_h");
        const bool aligned = ((uintptr_t)F.img % 16 == 0) && (F.pitch % 16 == 0);
        keys[i] = FrameKey{F.w, F.h, F.pitch, !aligned};
    }
    Plan* P = find_plan(H, keys, s);
    if (!P) {
        if ((int)H->plans.size() >= kMaxPlans) {
            auto it = std::min_element(H->plans.begin(), H->plans.end(),
                                       [](Plan* a, Plan* b) { return a->stamp < b->stamp; });
            OF_CK(cudaStreamSynchronize(H->stream));
            if (H->last == *it) H->last = nullptr;
            free_plan(*it);
            H->plans.erase(it);
        }
        const int rc = build_plan(H, keys, s, &P);
        if (rc != OF_OK) return rc;
        H->plans.push_back(P);
    }
    P->stamp = ++H->clock;
    for (int i = 0; i < n_frames; ++i) {
        if (!keys[i].copy) continue;
        const Img& I = P->h_img[i * levels];
        OF_CK(cudaMemcpy2DAsync(const_cast<uint8_t*>(I.img), I.pitch, frames[i].img, frames[i].pitch,
                                frames[i].w, frames[i].h, cudaMemcpyDeviceToDevice, H->stream));
    }
    const int rc = bind_plan(H, P, frames, out, counts);
    if (rc != OF_OK) return rc;
    *outP = P;
    return OF_OK;
}

// Time the candidate launch configurations of a bound plan on its own data
// and keep the fastest per stage:
//   pyramid  staged kernel with 128 x 32 or 128 x 64 output tiles, or the
//            persistent TMA kernel;
//   FAST     general kernel on 32-, 64-, 128- or 256-row tiles (the tall
//            ones when the threshold pass sets the flags) or the cell-tile
//            kernel; 1 .. max resident blocks per SM; round-robin or
//            contiguous tiles (timed together with NMS);
//   NMS      32-, 64- or 128-row tiles, blocks per SM, tile order;
//   groups   the batch as 1 .. 8 frame groups on forked graph branches.
// Stages are timed one at a time with CUDA events (mean of a few repetitions
// after a warm-up); select and orientation are not tuned.  The plan's graphs
// are re-captured with the winners.
int autotune_plan(of_handle* H, Plan* P, int reps) {
    cudaStream_t st = H->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    OF_CK(cudaEventCreate(&e0));
    OF_CK(cudaEventCreate(&e1));
    int tried = 0;
    auto timed = [&](auto&& enqueue, float* ms) -> int {
        enqueue();
        OF_CK(cudaEventRecord(e0, st));
        for (int i = 0; i < reps; ++i) enqueue();
        OF_CK(cudaEventRecord(e1, st));
        OF_CK(cudaEventSynchronize(e1));
        float t = 0.f;
        OF_CK(cudaEventElapsedTime(&t, e0, e1));
        *ms = t / reps;
        ++tried;
        return OF_OK;
    };
    const size_t ctr_bytes = 4 * sizeof(int32_t) * (size_t)P->n_img;
    int rc = OF_OK;
    enqueue_stages(H, P, 0, kStages, st);  // every buffer populated once
    // Pyramid (idempotent).
    // Candidates: the staged kernel with 32- or 64-row tiles, then the
    // persistent TMA kernel (on the levels it covers; staged 64 elsewhere).
    float best = 1e30f;
    int best_h = P->tun.resize_tile_h, best_tma = P->tun.resize_tma;
    for (int c = 0; c < 3 && rc == OF_OK; ++c) {
        P->tun.resize_tile_h = RS_TILE_HS[c == 0 ? 0 : 1];
        P->tun.resize_tma = c == 2;
        float ms = 0.f;
        rc = timed([&] { enqueue_stages(H, P, 0, 1, st); }, &ms);
        if (ms < best) best = ms, best_h = P->tun.resize_tile_h, best_tma = P->tun.resize_tma;
    }
    P->tun.resize_tile_h = best_h;
    P->tun.resize_tma = best_tma;
    P->tun.resize_ms = best;
    // FAST (idempotent: rewrites score maps, sets the same cell flags): the
    // general kernel (+ threshold pass, stage 2), and the cell-tile kernel
    // where the cell size allows it; fast_ms below is FAST + NMS.
    best = 1e30f;
    int bb = P->tun.fast_blocks_per_sm, bo = 0, bv = P->tun.fast_cell_tiles, bt = P->tun.fast_tile_h;
    // Forms: general kernel (32-, 64-, 128- or 256-row tiles), cell tiles (1),
    // cell-aligned general kernel (2), general kernel with per-warp pipelines
    // (3), cell strips with per-warp pipelines (4).
    for (int cand = 0; cand < 8 && rc == OF_OK; ++cand) {
        const int v = cand < 4 ? 0 : cand - 3, th = cand < 4 ? 32 << cand : 32;
        if ((v == 1 && !P->cell_tiles) || (v == 2 && !P->aligned_ok) || (v == 4 && !P->strip_ok)) continue;
        P->tun.fast_cell_tiles = v;
        P->tun.fast_tile_h = th;
        for (int bp = 1; bp <= plan_fast_bps(P) && rc == OF_OK; ++bp) {
            for (int order = 0; order < 2 && rc == OF_OK; ++order) {
                P->tun.fast_blocks_per_sm = bp;
                P->tun.fast_order = order;
                // FAST and NMS together (NMS appends candidates: clear the
                // counters): the general form's threshold pass runs in stage 2.
                float ms = 0.f;
                rc = timed(
                    [&] {
                        cudaMemsetAsync(H->arena, 0, ctr_bytes, st);
                        enqueue_stages(H, P, 1, 3, st);
                    },
                    &ms);
                if (ms < best) best = ms, bb = bp, bo = order, bv = v, bt = th;
            }
        }
    }
    P->tun.fast_cell_tiles = bv;
    P->tun.fast_tile_h = bt;
    P->tun.fast_blocks_per_sm = bb;
    P->tun.fast_order = bo;
    P->tun.fast_ms = best;
    // NMS + Harris (appends candidates: clear the counters before each run),
    // 32-, 64- or 128-row tiles.
    best = 1e30f;
    bb = P->tun.nms_blocks_per_sm, bo = 0;
    int bth = P->tun.nms_tile_h;
    for (int th = 32; th <= 128 && rc == OF_OK; th *= 2)
    for (int bp = 1; bp <= nms_blocks_per_sm(th, true) && rc == OF_OK; ++bp) {
        for (int order = 0; order < 2 && rc == OF_OK; ++order) {
            P->tun.nms_tile_h = th;
            P->tun.nms_blocks_per_sm = bp;
            P->tun.nms_order = order;
            float ms = 0.f;
            rc = timed(
                [&] {
                    cudaMemsetAsync(H->arena, 0, ctr_bytes, st);
                    enqueue_stages(H, P, 2, 3, st);
                },
                &ms);
            if (ms < best) best = ms, bb = bp, bo = order, bth = th;
        }
    }
    P->tun.nms_tile_h = bth;
    P->tun.nms_blocks_per_sm = bb;
    P->tun.nms_order = bo;
    P->tun.nms_ms = best;
    // Whole-call graph with the chosen stages: one group, or 2..kMaxGroups
    // frame groups on forked branches.
    int best_g = 1;
    {
        float bg = 1e30f;
        for (int k = 1; k <= kMaxGroups && k <= (int)P->frames.size() && rc == OF_OK; ++k) {
            P->tun.stream_groups = k;
            const cudaError_t ge = instantiate_graphs(H, P);
            if (ge != cudaSuccess) {
                rc = fail(OF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ge));
                break;
            }
            float ms = 0.f;
            rc = timed([&] { cudaGraphLaunch(P->exec, st); }, &ms);
            if (ms < bg) bg = ms, best_g = k;
        }
    }
    P->tun.stream_groups = best_g;
    P->tun.candidates_tried = tried;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != OF_OK) return rc;
    OF_CK(cudaGetLastError());
    const cudaError_t e = instantiate_graphs(H, P);
    if (e != cudaSuccess) return fail(OF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    P->tuned = true;
    return OF_OK;
}

int run_batch(of_handle* H, const of_frame* frames, int n_frames, int levels, float scale,
              int fast_t, float harris_k, int n_features, of_keypoint* out, int32_t* counts) {
    if (!H) return fail(OF_ERR_ARG, "null handle");
    DeviceGuard dg(H->device);
    Plan* P = nullptr;
    int rc = prepare_batch(H, frames, n_frames, levels, scale, fast_t, harris_k, n_features, out,
                           counts, &P);
    if (rc != OF_OK) return rc;
    rc = set_pmask(H, P, false);
    if (rc != OF_OK) return rc;
    if (H->p.autotune && !P->tuned) {
        rc = autotune_plan(H, P, 3);
        if (rc != OF_OK) return rc;
    }
    if (n_features == 0) OF_CK(cudaMemsetAsync(counts, 0, sizeof(int32_t) * n_frames, H->stream));
    if (H->stage_timing) {
        for (int st = 0; st < kStages; ++st) {
            OF_CK(cudaEventRecord(H->stage_ev[st], H->stream));
            OF_CK(cudaGraphLaunch(P->stage_exec[st], H->stream));
        }
        OF_CK(cudaEventRecord(H->stage_ev[kStages], H->stream));
        H->stage_timing = false;
    } else {
        OF_CK(cudaGraphLaunch(P->exec, H->stream));
    }
    H->last = P;
    return OF_OK;
}

}  // namespace

namespace ofk {
// Lets other translation units report through of_last_error().
void set_last_error(const std::string& msg) { g_err = msg; }

int encode_u8_map(CUtensorMap* m, const void* base, int w, int h, int pitch, int box_w, int box_h) {
    const int rc = resolve_encoder();
    if (rc != OF_OK) return rc;
    return encode_u8(m, base, w, h, pitch, box_w, box_h);
}
}  // namespace ofk

extern "C" {

int of_version(void) { return OF_VERSION; }

const char* of_last_error(void) { return g_err.c_str(); }

of_handle* of_create(const of_params* pin) {
    if (!pin) {
        fail(OF_ERR_ARG, "null params");
        return nullptr;
    }
    of_params p = *pin;
    if (p.max_levels == 0) p.max_levels = 8;
    if (p.max_features == 0) p.max_features = 1000;
    if (p.max_batch == 0) p.max_batch = 1;
    if (p.min_scale == 0.0f) p.min_scale = 1.2f;
    if (p.cell == 0) p.cell = 30;
    if (p.border == 0) p.border = 19;
    if (p.harris_block == 0) p.harris_block = 7;
    if (p.orient_radius == 0) p.orient_radius = 15;
    if (p.arena_bytes < 0) {
        fail(OF_ERR_ARG, "arena_bytes must be >= 0");
        return nullptr;
    }
    if (p.autotune != 0 && p.autotune != 1) {
        fail(OF_ERR_ARG, "autotune must be 0 or 1");
        return nullptr;
    }
    if (p.max_w < 1 || p.max_h < 1 || p.max_w > 65535 || p.max_h > 65535 || p.max_levels < 1 ||
        p.max_levels > 16 || p.max_features < 0 || p.max_features > 8192 || p.max_batch < 1 ||
        !(p.min_scale > 1.0f) || p.fast_t_lo < 0 || p.fast_t_lo > 255 || p.cell < 8 ||
        p.border < 4 || p.orient_radius < 1 || p.orient_radius > 15 ||
        p.border < p.orient_radius) {
        fail(OF_ERR_ARG, "invalid of_params");
        return nullptr;
    }
    if (p.harris_block != 7) {
        fail(OF_ERR_UNSUPPORTED, "only harris_block = 7 is implemented");
        return nullptr;
    }
    of_handle* H = new of_handle();
    H->p = p;
    auto bail = [&](cudaError_t e, const char* what) -> of_handle* {
        fail(OF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
        of_destroy(H);
        return nullptr;
    };
    cudaError_t e = cudaGetDevice(&H->device);
    if (e != cudaSuccess) return bail(e, "cudaGetDevice");
    H->stream = (cudaStream_t)p.stream;  // NULL: the CUDA default stream
    e = cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking);
    for (int g = 0; g < kMaxGroups - 1 && e == cudaSuccess; ++g)
        e = cudaStreamCreateWithFlags(&H->cap_branch[g], cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(e, "cudaStreamCreate");
    e = cudaEventCreateWithFlags(&H->fork_ev, cudaEventDisableTiming);
    for (int g = 0; g < kMaxGroups - 1 && e == cudaSuccess; ++g)
        e = cudaEventCreateWithFlags(&H->join_ev[g], cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(e, "cudaEventCreate");
    // Scratch for the largest batch: max_batch frames of max_w x max_h.
    Settings s{};
    s.levels = p.max_levels;
    s.scale = p.min_scale;
    s.n_features = p.max_features;
    s.border = p.border;
    s.cell = p.cell;
    if (p.arena_bytes > 0) {
        H->arena_bytes = (size_t)p.arena_bytes;
    } else {
        std::vector<FrameKey> worst(p.max_batch, FrameKey{p.max_w, p.max_h, (int)align_up(p.max_w, 16), true});
        H->arena_bytes = make_layout(worst, s, p.max_features).total;
    }
    e = cudaMalloc(&H->arena, H->arena_bytes);
    if (e != cudaSuccess) return bail(e, "cudaMalloc(arena)");
    e = cudaMalloc(&H->d_counts, sizeof(int32_t) * 8);
    if (e != cudaSuccess) return bail(e, "cudaMalloc(counts)");
    e = cudaMemset(H->d_counts, 0, sizeof(int32_t) * 8);
    if (e != cudaSuccess) return bail(e, "cudaMemset(counts)");
    e = cudaMallocHost(&H->h_count, sizeof(int32_t) * 8);
    if (e != cudaSuccess) return bail(e, "cudaMallocHost");
    e = cudaDeviceGetAttribute(&H->n_sms, cudaDevAttrMultiProcessorCount, H->device);
    if (e != cudaSuccess) return bail(e, "cudaDeviceGetAttribute");
    if (resolve_encoder() != OF_OK) {
        of_destroy(H);
        return nullptr;
    }
    if (e != cudaSuccess) return bail(e, "cudaMallocHost");
    ofk::set_select_smem_limit(ofk::select_smem_bytes(std::max(p.max_features, 1)));
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(e, "cudaFuncSetAttribute");
    return H;
}

void of_destroy(of_handle* H) {
    if (!H) return;
    if (H->stream) cudaStreamSynchronize(H->stream);
    for (Plan* P : H->plans) free_plan(P);
    if (H->arena) cudaFree(H->arena);
    if (H->d_counts) cudaFree(H->d_counts);
    if (H->h_count) cudaFreeHost(H->h_count);
    if (H->cap_stream) cudaStreamDestroy(H->cap_stream);
    for (int g = 0; g < kMaxGroups - 1; ++g) {
        if (H->cap_branch[g]) cudaStreamDestroy(H->cap_branch[g]);
        if (H->join_ev[g]) cudaEventDestroy(H->join_ev[g]);
    }
    if (H->fork_ev) cudaEventDestroy(H->fork_ev);
    if (H->own_stream && H->stream) cudaStreamDestroy(H->stream);
    delete H;
}

int of_detect_batch(of_handle* H, const of_frame* frames, int n_frames, int levels, float scale,
                    int fast_t, float harris_k, int n_features, of_keypoint* out_kpts,
                    int32_t* out_counts) {
    return run_batch(H, frames, n_frames, levels, scale, fast_t, harris_k, n_features, out_kpts,
                     out_counts);
}

int of_autotune(of_handle* H, const of_frame* frames, int n_frames, int levels, float scale,
                int fast_t, float harris_k, int n_features, of_keypoint* out_kpts,
                int32_t* out_counts, int reps, of_tuning* result) {
    if (!H) return fail(OF_ERR_ARG, "null handle");
    if (reps < 1 || reps > 100) return fail(OF_ERR_ARG, "reps must be 1..100");
    DeviceGuard dg(H->device);
    Plan* P = nullptr;
    int rc = prepare_batch(H, frames, n_frames, levels, scale, fast_t, harris_k, n_features, out_kpts,
                           out_counts, &P);
    if (rc != OF_OK) return rc;
    rc = autotune_plan(H, P, reps);
    if (rc != OF_OK) return rc;
    if (n_features == 0) OF_CK(cudaMemsetAsync(out_counts, 0, sizeof(int32_t) * n_frames, H->stream));
    OF_CK(cudaGraphLaunch(P->exec, H->stream));  // leave this call's results in the outputs
    H->last = P;
    if (result) *result = P->tun;
    return OF_OK;
}

int of_set_tuning(of_handle* H, const of_frame* frames, int n_frames, int levels, float scale, int fast_t,
                  float harris_k, int n_features, of_keypoint* out_kpts, int32_t* out_counts,
                  const of_tuning* t) {
    if (!H) return fail(OF_ERR_ARG, "null handle");
    if (!t) return fail(OF_ERR_ARG, "null tuning");
    DeviceGuard dg(H->device);
    if ((t->resize_tile_h != RS_TILE_HS[0] && t->resize_tile_h != RS_TILE_HS[1]) ||
        (t->resize_tma != 0 && t->resize_tma != 1) || t->fast_blocks_per_sm < 1 ||
        t->fast_blocks_per_sm > std::max(fast_blocks_per_sm(), fast_cells_blocks_per_sm(CT_MAX_CELL)) ||
        t->nms_blocks_per_sm < 1 ||
        (t->nms_tile_h != 32 && t->nms_tile_h != 64 && t->nms_tile_h != 128) ||
        (t->fast_tile_h != 32 && t->fast_tile_h != 64 && t->fast_tile_h != FT_HS[0] && t->fast_tile_h != FT_HS[1]) ||
        t->nms_blocks_per_sm > nms_blocks_per_sm(t->nms_tile_h, true) || (t->fast_order != 0 && t->fast_order != 1) ||
        (t->nms_order != 0 && t->nms_order != 1) || t->stream_groups < 1 || t->stream_groups > kMaxGroups ||
        t->fast_cell_tiles < 0 || t->fast_cell_tiles > 4)
        return fail(OF_ERR_ARG, "tuning field out of range");
    Plan* P = nullptr;
    const int rc = prepare_batch(H, frames, n_frames, levels, scale, fast_t, harris_k, n_features, out_kpts,
                                 out_counts, &P);
    if (rc != OF_OK) return rc;
    P->tun.resize_tile_h = t->resize_tile_h;
    P->tun.resize_tma = t->resize_tma;
    // Forms the cell size does not allow fall back: aligned -> cell tiles -> general.
    P->tun.fast_cell_tiles = t->fast_cell_tiles == 3                              ? 3
                             : t->fast_cell_tiles == 4                            ? (P->strip_ok ? 4 : 0)
                             : !P->cell_tiles                                     ? 0
                             : (t->fast_cell_tiles == 2 && !P->aligned_ok)        ? 1
                                                                                   : t->fast_cell_tiles;
    P->tun.fast_tile_h = t->fast_tile_h;
    P->tun.fast_blocks_per_sm = std::min(t->fast_blocks_per_sm, plan_fast_bps(P));
    P->tun.nms_blocks_per_sm = t->nms_blocks_per_sm;
    P->tun.nms_tile_h = t->nms_tile_h;
    P->tun.fast_order = t->fast_order;
    P->tun.nms_order = t->nms_order;
    P->tun.stream_groups = std::min(t->stream_groups, (int)P->frames.size());
    const cudaError_t e = instantiate_graphs(H, P);
    if (e != cudaSuccess) return fail(OF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    P->tuned = true;
    return OF_OK;
}

int of_variant_detect(int fast_variant, int harris_variant, const uint8_t* img, int w, int h, int pitch, int fast_t,
                      int border, float harris_k, of_var_point* out_points, int32_t* out_count, int64_t capacity,
                      void* stream) {
    if (fast_variant < OF_VAR_FAST_BASELINE || fast_variant > OF_VAR_FAST_SM_BINARY)
        return fail(OF_ERR_ARG, "fast_variant out of range");
    if (harris_variant < OF_VAR_HARRIS_NONE || harris_variant > OF_VAR_HARRIS_SEMI_SEP)
        return fail(OF_ERR_ARG, "harris_variant out of range");
    if (harris_variant > OF_VAR_HARRIS_BASELINE && fast_variant != OF_VAR_FAST_SM_BINARY)
        return fail(OF_ERR_ARG, "sep / para_sep / semi_sep Harris run fused after sm_binary FAST");
    if (!img || !out_count || (capacity > 0 && !out_points) || capacity < 0 || capacity > INT32_MAX)
        return fail(OF_ERR_ARG, "null pointer or bad capacity");
    if (w < 1 || h < 1 || pitch < w || fast_t < 1 || fast_t > 255 || border < 4)
        return fail(OF_ERR_ARG, "bad image size, pitch, threshold or border");
    int64_t knum = 0, kden = 1;
    if (!ofh::k_fraction(harris_k, &knum, &kden)) return fail(OF_ERR_ARG, "harris_k not representable");
    int dev = 0, n_sms = 0;
    OF_CK(cudaGetDevice(&dev));
    OF_CK(cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev));
    const cudaStream_t st = (cudaStream_t)stream;
    OF_CK(cudaMemsetAsync(out_count, 0, sizeof(int32_t), st));
    launch_variant(fast_variant, harris_variant, img, w, h, pitch, fast_t, border, knum, kden, out_points, out_count,
                   (int)capacity, n_sms, stream);
    OF_CK(cudaGetLastError());
    return OF_OK;
}

int64_t of_batch_bytes(const of_params* p, const int32_t* ws, const int32_t* hs, int n_frames,
                       int levels, float scale, int n_features) {
    if (!p || !ws || !hs || n_frames < 1 || levels < 1 || levels > 16 || !(scale > 1.0f) || n_features < 0)
        return fail(OF_ERR_ARG, "bad arguments");
    Settings s{};
    s.levels = levels;
    s.scale = scale;
    s.n_features = n_features;
    s.border = p->border ? p->border : 19;
    s.cell = p->cell ? p->cell : 30;
    if (s.cell < 8 || s.border < 4) return fail(OF_ERR_ARG, "bad border/cell");
    std::vector<FrameKey> fr(n_frames);
    for (int i = 0; i < n_frames; ++i) {
        if (ws[i] < 1 || hs[i] < 1) return fail(OF_ERR_ARG, "bad frame size");
        fr[i] = FrameKey{ws[i], hs[i], (int)align_up(ws[i], 16), true};
    }
    return (int64_t)make_layout(fr, s, -1).total;
}

int of_detect_learned(of_handle* H, const of_frame* frames, int n_frames, int levels, float scale, int fast_t,
                      float harris_k, int n_features, of_tcnn* net, float threshold, float min_confidence,
                      int dilate, of_keypoint* out_kpts, int32_t* out_counts, int32_t* stats) {
    if (!H) return fail(OF_ERR_ARG, "null handle");
    if (!net) return fail(OF_ERR_ARG, "null network");
    if (!(threshold <= 1.0f) || !(min_confidence >= 0.0f && min_confidence <= 1.0f) || (dilate != 0 && dilate != 1))
        return fail(OF_ERR_ARG, "threshold <= 1, 0 <= min_confidence <= 1, dilate 0/1");
    DeviceGuard dg(H->device);
    Plan* P = nullptr;
    int rc = prepare_batch(H, frames, n_frames, levels, scale, fast_t, harris_k, n_features, out_kpts,
                           out_counts, &P);
    if (rc != OF_OK) return rc;
    rc = ensure_learned(P);
    if (rc == OF_OK) rc = set_pmask(H, P, true);
    if (rc != OF_OK) return rc;
    cudaStream_t st = H->stream;
    const int n_list = (int)P->det_list.size();
    const int n_tiles = P->ptile_prefix[n_list];
    int32_t* d_stats = reinterpret_cast<int32_t*>(P->lbuf + P->off_stats);
    const int32_t* d_pp = reinterpret_cast<const int32_t*>(P->lbuf + P->off_pp);
    float* d_logit = reinterpret_cast<float*>(P->lbuf + P->off_logit);
    OF_CK(cudaMemsetAsync(d_stats, 0, 4 * sizeof(int32_t), st));
    if (n_features == 0) OF_CK(cudaMemsetAsync(out_counts, 0, sizeof(int32_t) * n_frames, st));
    OF_CK(cudaGraphLaunch(P->stage_exec[0], st));  // pyramid
    rc = tcnn_forward_tiles(net, P->d_img(), P->d_dl(), d_pp, n_list, n_tiles, P->s.border, d_logit, st);
    if (rc == OF_OK)
        rc = launch_propose(P->d_img(), P->d_dl(), d_pp, n_list, d_logit, P->lbuf + P->off_pos,
                            P->lbuf + P->off_mask, threshold, min_confidence, dilate, d_stats, st);
    if (rc != OF_OK) return rc;
    for (int k = 1; k < kStages; ++k) {
        if (k == 2) {
            learned_flag_pass(H, P, st);
            OF_CK(cudaGetLastError());
        }
        OF_CK(cudaGraphLaunch(P->stage_exec[k], st));
    }
    H->last = P;
    if (stats) {
        OF_CK(cudaMemcpyAsync(H->h_count + 4, d_stats, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        OF_CK(cudaStreamSynchronize(st));
        std::memcpy(stats, H->h_count + 4, 3 * sizeof(int32_t));
    }
    return OF_OK;
}

int of_extract_tiles(of_handle* H, int frame, int level, uint8_t* dst, int64_t cap_tiles, int32_t* grid) {
    if (!H) return fail(OF_ERR_ARG, "null handle");
    Plan* P = H->last;
    if (!P) return fail(OF_ERR_ARG, "no detect call to extract from");
    const int nl = P->s.levels;
    if (frame < 0 || frame >= (int)P->frames.size() || level < 0 || level >= nl)
        return fail(OF_ERR_ARG, "frame/level out of range");
    const int ii = frame * nl + level;
    const Img& I = P->h_img[ii];
    const int n = 4 * I.tiles_x * I.tiles_y;
    if (grid) {
        grid[0] = 4 * I.tiles_x;
        grid[1] = I.tiles_y;
    }
    if (!dst || n == 0) return n;
    if (cap_tiles < n) return fail(OF_ERR_ARG, "dst too small");
    DeviceGuard dg(H->device);
    const int rc = launch_extract(P->d_img(), ii, P->s.border, dst, n, H->stream);
    if (rc != OF_OK) return rc;
    OF_CK(cudaStreamSynchronize(H->stream));
    return n;
}

int of_time_stages(of_handle* H, void* const* events) {
    if (!H || !events) return fail(OF_ERR_ARG, "null argument");
    for (int i = 0; i <= kStages; ++i) {
        if (!events[i]) return fail(OF_ERR_ARG, "null event");
        H->stage_ev[i] = (cudaEvent_t)events[i];
    }
    H->stage_timing = true;
    return OF_OK;
}

int of_detect(of_handle* H, const uint8_t* img, int w, int h_px, int pitch, int levels,
              float scale, int fast_t, float harris_k, int n_features, of_keypoint* out_kpts) {
    if (!H) return fail(OF_ERR_ARG, "null handle");
    of_frame F{img, w, h_px, pitch};
    const int rc = run_batch(H, &F, 1, levels, scale, fast_t, harris_k, n_features, out_kpts,
                             H->d_counts);
    if (rc != OF_OK) return rc;
    DeviceGuard dg(H->device);
    OF_CK(cudaMemcpyAsync(H->h_count, H->d_counts, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost,
                          H->stream));
    OF_CK(cudaStreamSynchronize(H->stream));
    if (H->h_count[4] != 0) {
        OF_CK(cudaMemset(H->d_counts + 4, 0, sizeof(int32_t)));
        return fail(OF_ERR_TIMEOUT, "a device-side wait expired");
    }
    return H->h_count[0];
}

int of_sync(of_handle* H) {
    if (!H) return fail(OF_ERR_ARG, "null handle");
    DeviceGuard dg(H->device);
    OF_CK(cudaMemcpyAsync(H->h_count + 4, H->d_counts + 4, sizeof(int32_t), cudaMemcpyDeviceToHost,
                          H->stream));
    OF_CK(cudaStreamSynchronize(H->stream));
    if (H->h_count[4] != 0) {
        OF_CK(cudaMemset(H->d_counts + 4, 0, sizeof(int32_t)));
        return fail(OF_ERR_TIMEOUT, "a device-side wait expired");
    }
    return OF_OK;
}

int of_test_timeout(of_handle* H, int64_t limit_us) {
    if (!H || limit_us < 1 || limit_us > 10000000) return fail(OF_ERR_ARG, "limit_us must be 1..1e7");
    DeviceGuard dg(H->device);
    // Waits on a word of the handle's own block that nothing sets.
    launch_wait_test(H->d_counts + 6, H->d_counts + 4, (uint64_t)limit_us * 1000ull, H->stream);
    OF_CK(cudaGetLastError());
    return of_sync(H);
}

int64_t of_inspect(of_handle* H, int what, int frame, int level, void* dst, int64_t dst_bytes,
                   int32_t* dims) {
    if (!H) return fail(OF_ERR_ARG, "null handle");
    Plan* P = H->last;
    if (!P) return fail(OF_ERR_ARG, "no detect call to inspect");
    const int nl = P->s.levels;
    if (frame < 0 || frame >= (int)P->frames.size() || level < 0 || level >= nl)
        return fail(OF_ERR_ARG, "frame/level out of range");
    DeviceGuard dg(H->device);
    const Img& I = P->h_img[frame * nl + level];
    const Settings& s = P->s;
    int32_t d4[4] = {I.w, I.h, 0, 0};
    int64_t bytes = 0;
    int lj = -1;  // position of the image in the detect list (learned buffers)
    if (what == OF_BUF_LEVEL || what == OF_BUF_SCORE) {
        bytes = (int64_t)I.w * I.h;
    } else if (what == OF_BUF_CELLT) {
        d4[2] = I.ncx;
        d4[3] = I.ncy;
        bytes = (int64_t)I.ncx * I.ncy;
    } else if (what == OF_BUF_PMASK || what == OF_BUF_LOGIT) {
        if (!P->lbuf || !P->pmask_on) return fail(OF_ERR_ARG, "the last call was not of_detect_learned");
        const int ii = frame * nl + level;
        for (size_t j = 0; j < P->det_list.size(); ++j)
            if (P->det_list[j] == ii) {
                lj = (int)j;
                break;
            }
        d4[0] = 4 * I.tiles_x;
        d4[1] = I.tiles_y;
        if (lj < 0) d4[0] = d4[1] = 0;  // no detect region: no tiles
        bytes = (int64_t)d4[0] * d4[1] * (what == OF_BUF_LOGIT ? (int64_t)sizeof(float) : 1);
    } else if (what == OF_BUF_CAND) {
        int32_t n = 0;
        OF_CK(cudaStreamSynchronize(H->stream));
        OF_CK(cudaMemcpy(&n, I.ctr, sizeof(int32_t), cudaMemcpyDeviceToHost));
        n = std::min(n, I.cand_cap);
        d4[2] = n;
        bytes = 16 * (int64_t)n;
    } else {
        return fail(OF_ERR_ARG, "unknown buffer");
    }
    if (dims) std::memcpy(dims, d4, sizeof(d4));
    if (!dst || bytes == 0) return bytes;
    if (dst_bytes < bytes) return fail(OF_ERR_ARG, "dst too small");
    uint8_t* d = static_cast<uint8_t*>(dst);
    cudaStream_t st = H->stream;
    if (what == OF_BUF_LEVEL) {
        OF_CK(cudaMemcpy2DAsync(d, I.w, I.img, I.pitch, I.w, I.h, cudaMemcpyDeviceToDevice, st));
    } else if (what == OF_BUF_SCORE) {
        OF_CK(cudaMemsetAsync(d, 0, bytes, st));
        const int rw = I.w - 2 * s.border, rh = I.h - 2 * s.border;
        if (rw > 0 && rh > 0 && I.score)
            OF_CK(cudaMemcpy2DAsync(d + (size_t)s.border * I.w + s.border, I.w,
                                    I.score + (size_t)s.border * I.spitch + s.border, I.spitch, rw,
                                    rh, cudaMemcpyDeviceToDevice, st));
        // The maps hold s - (t_lo - 1); the thresholds may still be pending (NMS applies them itself).
        ofk::launch_inspect_score_final(P->d_img(), frame * nl + level, d, I.w, I.h, s.t_hi, s.t_lo, s.border,
                                        s.cell, st);
        OF_CK(cudaGetLastError());
    } else if (what == OF_BUF_CELLT) {
        ofk::launch_inspect_cells(P->d_img(), frame * nl + level, s.t_hi, s.t_lo, d, st);
        OF_CK(cudaGetLastError());
    } else if (what == OF_BUF_PMASK) {
        OF_CK(cudaMemcpyAsync(d, P->lbuf + P->off_mask + P->ptile_prefix[lj], bytes, cudaMemcpyDeviceToDevice, st));
    } else if (what == OF_BUF_LOGIT) {
        OF_CK(cudaMemcpyAsync(d, P->lbuf + P->off_logit + sizeof(float) * P->ptile_prefix[lj], bytes,
                              cudaMemcpyDeviceToDevice, st));
    } else {
        ofk::launch_inspect_cands(P->d_img(), frame * nl + level, (int)(bytes / 16), d, st);
        OF_CK(cudaGetLastError());
    }
    OF_CK(cudaStreamSynchronize(st));
    return bytes;
}

}  // extern "C"
