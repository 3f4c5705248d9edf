// Single-level detection that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured (allocation calls are illegal in a capture), real-time loops
// that must not touch the allocator after start-up, and plug-in hosts that own
// every device allocation and hand out only the buffers they manage.  For
// them, of_detect_level_noalloc runs FAST score, cell fallback, NMS, Harris,
// top-N and orientation on one pyramid level using the same kernels as
// of_detect, with all intermediate buffers carved out of one file-scope
// device array of OF_NOALLOC_SCRATCH_BYTES.  The caller passes the image and
// the output buffers.
//
// Notes for users:
//   - The array is a static part of this library: every GPU that loads it
//     holds these bytes until the process exits.
//   - Host code cannot use the array's name as a device address.  The first
//     call on each device looks the address up with cudaGetSymbolAddress
//     (and raises the top-N kernel's shared-memory limit) with that device
//     current; make that first call before any stream capture begins.  The
//     address is cached per device for the life of the process: a device
//     reset (cudaDeviceReset, primary-context teardown) is not supported
//     after it.
//   - Every call shares the array and it keeps the last call's contents; each
//     call clears the counters and flags it needs.  Calls whose work overlaps
//     on the GPU (different streams, or different host threads) race on the
//     array: serialise them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "of_internal.h"
#include "of_plan.h"
#include "ofast.h"

namespace ofk {
void set_select_smem_limit(int bytes);
void set_last_error(const std::string& msg);
int encode_u8_map(CUtensorMap* m, const void* base, int w, int h, int pitch, int box_w, int box_h);
int fast_blocks_per_sm();
int nms_blocks_per_sm();
}
using namespace ofk;

namespace {

static __device__ __align__(256) uint8_t g_noalloc_scratch[OF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
uint8_t* g_scratch_addr[kMaxDevices] = {};
int g_grid_fast[kMaxDevices] = {}, g_grid_nms[kMaxDevices] = {};
std::mutex g_setup_mutex;

int na_fail(int code, const std::string& msg) {
    set_last_error(msg);
    return code;
}

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Writes the descriptors and tensor maps into the scratch and clears what
// must start at zero.
__global__ void k_noalloc_setup(Img img, Call call, CUtensorMap img_map, CUtensorMap score_map,
                                Img* d_img, Call* d_call, CUtensorMap* d_maps, int32_t* d_list,
                                int32_t* zero, int zero_words, int32_t* out_count) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d_img = img;
        *d_call = call;
        d_maps[0] = img_map;
        d_maps[1] = score_map;
        asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
        d_list[0] = 0;  // the one image
        d_list[1] = 0;  // its first tile
        if (call.n_features == 0) *out_count = 0;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < zero_words; i += gridDim.x * blockDim.x)
        zero[i] = 0;
}

int device_scratch(uint8_t** out, int* grid_fast, int* grid_nms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(OF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(OF_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(OF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        set_select_smem_limit(select_smem_bytes(8192));
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        g_grid_fast[dev] = sms * fast_blocks_per_sm();
        g_grid_nms[dev] = sms * nms_blocks_per_sm();
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return na_fail(OF_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<uint8_t*>(p);
    }
    *out = g_scratch_addr[dev];
    *grid_fast = g_grid_fast[dev];
    *grid_nms = g_grid_nms[dev];
    return OF_OK;
}

}  // namespace

extern "C" int of_detect_level_noalloc(const uint8_t* img, int w, int h, int pitch, int fast_t,
                                       int fast_t_lo, float harris_k, int n_features,
                                       of_keypoint* out_kpts, int32_t* out_count, void* stream) {
    const int border = 19, cell = 30, radius = 15;
    if (!img || !out_count || (n_features > 0 && !out_kpts))
        return na_fail(OF_ERR_ARG, "null pointer");
    if (w < 1 || h < 1 || pitch < w || w > 65535 || h > 65535) return na_fail(OF_ERR_ARG, "bad frame size");
    if (fast_t < 1 || fast_t > 255 || fast_t_lo < 0 || fast_t_lo > 255)
        return na_fail(OF_ERR_ARG, "threshold out of range");
    if (n_features < 0 || n_features > 8192) return na_fail(OF_ERR_ARG, "n_features must be 0..8192");
    int64_t knum = 0, kden = 1;
    if (!ofh::k_fraction(harris_k, &knum, &kden))
        return na_fail(OF_ERR_ARG, "harris_k must be in [0, 0.25] with a reduced denominator <= 3000");
    const int t_lo = (fast_t_lo > 0 && fast_t_lo < fast_t) ? fast_t_lo : fast_t;
    cudaStream_t st = (cudaStream_t)stream;

    // Layout inside the static array.
    const int rw = w - 2 * border, rh = h - 2 * border;
    const bool det = rw > 0 && rh > 0;
    const bool copy = ((uintptr_t)img % 16 != 0) || (pitch % 16 != 0);
    const int spitch = (int)up(w, 16);
    const int ncx = det ? (rw + cell - 1) / cell : 0, ncy = det ? (rh + cell - 1) / cell : 0;
    const int cap = det ? ((rw + 1) / 2) * ((rh + 1) / 2) : 0;
    const int quota = det ? n_features : 0;
    size_t off = 0;
    const size_t o_img = off;
    off = up(off + sizeof(Img), 256);
    const size_t o_call = off;
    off = up(off + sizeof(Call), 256);
    const size_t o_maps = off;
    off = up(off + 2 * sizeof(CUtensorMap), 256);
    const size_t o_list = off;
    off = up(off + 2 * sizeof(int32_t), 256);
    const size_t o_zero = off;  // counters (4), status (4), then cell flags
    off = up(off + 8 * sizeof(int32_t) + sizeof(uint32_t) * (size_t)ncx * ncy, 256);
    const size_t zero_bytes = off - o_zero;
    const size_t o_copy = off;
    if (copy) off = up(off + (size_t)spitch * h, 256);
    const size_t o_score = off;
    if (det) off = up(off + (size_t)spitch * h, 256);
    const size_t o_ckey = off;
    off = up(off + sizeof(uint64_t) * (size_t)cap, 256);
    const size_t o_cyx = off;
    off = up(off + sizeof(uint32_t) * (size_t)cap, 256);
    const size_t o_kkey = off;
    off = up(off + sizeof(uint64_t) * (size_t)(quota > 0 ? quota : 1), 256);
    const size_t o_kyx = off;
    off = up(off + sizeof(uint32_t) * (size_t)(quota > 0 ? quota : 1), 256);
    if (off > (size_t)OF_NOALLOC_SCRATCH_BYTES)
        return na_fail(OF_ERR_TOO_LARGE, "frame needs " + std::to_string(off) +
                                             " bytes of scratch; the static array holds " +
                                             std::to_string((size_t)OF_NOALLOC_SCRATCH_BYTES));

    uint8_t* S = nullptr;
    int grid_fast = 0, grid_nms = 0;
    const int rc = device_scratch(&S, &grid_fast, &grid_nms);
    if (rc != OF_OK) return rc;

    Img I;
    std::memset(&I, 0, sizeof(I));
    I.img = copy ? S + o_copy : img;
    I.w = w;
    I.h = h;
    I.pitch = copy ? spitch : pitch;
    I.spitch = spitch;
    I.ncx = ncx;
    I.ncy = ncy;
    I.cand_cap = cap;
    I.quota = quota;
    I.ctr = reinterpret_cast<int32_t*>(S + o_zero);
    I.lscale = 1.0;
    if (det) {
        I.cell = reinterpret_cast<uint32_t*>(S + o_zero + 8 * sizeof(int32_t));
        I.score = S + o_score;
        I.ckey = reinterpret_cast<uint64_t*>(S + o_ckey);
        I.cyx = reinterpret_cast<uint32_t*>(S + o_cyx);
        I.kkey = reinterpret_cast<uint64_t*>(S + o_kkey);
        I.kyx = reinterpret_cast<uint32_t*>(S + o_kyx);
        I.tile_x0 = border & ~15;
        I.tiles_x = (w - border - I.tile_x0 + TILE_W - 1) / TILE_W;
        I.tiles_y = (rh + TILE_H - 1) / TILE_H;
    }
    Call Cl;
    std::memset(&Cl, 0, sizeof(Cl));
    Cl.out = out_kpts;
    Cl.counts = out_count;
    Cl.status = reinterpret_cast<int32_t*>(S + o_zero) + 4;  // a timeout shows up as *out_count < 0
    Cl.knum = knum;
    Cl.kden = kden;
    Cl.resp_scale = ofh::response_scale(kden);
    Cl.n_frames = 1;
    Cl.levels = 1;
    Cl.n_features = n_features;
    Cl.t_hi = fast_t;
    Cl.t_lo = t_lo;
    Cl.border = border;
    Cl.cell = cell;
    Cl.radius = radius;
    Cl.n_img = 1;
    Cl.total_slots = n_features;

    CUtensorMap maps[2];
    int mrc = encode_u8_map(&maps[0], I.img, w, h, I.pitch, SROW, IMG_BOX_ROWS);
    if (mrc == OF_OK) mrc = encode_u8_map(&maps[1], det ? I.score : nullptr, w, h, spitch, SROW, SCORE_BOX_ROWS);
    if (mrc != OF_OK) return mrc;
    Img* d_img = reinterpret_cast<Img*>(S + o_img);
    Call* d_call = reinterpret_cast<Call*>(S + o_call);
    CUtensorMap* d_maps = reinterpret_cast<CUtensorMap*>(S + o_maps);
    int32_t* d_list = reinterpret_cast<int32_t*>(S + o_list);
    const int zero_words = (int)(zero_bytes / sizeof(int32_t));
    k_noalloc_setup<<<4, 256, 0, st>>>(I, Cl, maps[0], maps[1], d_img, d_call, d_maps, d_list,
                                       reinterpret_cast<int32_t*>(S + o_zero), zero_words, out_count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(OF_ERR_CUDA, std::string("setup kernel: ") + cudaGetErrorString(e));
    if (copy) {
        e = cudaMemcpy2DAsync(S + o_copy, spitch, img, pitch, w, h, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return na_fail(OF_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
    }
    const int tiles = I.tiles_x * I.tiles_y;
    launch_fast(d_img, d_list, d_list + 1, 1, tiles, d_maps, d_call, fast_t, t_lo, border, cell, grid_fast, 0, st);
    launch_nms_harris(d_img, d_list, d_list + 1, 1, tiles, d_maps, d_maps + 1, d_call, fast_t, t_lo, border, cell,
                      grid_nms, 0, st);
    launch_select(d_img, 1, d_call, quota > 0 ? quota : 1, st);
    launch_orient(d_img, 1, d_call, n_features, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(OF_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return OF_OK;
}
