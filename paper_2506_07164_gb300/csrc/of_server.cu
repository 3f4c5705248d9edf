// Serving loop with continuous batching (host runtime, C++).
//
// A server owns `slots` engines.  Each slot is one detector handle with its
// own CUDA stream, a share of the device-memory budget (scratch arena +
// device input frames + outputs) and pinned host staging.  Requests (host
// frames) are queued on submit.  A dispatcher thread:
//   - completes slots whose batch finished (event query), copying each
//     request's keypoints into its result and freeing the slot's memory;
//   - whenever a slot is free, admits the oldest queued request and every
//     later queued request of the same resolution, in arrival order, while the
//     batch still fits the slot's scratch and input bytes and max_batch;
//   - launches the batch asynchronously on the slot's stream: one copy per
//     frame from its pinned request buffer to the device, the cached batch
//     graph, device -> pinned results, an event.
// A submitting thread copies its frame straight into a pinned buffer from the
// server's pool (reused after the frame's batch completes; grown up to a cap,
// beyond which a request falls back to pageable memory and the slot's pinned
// staging), so the host copies run on the callers' threads, not on the
// dispatcher.
// Requests that arrive while other batches are on the GPU are admitted as
// soon as a slot and its memory free up, and batches on different slots run
// concurrently on the device.  A batch's pyramids stay resident in its
// slot's arena until the slot takes its next batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ofast.h"

namespace ofk {
void set_last_error(const std::string& msg);
}

namespace {

int sfail(int code, const std::string& msg) {
    ofk::set_last_error(msg);
    return code;
}

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t up16(size_t x) { return (x + 15) / 16 * 16; }

struct Request {
    int64_t id = 0, tag = 0;
    int w = 0, h = 0;
    uint8_t* pin = nullptr;       // pinned pool buffer holding the packed rows (w bytes each), or null:
    size_t pin_cap = 0;
    std::vector<uint8_t> pixels;  // the packed rows in pageable memory
    double t_submit = 0, t_launch = 0;
};

struct Done {
    of_server_result r;
    std::vector<of_keypoint> kpts;
};

struct Slot {
    of_handle* H = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t* d_in = nullptr;
    uint8_t* h_in = nullptr;
    size_t in_cap = 0;
    of_keypoint* d_out = nullptr;
    int32_t* d_counts = nullptr;
    of_keypoint* h_out = nullptr;
    int32_t* h_counts = nullptr;
    int64_t arena_cap = 0;
    std::vector<Request> batch;
    bool busy = false;
};

}  // namespace

struct of_server {
    of_server_params p{};
    of_params hp{};
    int device = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_in, cv_out;
    std::deque<Request> queue;
    std::deque<Done> done;
    std::thread worker;
    std::atomic<bool> stop{false};
    int64_t next_id = 0;
    of_server_stats st{};
    std::string fatal;
    // Pinned request buffers: free list (capacity, buffer) and bytes allocated.
    std::mutex pool_mu;
    std::vector<std::pair<size_t, uint8_t*>> pool_free;
    size_t pool_bytes = 0, pool_cap = 0;
};

namespace {

int64_t batch_bytes(of_server* S, int w, int h, int n) {
    std::vector<int32_t> ws(n, w), hs(n, h);
    return of_batch_bytes(&S->hp, ws.data(), hs.data(), n, S->p.levels, S->p.scale, S->p.n_features);
}

// A pinned buffer of at least `need` bytes from the pool (the smallest that
// fits), a new one while the pool is under its cap, else null.
uint8_t* pool_take(of_server* S, size_t need, size_t* cap) {
    {
        std::lock_guard<std::mutex> lk(S->pool_mu);
        int best = -1;
        for (int i = 0; i < (int)S->pool_free.size(); ++i)
            if (S->pool_free[i].first >= need && (best < 0 || S->pool_free[i].first < S->pool_free[best].first))
                best = i;
        if (best >= 0) {
            uint8_t* b = S->pool_free[best].second;
            *cap = S->pool_free[best].first;
            S->pool_free.erase(S->pool_free.begin() + best);
            return b;
        }
        if (S->pool_bytes + need > S->pool_cap) return nullptr;
        S->pool_bytes += need;
    }
    void* b = nullptr;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != S->device) cudaSetDevice(S->device);
    const cudaError_t e = cudaHostAlloc(&b, need, cudaHostAllocPortable);
    if (prev >= 0 && prev != S->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(S->pool_mu);
        S->pool_bytes -= need;
        return nullptr;
    }
    *cap = need;
    return static_cast<uint8_t*>(b);
}

void pool_give(of_server* S, Request& rq) {
    if (!rq.pin) return;
    std::lock_guard<std::mutex> lk(S->pool_mu);
    S->pool_free.emplace_back(rq.pin_cap, rq.pin);
    rq.pin = nullptr;
    rq.pin_cap = 0;
}

// Completes every finished slot.  Called by the dispatcher only.
void reap(of_server* S) {
    for (Slot& sl : S->slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        const double t = now_s();
        int sync_rc = (q == cudaSuccess) ? OF_OK : OF_ERR_CUDA;
        for (size_t i = 0; i < sl.batch.size() && sync_rc == OF_OK; ++i)
            if (sl.h_counts[i] == OF_ERR_TIMEOUT) sync_rc = of_sync(sl.H);  // reports and clears it
        std::vector<Done> out;
        const int nf = S->p.n_features;
        for (size_t i = 0; i < sl.batch.size(); ++i) {
            const Request& rq = sl.batch[i];
            Done d;
            d.r.id = rq.id;
            d.r.tag = rq.tag;
            d.r.w = rq.w;
            d.r.h = rq.h;
            d.r.t_submit = rq.t_submit;
            d.r.t_launch = rq.t_launch;
            d.r.t_done = t;
            d.r.batch_frames = (int32_t)sl.batch.size();
            int32_t c = (sync_rc == OF_OK) ? sl.h_counts[i] : sync_rc;
            if (c > nf) c = OF_ERR_CUDA;
            d.r.count = c;
            if (c > 0) d.kpts.assign(sl.h_out + i * (size_t)nf, sl.h_out + i * (size_t)nf + c);
            out.push_back(std::move(d));
        }
        for (Request& rq : sl.batch) pool_give(S, rq);  // the batch's copies are done
        sl.batch.clear();
        sl.busy = false;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (auto& d : out) {
                S->done.push_back(std::move(d));
                S->st.completed++;
            }
            S->st.in_flight_batches--;
        }
        S->cv_out.notify_all();
    }
}

// Forms one batch for a free slot from the queue (lock held).  Returns the
// number of requests moved into the slot.
int admit(of_server* S, Slot& sl) {
    if (S->queue.empty()) return 0;
    const int w = S->queue.front().w, h = S->queue.front().h;
    const size_t fbytes = up16(w) * (size_t)h;
    int n = 0;
    for (auto it = S->queue.begin(); it != S->queue.end() && n < S->p.max_batch;) {
        if (it->w != w || it->h != h) {
            ++it;
            continue;
        }
        const int64_t need = batch_bytes(S, w, h, n + 1);
        if (need < 0 || need > sl.arena_cap || (size_t)(n + 1) * fbytes > sl.in_cap) break;
        sl.batch.push_back(std::move(*it));
        it = S->queue.erase(it);
        ++n;
    }
    return n;
}

int launch(of_server* S, Slot& sl) {
    const int w = sl.batch[0].w, h = sl.batch[0].h;
    const int pitch = (int)up16(w);
    const size_t fbytes = (size_t)pitch * h;
    const int n = (int)sl.batch.size();
    std::vector<of_frame> frames(n);
    const double t = now_s();
    for (int i = 0; i < n; ++i) {
        Request& rq = sl.batch[i];
        rq.t_launch = t;
        const uint8_t* src = rq.pin;
        size_t spitch = (size_t)w;
        if (!src) {  // pageable request: through the slot's pinned staging
            uint8_t* dst = sl.h_in + i * fbytes;
            for (int y = 0; y < h; ++y) std::memcpy(dst + (size_t)y * pitch, rq.pixels.data() + (size_t)y * w, w);
            std::vector<uint8_t>().swap(rq.pixels);
            src = dst;
            spitch = (size_t)pitch;
        }
        if (cudaMemcpy2DAsync(sl.d_in + i * fbytes, pitch, src, spitch, w, h, cudaMemcpyHostToDevice, sl.stream) !=
            cudaSuccess)
            return OF_ERR_CUDA;
        frames[i] = of_frame{sl.d_in + i * fbytes, w, h, pitch};
    }
    const int rc = of_detect_batch(sl.H, frames.data(), n, S->p.levels, S->p.scale, S->p.fast_t,
                                   S->p.harris_k, S->p.n_features, sl.d_out, sl.d_counts);
    if (rc != OF_OK) return rc;
    if (cudaMemcpyAsync(sl.h_counts, sl.d_counts, n * sizeof(int32_t), cudaMemcpyDeviceToHost, sl.stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)n * S->p.n_features * sizeof(of_keypoint),
                        cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
        cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
        return OF_ERR_CUDA;
    sl.busy = true;
    return OF_OK;
}

void dispatcher(of_server* S) {
    cudaSetDevice(S->device);
    while (!S->stop.load()) {
        reap(S);
        bool launched = false;
        for (Slot& sl : S->slots) {
            if (sl.busy) continue;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                if (admit(S, sl) == 0) break;
                S->st.batches++;
                S->st.in_flight_batches++;
                S->st.frames_launched += (int64_t)sl.batch.size();
            }
            const int rc = launch(S, sl);
            if (rc != OF_OK) {
                // Report every request of the failed batch (its copies queued so far finish first).
                cudaStreamSynchronize(sl.stream);
                for (Request& rq : sl.batch) pool_give(S, rq);
                std::lock_guard<std::mutex> lk(S->mu);
                for (auto& rq : sl.batch) {
                    Done d;
                    d.r.id = rq.id;
                    d.r.tag = rq.tag;
                    d.r.w = rq.w;
                    d.r.h = rq.h;
                    d.r.t_submit = rq.t_submit;
                    d.r.t_launch = d.r.t_done = now_s();
                    d.r.count = rc;
                    S->done.push_back(std::move(d));
                    S->st.completed++;
                }
                sl.batch.clear();
                S->st.in_flight_batches--;
                S->cv_out.notify_all();
                continue;
            }
            launched = true;
        }
        if (!launched) {
            bool any_busy = false;
            for (Slot& sl : S->slots) any_busy |= sl.busy;
            std::unique_lock<std::mutex> lk(S->mu);
            if (any_busy)
                S->cv_in.wait_for(lk, std::chrono::microseconds(20));
            else
                S->cv_in.wait_for(lk, std::chrono::milliseconds(5),
                                  [&] { return !S->queue.empty() || S->stop.load(); });
        }
    }
}

void free_slot(Slot& sl) {
    if (sl.H) of_destroy(sl.H);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.d_in) cudaFree(sl.d_in);
    if (sl.d_out) cudaFree(sl.d_out);
    if (sl.d_counts) cudaFree(sl.d_counts);
    if (sl.h_in) cudaFreeHost(sl.h_in);
    if (sl.h_out) cudaFreeHost(sl.h_out);
    if (sl.h_counts) cudaFreeHost(sl.h_counts);
    sl = Slot();
}

}  // namespace

extern "C" {

of_server* of_server_create(const of_server_params* pin) {
    if (!pin) {
        sfail(OF_ERR_ARG, "null params");
        return nullptr;
    }
    of_server_params p = *pin;
    if (p.levels == 0) p.levels = 8;
    if (p.scale == 0.0f) p.scale = 1.2f;
    if (p.fast_t == 0) p.fast_t = 20;
    if (p.harris_k == 0.0f) p.harris_k = 0.04f;
    if (p.n_features == 0) p.n_features = 1000;
    if (p.slots == 0) p.slots = 3;
    if (p.max_batch == 0) p.max_batch = 8;
    if (p.max_w < 1 || p.max_h < 1 || p.slots < 1 || p.slots > 16 || p.max_batch < 1 ||
        p.max_batch > 256 || p.memory_budget <= 0 || p.levels < 1 || p.levels > 16 ||
        p.n_features < 1 || p.n_features > 8192) {
        sfail(OF_ERR_ARG, "invalid of_server_params");
        return nullptr;
    }
    of_server* S = new of_server();
    S->p = p;
    cudaGetDevice(&S->device);
    of_params& hp = S->hp;
    hp.max_w = p.max_w;
    hp.max_h = p.max_h;
    hp.max_levels = p.levels;
    hp.max_features = p.n_features;
    hp.max_batch = p.max_batch;
    hp.min_scale = p.scale;
    hp.fast_t_lo = p.fast_t_lo;
    hp.border = p.border;
    hp.cell = p.cell;
    hp.orient_radius = p.orient_radius;
    // Per slot: inputs (max_batch frames, at least one max-size frame), outputs, arena.
    const int64_t per_slot = p.memory_budget / p.slots;
    const size_t max_frame = up16(p.max_w) * (size_t)p.max_h;
    const size_t out_bytes = (size_t)p.max_batch * p.n_features * sizeof(of_keypoint) + 256;
    size_t in_cap = std::max(max_frame, (size_t)(per_slot / 10) / max_frame * max_frame);
    in_cap = std::min(in_cap, (size_t)p.max_batch * max_frame);
    const int32_t mw = p.max_w, mh = p.max_h;
    const int64_t one = of_batch_bytes(&hp, &mw, &mh, 1, p.levels, p.scale, p.n_features);
    const int64_t arena = per_slot - (int64_t)in_cap - (int64_t)out_bytes;
    if (one < 0 || arena < one) {
        sfail(OF_ERR_TOO_LARGE, "memory_budget too small for one " + std::to_string(p.max_w) + "x" +
                                    std::to_string(p.max_h) + " frame per slot (needs " +
                                    std::to_string(one + (int64_t)in_cap + (int64_t)out_bytes) + " bytes)");
        delete S;
        return nullptr;
    }
    hp.arena_bytes = arena;
    S->slots.resize(p.slots);
    for (Slot& sl : S->slots) {
        bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMalloc(&sl.d_in, in_cap) == cudaSuccess &&
                  cudaMallocHost(&sl.h_in, in_cap) == cudaSuccess &&
                  cudaMalloc(&sl.d_out, out_bytes) == cudaSuccess &&
                  cudaMalloc(&sl.d_counts, sizeof(int32_t) * p.max_batch) == cudaSuccess &&
                  cudaMallocHost(&sl.h_out, out_bytes) == cudaSuccess &&
                  cudaMallocHost(&sl.h_counts, sizeof(int32_t) * p.max_batch) == cudaSuccess;
        if (ok) {
            of_params q = hp;
            q.stream = sl.stream;
            sl.H = of_create(&q);
            ok = sl.H != nullptr;
        }
        if (!ok) {
            sfail(OF_ERR_CUDA, "server slot allocation failed");
            for (Slot& x : S->slots) free_slot(x);
            delete S;
            return nullptr;
        }
        sl.in_cap = in_cap;
        sl.arena_cap = arena;
    }
    // Pinned request buffers: enough for two full batches per slot, at most 2 GiB.
    S->pool_cap = std::min((size_t)2 << 30, (size_t)2 * p.slots * p.max_batch * (size_t)p.max_w * p.max_h);
    S->st.slot_arena_bytes = arena;
    S->st.slot_input_bytes = (int64_t)in_cap;
    S->worker = std::thread(dispatcher, S);
    return S;
}

void of_server_destroy(of_server* S) {
    if (!S) return;
    S->stop.store(true);
    S->cv_in.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Slot& sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        for (Request& rq : sl.batch) pool_give(S, rq);
        free_slot(sl);
    }
    for (Request& rq : S->queue) pool_give(S, rq);
    for (auto& b : S->pool_free) cudaFreeHost(b.second);
    S->pool_free.clear();
    delete S;
}

int64_t of_server_submit(of_server* S, const uint8_t* img, int w, int h, int pitch, int64_t tag) {
    if (!S || !img || w < 1 || h < 1 || pitch < w) return sfail(OF_ERR_ARG, "bad request");
    if (w > S->p.max_w || h > S->p.max_h) return sfail(OF_ERR_TOO_LARGE, "frame larger than max_w x max_h");
    Request rq;
    rq.tag = tag;
    rq.w = w;
    rq.h = h;
    const size_t need = (size_t)w * h;
    rq.pin = pool_take(S, need, &rq.pin_cap);
    uint8_t* dst = rq.pin;
    if (!dst) {
        rq.pixels.resize(need);
        dst = rq.pixels.data();
    }
    if (pitch == w) std::memcpy(dst, img, need);
    else
        for (int y = 0; y < h; ++y) std::memcpy(dst + (size_t)y * w, img + (size_t)y * pitch, w);
    rq.t_submit = now_s();
    int64_t id;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        id = rq.id = S->next_id++;
        S->queue.push_back(std::move(rq));
        S->st.submitted++;
    }
    S->cv_in.notify_one();
    return id;
}

int of_server_poll(of_server* S, of_server_result* results, of_keypoint* kpts, int max_results,
                   int wait_ms) {
    if (!S || !results || max_results < 1) return sfail(OF_ERR_ARG, "bad poll arguments");
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_ms > 0)
        S->cv_out.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
    int n = 0;
    while (n < max_results && !S->done.empty()) {
        Done& d = S->done.front();
        results[n] = d.r;
        if (kpts && d.r.count > 0)
            std::memcpy(kpts + (size_t)n * S->p.n_features, d.kpts.data(), sizeof(of_keypoint) * d.r.count);
        S->done.pop_front();
        ++n;
    }
    return n;
}

int of_server_stats_get(of_server* S, of_server_stats* out) {
    if (!S || !out) return sfail(OF_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->queued = (int64_t)S->queue.size();
    return OF_OK;
}

}  // extern "C"
