// serve.cu -- the serving loop of include/rmusic_serve.h: stream admission under an HBM budget,
// per-stream rings of device frame slots, continuous batching onto the FP32-batched path with
// several batches in flight on separate CUDA streams, and a completion queue with timestamps.
//
// Device memory, allocated once at creation: three arenas sharing one element index space of
// E pixel slots -- frames (4 B per slot, enough for float32 or uint16), derivative maps (4 B) and
// status maps (1 B) -- so a slot's frame, map and status sit at the same element offset and one
// descriptor offset addresses all three; plus one rmusic context (analytic-signal workspace) per
// batch slot. A RangeAllocator hands out the rings of admitted streams.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/rmusic.h"
#include "../../include/rmusic_serve.h"
#include "serve_arena.h"

using rmusic::RangeAllocator;

namespace {

constexpr uint64_t kSlotAlign = 64;  // element alignment of a slot (256 B in the frame arena)

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int32_t stream;
    int32_t slot;
    const void* h_in;
    float* h_out;
    uint8_t* h_status;
    uint64_t tag;
    double t_submit;
    double t_launch;
};

struct StreamState {
    bool open = false;
    bool closing = false;
    int32_t H = 0, W = 0, dtype = 0;
    uint64_t px = 0;
    uint64_t ring_off = 0;  // element offset of slot 0; slot k at ring_off + k * slot_stride
    uint64_t slot_stride = 0;
    uint64_t ring_units = 0;
    std::vector<uint8_t> busy;
    int32_t queued = 0;  // frames queued or in flight
};

struct BatchSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    rmusic_ctx* ctx = nullptr;
    bool busy = false;
    int status = RMUSIC_OK;
    std::vector<Request> reqs;
    std::vector<rmusic_frame_desc> descs;
};

}  // namespace

struct rmusic_server {
    rmusic_params params{};
    rmusic_serve_config cfg{};
    int device = 0;
    unsigned char* d_in = nullptr;
    float* d_out = nullptr;
    uint8_t* d_st = nullptr;
    uint64_t E = 0;  // pixel slots in the arenas
    uint64_t device_bytes = 0;
    RangeAllocator alloc;
    std::vector<StreamState> streams;
    std::deque<Request> pending;
    std::vector<BatchSlot> batches;
    std::deque<rmusic_completion> done;
    std::mutex mu;
    std::condition_variable cv_work;  // worker: new request, or stop
    std::condition_variable cv_done;  // pollers and closers: a frame finished
    std::thread worker;
    bool stop = false;
    rmusic_serve_stats st{};
};

namespace {

// Launch one batch from the pending queue on batch slot b (called with the lock held; the CUDA
// calls are asynchronous and do not block on the GPU).
void launch_batch(rmusic_server* s, BatchSlot& b) {
    b.reqs.clear();
    b.descs.clear();
    uint64_t px = 0;
    while (!s->pending.empty() && (int)b.reqs.size() < s->cfg.max_batch_frames) {
        const Request& r = s->pending.front();
        const StreamState& ss = s->streams[r.stream];
        if (!b.reqs.empty() && px + ss.px > s->cfg.max_batch_pixels) break;
        px += ss.px;
        b.reqs.push_back(r);
        s->pending.pop_front();
    }
    const double t = now_s();
    b.status = RMUSIC_OK;
    for (Request& r : b.reqs) {
        r.t_launch = t;
        const StreamState& ss = s->streams[r.stream];
        const uint64_t o = ss.ring_off + (uint64_t)r.slot * ss.slot_stride;
        const size_t esz = ss.dtype == RMUSIC_DTYPE_U16 ? 2 : 4;
        if (cudaMemcpyAsync(s->d_in + 4 * o, r.h_in, ss.px * esz, cudaMemcpyHostToDevice, b.stream) != cudaSuccess)
            b.status = RMUSIC_ECUDA;
        rmusic_frame_desc d;
        memset(&d, 0, sizeof(d));
        d.offset_bytes = 4 * o;
        d.height = ss.H;
        d.width = ss.W;
        d.dtype = ss.dtype;
        d.out_offset = o;
        b.descs.push_back(d);
    }
    if (b.status == RMUSIC_OK)
        b.status = rmusic_demodulate_frames(b.ctx, s->d_in, b.descs.data(), (int32_t)b.descs.size(), s->d_out,
                                            s->d_st, b.stream);
    for (const Request& r : b.reqs) {
        const StreamState& ss = s->streams[r.stream];
        const uint64_t o = ss.ring_off + (uint64_t)r.slot * ss.slot_stride;
        if (b.status == RMUSIC_OK &&
            cudaMemcpyAsync(r.h_out, s->d_out + o, ss.px * sizeof(float), cudaMemcpyDeviceToHost, b.stream) !=
                cudaSuccess)
            b.status = RMUSIC_ECUDA;
        if (b.status == RMUSIC_OK && r.h_status &&
            cudaMemcpyAsync(r.h_status, s->d_st + o, ss.px, cudaMemcpyDeviceToHost, b.stream) != cudaSuccess)
            b.status = RMUSIC_ECUDA;
    }
    cudaEventRecord(b.done, b.stream);
    b.busy = true;
    s->st.batches += 1;
}

// Retire a finished batch (lock held): completions, free ring slots.
void retire_batch(rmusic_server* s, BatchSlot& b) {
    const double t = now_s();
    for (const Request& r : b.reqs) {
        StreamState& ss = s->streams[r.stream];
        ss.busy[r.slot] = 0;
        ss.queued -= 1;
        rmusic_completion c;
        memset(&c, 0, sizeof(c));
        c.stream_id = r.stream;
        c.status = b.status;
        c.tag = r.tag;
        c.t_submit = r.t_submit;
        c.t_launch = r.t_launch;
        c.t_done = t;
        c.batch_frames = (int32_t)b.reqs.size();
        s->done.push_back(c);
        s->st.frames_done += 1;
        s->st.pixels_done += ss.px;
    }
    b.reqs.clear();
    b.busy = false;
}

void worker_main(rmusic_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        bool any_busy = false, retired = false;
        for (BatchSlot& b : s->batches) {
            if (!b.busy) continue;
            cudaError_t q = cudaEventQuery(b.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            if (q != cudaSuccess && b.status == RMUSIC_OK) b.status = RMUSIC_ECUDA;
            retire_batch(s, b);
            retired = true;
        }
        if (retired) s->cv_done.notify_all();
        for (BatchSlot& b : s->batches) {
            if (s->pending.empty()) break;
            if (b.busy) continue;
            launch_batch(s, b);
            any_busy = true;
        }
        if (s->stop && s->pending.empty() && !any_busy) break;
        if (any_busy) {
            // batches on the GPU: poll their events at a fine interval, wake early on new work
            s->cv_work.wait_for(lock, std::chrono::microseconds(50));
        } else {
            s->cv_work.wait(lock, [s] { return s->stop || !s->pending.empty(); });
        }
    }
}

bool config_ok(const rmusic_serve_config& c) {
    return c.max_streams >= 1 && c.max_streams <= 4096 && c.ring_depth >= 1 && c.ring_depth <= 64 &&
           c.max_batch_frames >= 1 && c.max_batch_frames <= 1024 && c.inflight_batches >= 1 &&
           c.inflight_batches <= 8 && c.max_batch_pixels >= 1;
}

void free_server(rmusic_server* s) {
    for (BatchSlot& b : s->batches) {
        if (b.ctx) rmusic_destroy(b.ctx);
        if (b.done) cudaEventDestroy(b.done);
        if (b.stream) cudaStreamDestroy(b.stream);
    }
    if (s->d_in) cudaFree(s->d_in);
    if (s->d_out) cudaFree(s->d_out);
    if (s->d_st) cudaFree(s->d_st);
    delete s;
}

}  // namespace

extern "C" {

int rmusic_serve_create(const rmusic_params* params, int device, const rmusic_serve_config* cfg,
                        rmusic_server** out) {
    if (!params || !cfg || !out) return RMUSIC_EINVAL;
    *out = nullptr;
    if (!config_ok(*cfg)) return RMUSIC_EINVAL;
    if (params->precision != RMUSIC_FP32_BATCHED) return RMUSIC_EUNSUPPORTED;
    if (params->geometry != RMUSIC_GEOM_ROW) return RMUSIC_EUNSUPPORTED;  // one map per frame slot
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return ndev == 0 ? RMUSIC_ECUDA : RMUSIC_EINVAL;
    }
    // budget: batch workspaces first, the rest to the arenas (9 bytes per pixel slot)
    const uint64_t ws = 8 * cfg->max_batch_pixels + (1u << 20);
    const uint64_t ws_total = ws * (uint64_t)cfg->inflight_batches;
    if (cfg->hbm_budget_bytes <= ws_total) return RMUSIC_ENOMEM;
    const uint64_t E = (cfg->hbm_budget_bytes - ws_total) / 9 / kSlotAlign * kSlotAlign;
    if (E < kSlotAlign) return RMUSIC_ENOMEM;
    rmusic_server* s = new (std::nothrow) rmusic_server();
    if (!s) return RMUSIC_ENOMEM;
    s->params = *params;
    s->params.use_graph = 0;  // every batch differs: capture would not pay
    s->params.timing = 0;
    s->cfg = *cfg;
    s->device = device;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int rc = RMUSIC_OK;
    if (cudaMalloc(&s->d_in, 4 * E) != cudaSuccess || cudaMalloc(&s->d_out, 4 * E) != cudaSuccess ||
        cudaMalloc(&s->d_st, E) != cudaSuccess) {
        cudaGetLastError();
        rc = RMUSIC_ENOMEM;
    }
    s->E = E;
    s->device_bytes = 9 * E;
    s->alloc.reset(E);
    s->streams.resize(cfg->max_streams);
    s->batches.resize(cfg->inflight_batches);
    for (BatchSlot& b : s->batches) {
        if (rc) break;
        if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess) {
            rc = RMUSIC_ECUDA;
            break;
        }
        rc = rmusic_create(&s->params, device, ws, &b.ctx);
        // the whole workspace a batch can need, now: a workspace that grew during serving would
        // free device memory, which synchronises the device and stalls every batch in flight
        if (!rc) rc = rmusic_reserve(b.ctx, cfg->max_batch_pixels, cfg->max_batch_frames);
        s->device_bytes += ws;
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (rc) {
        free_server(s);
        return rc;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return RMUSIC_OK;
}

int rmusic_serve_open_stream(rmusic_server* s, int32_t height, int32_t width, int32_t dtype, int32_t* stream_id) {
    if (!s || !stream_id || height < 1 || width < 1) return RMUSIC_EINVAL;
    if (dtype != RMUSIC_DTYPE_F32 && dtype != RMUSIC_DTYPE_U16) return RMUSIC_EINVAL;
    const uint64_t px = (uint64_t)height * (uint64_t)width;
    std::lock_guard<std::mutex> lock(s->mu);
    int id = -1;
    for (int i = 0; i < (int)s->streams.size(); ++i)
        if (!s->streams[i].open) {
            id = i;
            break;
        }
    if (id < 0 || px > s->cfg.max_batch_pixels) {
        s->st.opens_rejected += 1;
        return RMUSIC_ENOMEM;
    }
    const uint64_t stride = (px + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
    const uint64_t units = stride * (uint64_t)s->cfg.ring_depth;
    uint64_t off = 0;
    if (!s->alloc.allocate(units, kSlotAlign, &off)) {
        s->st.opens_rejected += 1;
        return RMUSIC_ENOMEM;
    }
    StreamState& ss = s->streams[id];
    ss = StreamState();
    ss.open = true;
    ss.H = height;
    ss.W = width;
    ss.dtype = dtype;
    ss.px = px;
    ss.ring_off = off;
    ss.slot_stride = stride;
    ss.ring_units = units;
    ss.busy.assign(s->cfg.ring_depth, 0);
    *stream_id = id;
    return RMUSIC_OK;
}

int rmusic_serve_submit(rmusic_server* s, int32_t stream_id, const void* h_frame, float* h_out, uint8_t* h_status,
                        uint64_t tag) {
    if (!s || !h_frame || !h_out) return RMUSIC_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (stream_id < 0 || stream_id >= (int)s->streams.size()) return RMUSIC_EINVAL;
    StreamState& ss = s->streams[stream_id];
    if (!ss.open || ss.closing) return RMUSIC_EINVAL;
    int slot = -1;
    for (int k = 0; k < (int)ss.busy.size(); ++k)
        if (!ss.busy[k]) {
            slot = k;
            break;
        }
    if (slot < 0) {
        s->st.submits_rejected += 1;
        return RMUSIC_EAGAIN;
    }
    ss.busy[slot] = 1;
    ss.queued += 1;
    Request r;
    r.stream = stream_id;
    r.slot = slot;
    r.h_in = h_frame;
    r.h_out = h_out;
    r.h_status = h_status;
    r.tag = tag;
    r.t_submit = now_s();
    r.t_launch = 0.0;
    s->pending.push_back(r);
    s->cv_work.notify_one();
    return RMUSIC_OK;
}

int rmusic_serve_poll(rmusic_server* s, rmusic_completion* out, int32_t max, int32_t timeout_ms) {
    if (!s || (max > 0 && !out) || max < 0) return RMUSIC_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->done.empty() && timeout_ms > 0)
        s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), [s] { return !s->done.empty(); });
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return n;
}

int rmusic_serve_close_stream(rmusic_server* s, int32_t stream_id) {
    if (!s) return RMUSIC_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    if (stream_id < 0 || stream_id >= (int)s->streams.size() || !s->streams[stream_id].open) return RMUSIC_EINVAL;
    StreamState& ss = s->streams[stream_id];
    ss.closing = true;
    s->cv_done.wait(lock, [&ss] { return ss.queued == 0; });
    s->alloc.release(ss.ring_off, ss.ring_units);
    ss = StreamState();
    return RMUSIC_OK;
}

int rmusic_serve_get_stats(rmusic_server* s, rmusic_serve_stats* out) {
    if (!s || !out) return RMUSIC_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->st;
    out->device_bytes = s->device_bytes;
    out->arena_free_pixels = s->alloc.free_units();
    int open = 0, queued = 0, inflight = 0;
    for (const StreamState& ss : s->streams)
        if (ss.open) ++open;
    queued = (int)s->pending.size();
    for (const BatchSlot& b : s->batches)
        if (b.busy) ++inflight;
    out->streams_open = open;
    out->frames_queued = queued;
    out->batches_inflight = inflight;
    return RMUSIC_OK;
}

void rmusic_serve_destroy(rmusic_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    free_server(s);
    if (prev >= 0) cudaSetDevice(prev);
}

}  // extern "C"
