// capi.cu -- the library's C ABI (include/rmusic.h): contexts, workspaces, frame tables,
// batching under an HBM budget, CUDA-graph capture and replay, and the host-buffer entry.
//
// A call is: validate descriptors -> build the device frame table (band bins, window-line
// geometry, work-item ranges) -> band-pass every carrier line (analytic.cu) -> either one
// thread-per-pixel launch per frame (plain.cu) or one persistent launch per covariance order
// over all frames (batched.cu; square.cu for the paper's square block, one launch per
// half-width). Frames whose analytic signal does not fit the workspace budget together are
// processed in consecutive groups.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/rmusic.h"
#include "rmusic_device.cuh"
#include "rmusic_launch.h"
#include "rmusic_validate.h"

using namespace rmusic;

namespace rmusic {

static bool params_ok(const rmusic_params& p) {
    if (p.geometry == RMUSIC_GEOM_SQUARE) {
        if (p.half_width < 1 || p.half_width > kMaxSquareLp) return false;
    } else if (p.geometry == RMUSIC_GEOM_ROW) {
        if (p.window_len < 2 || p.window_len > kMaxN) return false;
        if (p.cov_order < 2 || p.cov_order > kMaxL || p.cov_order > p.window_len) return false;
        if (p.forward_backward != 0 && p.forward_backward != 1) return false;
        if (p.deriv_axis != 0 && p.deriv_axis != 1) return false;
    } else {
        return false;
    }
    if (p.carrier_axis != 0 && p.carrier_axis != 1) return false;
    if (p.unwrap != 0 && p.unwrap != 1) return false;
    if (p.raw_input != 0 && p.raw_input != 1) return false;
    if (p.exhaustive != 0 && p.exhaustive != 1) return false;
    if (p.raw_input && (p.geometry != RMUSIC_GEOM_ROW || p.deriv_axis != p.carrier_axis)) return false;
    if (p.geometry == RMUSIC_GEOM_ROW && p.model_order >= p.cov_order) return false;
    if (p.unwrap && p.geometry != RMUSIC_GEOM_SQUARE) return false;
    if (!(p.carrier_freq >= 0.0 && p.carrier_freq < 0.5)) return false;
    if (!(p.band_halfwidth >= 0.0 && p.band_halfwidth < 0.5)) return false;
    if (!(p.band_cross >= 0.0 && p.band_cross < 0.5)) return false;
    if (p.precision < RMUSIC_PLAIN_FP64 || p.precision > RMUSIC_FP32_BATCHED) return false;
    if (p.max_sweeps < 0 || p.max_root_iters < 0) return false;
    return true;
}

int params_check(const rmusic_params& p) {
    if (p.model_order < 1) return RMUSIC_EINVAL;
    if (p.model_order > kMaxModelOrder) return RMUSIC_EUNSUPPORTED;
    if (!params_ok(p)) return RMUSIC_EINVAL;
    // the batched model-order solver works on raw real lines along the carrier (row windows)
    if (p.model_order > 1 && p.precision == RMUSIC_FP32_BATCHED && (p.geometry != RMUSIC_GEOM_ROW || !p.raw_input))
        return RMUSIC_EUNSUPPORTED;
    if (p.geometry == RMUSIC_GEOM_SQUARE && p.precision != RMUSIC_FP32_BATCHED) return RMUSIC_EUNSUPPORTED;
    return RMUSIC_OK;
}

int describe_frame(const rmusic_params& p, const rmusic_frame_desc& d, FrameDev* F) {
    if (d.height < 1 || d.width < 1) return RMUSIC_EINVAL;
    const int pitch = d.pitch_elems == 0 ? d.width : d.pitch_elems;
    if (pitch < d.width) return RMUSIC_EINVAL;
    if (d.dtype != RMUSIC_DTYPE_F32 && d.dtype != RMUSIC_DTYPE_U16 && d.dtype != RMUSIC_DTYPE_C64)
        return RMUSIC_EINVAL;
    const int esz = d.dtype == RMUSIC_DTYPE_C64 ? 8 : d.dtype == RMUSIC_DTYPE_F32 ? 4 : 2;
    if (d.offset_bytes % esz) return RMUSIC_EINVAL;
    const bool square = p.geometry == RMUSIC_GEOM_SQUARE;
    int N, L;
    if (square) {
        // the paper's block: L holds the half-width Lp, N the block side 2 Lp + 1
        L = p.half_width;
        N = 2 * L + 1;
        if (!square_supports(L)) return RMUSIC_EUNSUPPORTED;
    } else {
        N = d.window_len ? d.window_len : p.window_len;
        L = d.cov_order ? d.cov_order : p.cov_order;
        if (N < 2 || N > kMaxN || L < 2 || L > kMaxL || L > N) return RMUSIC_EINVAL;
        if (p.precision == RMUSIC_FP32_BATCHED && p.model_order > 1 &&
            (d.dtype == RMUSIC_DTYPE_C64 || !batched_p_supports(p.model_order, L)))
            return RMUSIC_EUNSUPPORTED;  // real frames only: the solver takes R as real symmetric
        if (p.precision == RMUSIC_FP32_BATCHED && p.model_order == 1 &&
            !(p.forward_backward ? batched_supports(L) : batched_fwd_supports(L)))
            return RMUSIC_EUNSUPPORTED;
    }
    memset(F, 0, sizeof(*F));
    F->in_off = d.offset_bytes;
    F->out_off = d.out_offset;
    F->H = d.height;
    F->W = d.width;
    F->pitch = pitch;
    F->dtype = d.dtype;
    F->N = N;
    F->L = L;
    F->carrier_axis = p.carrier_axis;
    F->deriv_axis = square ? 0 : p.deriv_axis;  // the square block reads a row-major workspace
    F->raw = p.raw_input && d.dtype != RMUSIC_DTYPE_C64;
    F->geom = square ? kGeomSquare : kGeomRow;
    F->nlines = p.carrier_axis == 0 ? d.height : d.width;
    F->len = p.carrier_axis == 0 ? d.width : d.height;
    if (F->len > kMaxLine) return RMUSIC_EUNSUPPORTED;
    // kept band: 1 <= k < len/2 and |k/len - f0| < B (a contiguous run of bins)
    const double f0 = p.carrier_freq;
    const double B = p.band_halfwidth > 0.0 ? p.band_halfwidth : 0.5 * f0;
    int klo = -1, nb = 0;
    for (int k = 1; 2 * k < F->len; ++k) {
        if (fabs((double)k / (double)F->len - f0) < B) {
            if (klo < 0) klo = k;
            ++nb;
        }
    }
    F->k_lo = klo < 0 ? 1 : klo;
    F->nb = nb;
    if (p.band_cross > 0.0) {
        // kept cross bins: signed k with |k| < B_c len across the carrier
        const int lenc = p.carrier_axis == 0 ? d.height : d.width;
        const double lim = p.band_cross * (double)lenc;
        int kc = 0;
        while ((double)(kc + 1) < lim) ++kc;
        if (kc > kMaxCrossKc) return RMUSIC_EUNSUPPORTED;
        F->cross_kc = kc;
    }
    F->wlines = F->deriv_axis == 0 ? d.height : d.width;
    F->wlen = F->deriv_axis == 0 ? d.width : d.height;
    F->f0 = f0;
    if (square) {
        F->nchunks = (d.width + kSqTX - 1) / kSqTX;  // 32-pixel items across a row
        F->omega_ref = 6.283185307179586476925 * f0;
    } else {
        F->rowp_shift = row_pixels_per_lane_shift(F->wlen);
        const int run = 32 << F->rowp_shift;
        F->nchunks = (F->wlen + run - 1) / run;
        F->omega_ref = p.deriv_axis == p.carrier_axis ? 6.283185307179586476925 * f0 : 0.0;
    }
    // the solvers split a frame's work-item index with 32-bit arithmetic (far above any frame whose
    // analytic signal fits a GPU)
    const int64_t rows = square ? (int64_t)d.height : (int64_t)F->wlines;
    if (rows * (int64_t)F->nchunks >= (int64_t)1 << 31) return RMUSIC_EUNSUPPORTED;
    return RMUSIC_OK;
}

}  // namespace rmusic

namespace {

constexpr int kMaxGraphs = 8;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

constexpr int kCounterSlots = 64;  // [0, kStatSlot) work counters, [kStatSlot ..] statistics
constexpr int kStatSlot = 32;

// A solver key names one compiled solver family: the covariance order L of the row-window
// solver (2 .. kMaxL), kSquareKey0 + Lp for the square-block solver, kFwdKey0 + L for the row-window
// solver of the forward estimate (no forward-backward average), kModelKey0 + 16 (p - 2) + L for the
// row-window solver of model order p = 2 or 3.
constexpr int kSquareKey0 = 16;
constexpr int kFwdKey0 = 32;
constexpr int kModelKey0 = 48;
constexpr int kKeys = kModelKey0 + 32;
static_assert(kMaxL < kSquareKey0 && kSquareKey0 + kMaxSquareLp < kFwdKey0 && kFwdKey0 + kMaxL < kModelKey0 &&
                  kMaxL < 16,
              "solver keys overlap");

bool key_square(int key) { return key >= kSquareKey0 && key < kFwdKey0; }
bool key_fwd(int key) { return key >= kFwdKey0 && key < kModelKey0; }
bool key_model(int key) { return key >= kModelKey0; }
int key_model_p(int key) { return 2 + (key - kModelKey0) / 16; }
int key_model_L(int key) { return (key - kModelKey0) % 16; }
bool solver_supports(int key) {
    return key_model(key) ? batched_p_supports(key_model_p(key), key_model_L(key))
         : key_fwd(key) ? batched_fwd_supports(key - kFwdKey0)
         : key_square(key) ? square_supports(key - kSquareKey0) : batched_supports(key);
}
int solver_num_variants(int key) {
    return key_model(key) ? 1
         : key_fwd(key) ? batched_fwd_num_variants(key - kFwdKey0)
         : key_square(key) ? square_num_variants(key - kSquareKey0) : batched_num_variants(key);
}
int solver_default_variant(int key) {
    return key_model(key) ? 0
         : key_fwd(key) ? batched_fwd_default_variant(key - kFwdKey0)
         : key_square(key) ? square_default_variant(key - kSquareKey0) : batched_default_variant(key);
}
int solver_ctas(int key, int v) {
    return key_model(key) ? batched_p_ctas(key_model_L(key))
         : key_fwd(key) ? batched_fwd_variant_ctas(key - kFwdKey0, v)
         : key_square(key) ? square_variant_ctas(key - kSquareKey0, v) : batched_variant_ctas(key, v);
}
// The solver key of a row-window frame of covariance order L under the parameters p.
int row_key(const rmusic_params& p, int L) {
    if (p.model_order > 1) return kModelKey0 + 16 * (p.model_order - 2) + L;
    return p.forward_backward ? L : kFwdKey0 + L;
}
// The solver key of a frame of the plan (its table entry's geometry and covariance order).
int frame_key(const rmusic_params& p, const FrameDev& F) {
    if (F.geom == kGeomSquare) return kSquareKey0 + F.L;
    return row_key(p, F.L);
}

struct GraphEntry {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    FrameDev* h_table = nullptr;  // pinned; read by the graph's upload node at every replay
    int launches = 0;
    uint64_t stamp = 0;
    std::vector<cudaEvent_t> a1_ev, solver_ev;  // timing events recorded by the graph
    std::vector<cudaEvent_t> owned;              // every event the graph records (it owns them)
};

}  // namespace

struct rmusic_ctx {
    rmusic_params p{};
    int device = 0;
    size_t budget = 0;
    int num_sms = 0;
    // device workspaces
    void* d_gamma = nullptr;
    size_t gamma_cap = 0;  // bytes
    FrameDev* d_table = nullptr;
    size_t table_cap = 0;  // entries
    unsigned long long* d_counters = nullptr;  // one per covariance order
    // pinned staging of the frame table for non-graph calls
    FrameDev* h_table = nullptr;
    size_t h_table_cap = 0;
    cudaEvent_t table_free = nullptr;  // recorded after the last table upload
    // host-buffer entry staging
    void* d_in = nullptr;
    size_t in_cap = 0;
    float* d_out = nullptr;
    size_t out_cap = 0;
    uint8_t* d_st = nullptr;
    size_t st_cap = 0;
    // phase-assembly workspace
    void* d_unwrap = nullptr;
    size_t unwrap_cap = 0;
    // graphs
    GraphEntry graphs[kMaxGraphs];
    uint64_t graph_clock = 0;
    cudaStream_t cap_stream = nullptr;  // graphs are captured here, then launched on the caller's stream
    // statistics and timing
    cudaEvent_t call_done = nullptr;
    std::vector<cudaEvent_t> ev_pool;  // events recorded directly by calls (reused call after call)
    int ev_used = 0;
    std::vector<cudaEvent_t> gev_free;                  // events released by dropped graphs
    std::vector<cudaEvent_t>* capture_owned = nullptr;  // the graph being captured takes its events here
    std::vector<cudaEvent_t> a1_ev, solver_ev;          // pairs of events of the last call
    uint64_t last_pixels = 0;
    // bookkeeping
    size_t held = 0;
    rmusic_stats stats{};
    char last_err[256] = {0};
    int grid_by_Lv[kKeys][4] = {{0}};
    int variant_by_L[kKeys];  // solver variant chosen for each solver key, -1 = none yet
};

namespace {

int cuda_fail(rmusic_ctx* c, cudaError_t e, const char* what) {
    if (c) snprintf(c->last_err, sizeof(c->last_err), "%s: %s", what, cudaGetErrorString(e));
    return RMUSIC_ECUDA;
}

#define RM_CUDA(call)                                          \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
    } while (0)

// Release a cached graph: its executable, its pinned frame table, and its timing events (kept for
// later captures).
void drop_graph(rmusic_ctx* ctx, GraphEntry& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.h_table) cudaFreeHost(g.h_table);
    ctx->gev_free.insert(ctx->gev_free.end(), g.owned.begin(), g.owned.end());
    g = GraphEntry{};
}

// Grow a device buffer to at least `bytes` (never shrinks). Keeps the budget.
int ensure(rmusic_ctx* ctx, void** ptr, size_t* cap_bytes, size_t bytes) {
    if (*cap_bytes >= bytes) return RMUSIC_OK;
    size_t want = std::max(bytes, *cap_bytes + *cap_bytes / 2);
    if (ctx->budget && ctx->held - *cap_bytes + want > ctx->budget) {
        want = bytes;
        if (ctx->held - *cap_bytes + want > ctx->budget) return RMUSIC_ENOMEM;
    }
    if (*ptr) {
        cudaStreamSynchronize(nullptr);
        cudaDeviceSynchronize();
        cudaFree(*ptr);
        ctx->held -= *cap_bytes;
        *ptr = nullptr;
        *cap_bytes = 0;
    }
    void* np = nullptr;
    cudaError_t e = cudaMalloc(&np, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RMUSIC_ENOMEM;
    }
    *ptr = np;
    *cap_bytes = want;
    ctx->held += want;
    // any cached graph may reference the old buffer
    for (auto& g : ctx->graphs) drop_graph(ctx, g);
    return RMUSIC_OK;
}

// Everything the kernels need to know about one frame, derived from its descriptor.
struct Plan {
    std::vector<FrameDev> frames;  // in launch order (grouped by L for the batched path)
    std::vector<int> group_L;      // batched: solver key of each group (L, or kSquareKey0 + Lp)
    std::vector<int> group_first;  // batched: first table entry of each group
    std::vector<int> group_count;
    std::vector<int64_t> group_items;
    int64_t total_lines = 0;  // band-pass CTAs
    int band_sched = 0;       // kBand* bits of the band-pass schedules the frames take
    int64_t cross_groups = 0;  // 32-line groups of the cross-band pass (0: no cross band)
    int max_kc = 0;
    int max_len = 0;
    uint64_t gamma_elems = 0;
    // square geometry with complex64 frames only: the frames are the analytic signal already, and
    // the solver reads them in place (no band-pass launch, no copy into the workspace)
    bool square_direct = false;
};

int describe(const rmusic_ctx* ctx, const rmusic_frame_desc& d, FrameDev* F) { return describe_frame(ctx->p, d, F); }

// Bytes per pixel of the analytic-signal workspace: complex128 for the plain FP64 path.
size_t gamma_elem_bytes(const rmusic_ctx* ctx) {
    return ctx->p.precision == RMUSIC_PLAIN_FP64 ? sizeof(double2) : sizeof(float2);
}

int build_plan(const rmusic_ctx* ctx, const rmusic_frame_desc* descs, int n, Plan* plan) {
    plan->frames.resize(n);
    for (int i = 0; i < n; ++i) {
        int rc = describe(ctx, descs[i], &plan->frames[i]);
        if (rc) return rc;
    }
    if (ctx->p.precision == RMUSIC_FP32_BATCHED)
        std::stable_sort(plan->frames.begin(), plan->frames.end(),
                         [](const FrameDev& a, const FrameDev& b) { return a.L < b.L; });
    uint64_t goff = 0;
    int64_t lines = 0;
    for (int i = 0; i < n; ++i) {
        FrameDev& F = plan->frames[i];
        F.gam_off = goff;
        goff += (uint64_t)F.H * (uint64_t)F.W;
        F.line_start = lines;
        lines += band_assign(&F, ctx->p.precision == RMUSIC_PLAIN_FP64);
        plan->band_sched |= band_schedule_bit(F);
        if (ctx->p.band_cross > 0.0) {
            F.cross_start = plan->cross_groups;
            plan->cross_groups += ((F.carrier_axis == 0 ? F.W : F.H) + 31) / 32;
            plan->max_kc = std::max(plan->max_kc, F.cross_kc);
        }
        plan->max_len = std::max(plan->max_len, F.len);
        const int key = frame_key(ctx->p, F);
        if (i == 0 || F.L != plan->frames[i - 1].L) {
            plan->group_L.push_back(key);
            plan->group_first.push_back(i);
            plan->group_count.push_back(0);
            plan->group_items.push_back(0);
        }
        F.item_start = plan->group_items.back();
        if (F.geom == kGeomSquare) {
            F.sq_strip_rows = square_strip_rows(F.H);
            plan->group_items.back() += (int64_t)(F.sq_strip_rows / kSqTY) * F.nchunks;
        } else {
            plan->group_items.back() += (int64_t)F.wlines * F.nchunks;
        }
        plan->group_count.back() += 1;
    }
    // square geometry: every group's single-row items after all of its strips
    for (size_t g = 0; g < plan->group_first.size(); ++g) {
        for (int j = 0; j < plan->group_count[g]; ++j) {
            FrameDev& F = plan->frames[(size_t)(plan->group_first[g] + j)];
            if (F.geom != kGeomSquare) continue;
            F.item_start2 = plan->group_items[g];
            plan->group_items[g] += (int64_t)(F.H - F.sq_strip_rows) * F.nchunks;
        }
    }
    plan->total_lines = lines;
    plan->gamma_elems = goff;
    plan->square_direct = ctx->p.geometry == RMUSIC_GEOM_SQUARE && n > 0 && plan->cross_groups == 0;
    for (const FrameDev& F : plan->frames) plan->square_direct = plan->square_direct && F.dtype == kDtC64;
    return RMUSIC_OK;
}

// Queue the work of one plan (whose frame table has just been copied to d_table) on `s`.
// Record a timing event on s (an event-record node when s is capturing). Returns it, or nullptr
// without timing. A graph being captured owns the events it records (taken from the released ones
// or created), so no later call or capture records into them while the graph is cached.
cudaEvent_t stamp(rmusic_ctx* ctx, cudaStream_t s) {
    if (!ctx->p.timing) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    const bool capturing = cs == cudaStreamCaptureStatusActive;
    cudaEvent_t e = nullptr;
    if (capturing) {
        if (!ctx->gev_free.empty()) {
            e = ctx->gev_free.back();
            ctx->gev_free.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            return nullptr;
        }
        if (ctx->capture_owned) ctx->capture_owned->push_back(e);
    } else {
        if (ctx->ev_used >= (int)ctx->ev_pool.size()) {
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            ctx->ev_pool.push_back(e);
        }
        e = ctx->ev_pool[ctx->ev_used++];
    }
    const cudaError_t r = capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
    return r == cudaSuccess ? e : nullptr;
}

void stamp_pair(std::vector<cudaEvent_t>& v, cudaEvent_t a, cudaEvent_t b) {
    if (a && b) {
        v.push_back(a);
        v.push_back(b);
    }
}

// ---- solver variant selection (the autotuner) ---------------------------------------------------
// Each solver key (covariance order, or square half-width) has several register-cap variants of
// its solver (batched_variants.h, square_variants.h). A variant is chosen per device and key by
// timing all of them on real work (the first call with `autotune` set, or rmusic_autotune); the
// choice is shared by every context on the device and, when RMUSIC_TUNE_CACHE names a file,
// appended to it as a JSON line
//   {"device": "<name>/<SMs>sm", "key": 8, "L": 8, "variant": 1, "ctas_per_sm": 6, "ms": 1.917}
// ("key" is L for row windows and 16 + Lp for the square block) and read back by later
// processes. Untuned keys use the default variant.
constexpr int kTuneDevices = 64;
std::mutex g_tune_mu;
int g_tuned[kTuneDevices][kKeys];
bool g_tune_loaded[kTuneDevices];
bool g_tune_ready = false;

void tune_init_locked() {
    if (g_tune_ready) return;
    for (int d = 0; d < kTuneDevices; ++d) {
        g_tune_loaded[d] = false;
        for (int l = 0; l < kKeys; ++l) g_tuned[d][l] = -1;
    }
    g_tune_ready = true;
}

std::string device_key(int device) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
    return std::string(prop.name) + "/" + std::to_string(prop.multiProcessorCount) + "sm";
}

// Value of "key": in a JSON line written by store_tune (strings without escapes, integers).
bool json_field(const char* line, const char* key, std::string* out) {
    std::string pat = std::string("\"") + key + "\": ";
    const char* p = strstr(line, pat.c_str());
    if (!p) return false;
    p += pat.size();
    if (*p == '"') {
        const char* e = strchr(p + 1, '"');
        if (!e) return false;
        *out = std::string(p + 1, e);
    } else {
        const char* e = p;
        while (*e && *e != ',' && *e != '}') ++e;
        *out = std::string(p, e);
    }
    return true;
}

void load_tune_locked(int device) {
    if (device < 0 || device >= kTuneDevices || g_tune_loaded[device]) return;
    g_tune_loaded[device] = true;
    const char* path = getenv("RMUSIC_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    const std::string key = device_key(device);
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        std::string dev, ks, vs;
        if (!json_field(line, "device", &dev) || dev != key) continue;
        if (!(json_field(line, "key", &ks) || json_field(line, "L", &ks)) || !json_field(line, "variant", &vs))
            continue;
        const int k = atoi(ks.c_str()), v = atoi(vs.c_str());
        if (k >= 0 && k < kKeys && solver_supports(k) && v >= 0 && v < solver_num_variants(k))
            g_tuned[device][k] = v;
    }
    fclose(f);
}

void store_tune(int device, int key, int v, float ms) {
    const char* path = getenv("RMUSIC_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{\"device\": \"%s\", \"key\": %d, \"%s\": %d, \"variant\": %d, \"ctas_per_sm\": %d, "
            "\"ms\": %.4f}\n",
            device_key(device).c_str(), key,
            key_square(key) ? "Lp" : key_fwd(key) ? "L_fwd" : key_model(key) ? (key_model_p(key) == 2 ? "L_p2" : "L_p3") : "L",
            key_square(key) ? key - kSquareKey0 : key_fwd(key) ? key - kFwdKey0 : key_model(key) ? key_model_L(key) : key,
            v, solver_ctas(key, v), ms);
    fclose(f);
}

int solver_variant(rmusic_ctx* ctx, int L) {
    if (ctx->variant_by_L[L] >= 0) return ctx->variant_by_L[L];
    int v = -1;
    if (ctx->device < kTuneDevices) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_init_locked();
        load_tune_locked(ctx->device);
        v = g_tuned[ctx->device][L];
    }
    return v >= 0 ? v : solver_default_variant(L);
}

bool solver_tuned(rmusic_ctx* ctx, int L) {
    if (ctx->variant_by_L[L] >= 0) return true;
    if (ctx->device >= kTuneDevices) return false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_init_locked();
    load_tune_locked(ctx->device);
    return g_tuned[ctx->device][L] >= 0;
}

int solver_grid(rmusic_ctx* ctx, int L, int v) {
    if (ctx->grid_by_Lv[L][v] == 0)
        ctx->grid_by_Lv[L][v] =
            key_model(L) ? batched_p_grid(key_model_p(L), key_model_L(L), ctx->device)
            : key_fwd(L) ? batched_fwd_grid(L - kFwdKey0, v, ctx->device)
            : key_square(L) ? square_grid(L - kSquareKey0, v, ctx->device) : batched_grid(L, v, ctx->device);
    return ctx->grid_by_Lv[L][v];
}

// Launch variant v of the solver of group g of `plan` (solver key plan.group_L[g]) on s; the
// group's work counter must be zero. stat_counters receives the iteration statistics or is NULL.
cudaError_t launch_solver(rmusic_ctx* ctx, const Plan& plan, size_t g, int v, const void* d_frames, float* d_out,
                          uint8_t* d_status, unsigned long long* stat_counters, cudaStream_t s) {
    const rmusic_params& p = ctx->p;
    const int key = plan.group_L[g];
    const float2* gamma = static_cast<const float2*>(ctx->d_gamma);
    if (key_square(key)) {
        SquareArgs a;
        a.max_power_iters = p.max_sweeps ? p.max_sweeps : 100;
        a.max_iters = p.max_root_iters ? p.max_root_iters : 32;
        a.polish64 = p.polish_fp64;
        a.exhaustive = p.exhaustive;
        a.tol2 = 1e-9f;  // power iteration: stop at a step below 3.2e-5 (u1 to ~1e-5)
        a.counters = stat_counters;
        a.direct = plan.square_direct ? static_cast<const unsigned char*>(d_frames) : nullptr;
        return launch_square(key - kSquareKey0, v, ctx->d_table + plan.group_first[g], plan.group_count[g],
                             plan.group_items[g], ctx->d_counters + g, gamma, d_out, d_status, a,
                             solver_grid(ctx, key, v), s);
    }
    BatchedArgs a;
    a.max_sweeps = p.max_sweeps ? p.max_sweeps : 6;
    // the model-order solver takes every root by Aberth's method (noise-free windows put p double
    // roots on the circle, where it converges linearly): more sweeps by default
    a.max_iters = p.max_root_iters ? p.max_root_iters : key_model(key) ? 32 : 16;
    a.polish64 = p.polish_fp64;
    a.exhaustive = p.exhaustive;
    a.counters = stat_counters;
    a.fb = p.forward_backward;
    if (key_model(key))
        return launch_batched_p(key_model_p(key), key_model_L(key), ctx->d_table + plan.group_first[g],
                                plan.group_count[g], plan.group_items[g], ctx->d_counters + g, gamma, d_out, d_status,
                                a, solver_grid(ctx, key, v), s);
    if (key_fwd(key))
        return launch_batched_fwd(key - kFwdKey0, v, ctx->d_table + plan.group_first[g], plan.group_count[g],
                                  plan.group_items[g], ctx->d_counters + g, gamma, d_out, d_status, a,
                                  solver_grid(ctx, key, v), s);
    return launch_batched(key, v, ctx->d_table + plan.group_first[g], plan.group_count[g], plan.group_items[g],
                          ctx->d_counters + g, gamma, d_out, d_status, a, solver_grid(ctx, key, v), s);
}

// Time every solver variant on `plan`, whose table and analytic signal are already on the device
// (queued on s), and keep the fastest for each covariance order not tuned yet (all of them when
// `force`). Synchronises s; the maps it writes are the call's results.
int tune_plan(rmusic_ctx* ctx, const Plan& plan, const void* d_frames, float* d_out, uint8_t* d_status, cudaStream_t s,
              bool force) {
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    RM_CUDA(cudaEventCreate(&t0));
    RM_CUDA(cudaEventCreate(&t1));
    int rc = RMUSIC_OK;
    for (size_t g = 0; g < plan.group_L.size() && rc == RMUSIC_OK; ++g) {
        const int L = plan.group_L[g];
        if (!force && solver_tuned(ctx, L)) continue;
        float best = 1e30f;
        int bestv = solver_default_variant(L);
        // highest variant first: the last one run (variant 0, a register-cap variant) leaves the
        // call's maps exactly as the default variant computes them
        for (int v = solver_num_variants(L) - 1; v >= 0 && rc == RMUSIC_OK; --v) {
            float tmin = 1e30f;
            for (int rep = 0; rep < 2 && rc == RMUSIC_OK; ++rep) {
                cudaError_t e = cudaMemsetAsync(ctx->d_counters + g, 0, sizeof(unsigned long long), s);
                if (e == cudaSuccess) e = cudaEventRecord(t0, s);
                if (e == cudaSuccess) e = launch_solver(ctx, plan, g, v, d_frames, d_out, d_status, nullptr, s);
                if (e == cudaSuccess) e = cudaEventRecord(t1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e != cudaSuccess) {
                    rc = cuda_fail(ctx, e, "autotune");
                    break;
                }
                tmin = std::min(tmin, ms);
            }
            if (tmin < best) {
                best = tmin;
                bestv = v;
            }
        }
        if (rc) break;
        ctx->variant_by_L[L] = bestv;
        if (ctx->device < kTuneDevices) {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            tune_init_locked();
            g_tuned[ctx->device][L] = bestv;
        }
        store_tune(ctx->device, L, bestv, best);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return rc;
}

// An NVTX range around the host-side enqueue of one stage, so that timeline tools (Nsight Systems)
// group the stage's kernels under its name; a no-op unless such a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

int enqueue(rmusic_ctx* ctx, const Plan& plan, const void* d_frames, float* d_out, uint8_t* d_status,
            cudaStream_t s, int* launches) {
    const int n = (int)plan.frames.size();
    cudaEvent_t e0 = stamp(ctx, s);
    const bool fp64 = ctx->p.precision == RMUSIC_PLAIN_FP64;
    if (!plan.square_direct) {
        NvtxRange r("rmusic.bandpass");
        RM_CUDA(launch_analytic(ctx->d_table, n, plan.total_lines, plan.max_len, plan.band_sched, d_frames,
                                ctx->d_gamma, fp64, s));
        ++*launches;
        if (plan.cross_groups > 0) {
            RM_CUDA(launch_crossband(ctx->d_table, n, plan.cross_groups, plan.max_kc, ctx->d_gamma, fp64, s));
            ++*launches;
        }
    }
    stamp_pair(ctx->a1_ev, e0, stamp(ctx, s));
    const rmusic_params& p = ctx->p;
    if (p.precision == RMUSIC_FP32_BATCHED) {
        for (size_t g = 0; g < plan.group_L.size(); ++g) {
            const int L = plan.group_L[g];
            const int v = solver_variant(ctx, L);
            NvtxRange r("rmusic.solver");
            RM_CUDA(cudaMemsetAsync(ctx->d_counters + g, 0, sizeof(unsigned long long), s));
            cudaEvent_t e1 = stamp(ctx, s);
            RM_CUDA(launch_solver(ctx, plan, g, v, d_frames, d_out, d_status, ctx->d_counters + kStatSlot, s));
            stamp_pair(ctx->solver_ev, e1, stamp(ctx, s));
            ctx->stats.solver_ctas_per_sm = solver_ctas(L, v);
            ctx->stats.solver_variant = v;
            ++*launches;
        }
        if (p.unwrap) {
            // phase assembly: the alpha maps (third map) unwrapped into the fourth map
            NvtxRange r("rmusic.unwrap");
            int64_t maxnodes = 0;
            for (const FrameDev& F : plan.frames) maxnodes = std::max<int64_t>(maxnodes, unwrap_frame_nodes(F.H, F.W));
            RM_CUDA(launch_unwrap(ctx->d_table, n, (int64_t)plan.gamma_elems, maxnodes, d_out, 2, d_out, 3,
                                  ctx->d_unwrap, -1, ctx->d_counters + kStatSlot + kWaitSlot, launches, s));
        }
    } else {
        PlainArgs a;
        a.p = p.model_order;
        a.fb = p.forward_backward;
        a.max_sweeps = p.max_sweeps ? p.max_sweeps : 30;
        a.max_iters = p.max_root_iters ? p.max_root_iters : 500;
        NvtxRange r("rmusic.plain");
        cudaEvent_t e1 = stamp(ctx, s);
        for (int f = 0; f < n; ++f) {
            if (p.precision == RMUSIC_PLAIN_FP64)
                RM_CUDA(launch_plain_fp64(ctx->d_table + f, plan.frames[f], static_cast<const double2*>(ctx->d_gamma),
                                          d_out, d_status, a, s));
            else
                RM_CUDA(launch_plain_fp32(ctx->d_table + f, plan.frames[f], static_cast<const float2*>(ctx->d_gamma),
                                          d_out, d_status, a, s));
            ++*launches;
        }
        stamp_pair(ctx->solver_ev, e1, stamp(ctx, s));
    }
    return RMUSIC_OK;
}

int ensure_tables(rmusic_ctx* ctx, size_t nframes) {
    if (ctx->table_cap < nframes) {
        size_t bytes = ctx->table_cap * sizeof(FrameDev);
        void* ptr = ctx->d_table;
        int rc = ensure(ctx, &ptr, &bytes, std::max<size_t>(nframes, 64) * sizeof(FrameDev));
        if (rc) return rc;
        ctx->d_table = (FrameDev*)ptr;
        ctx->table_cap = bytes / sizeof(FrameDev);
    }
    if (ctx->h_table_cap < nframes) {
        if (ctx->h_table) {
            cudaEventSynchronize(ctx->table_free);
            cudaFreeHost(ctx->h_table);
        }
        size_t cap = std::max<size_t>(nframes, 64);
        if (cudaMallocHost(&ctx->h_table, cap * sizeof(FrameDev)) != cudaSuccess) {
            ctx->h_table = nullptr;
            ctx->h_table_cap = 0;
            return RMUSIC_ENOMEM;
        }
        ctx->h_table_cap = cap;
    }
    return RMUSIC_OK;
}

// Process frames [first, first + count) of descs as one workspace group.
int run_group(rmusic_ctx* ctx, const void* d_frames, const rmusic_frame_desc* descs, int count,
              float* d_out, uint8_t* d_status, cudaStream_t s, bool force_tune) {
    Plan plan;
    int rc = build_plan(ctx, descs, count, &plan);
    if (rc) return rc;
    rc = ensure(ctx, &ctx->d_gamma, &ctx->gamma_cap, std::max<uint64_t>(plan.gamma_elems, 1) * gamma_elem_bytes(ctx));
    if (rc) return rc;
    rc = ensure_tables(ctx, plan.frames.size());
    if (rc) return rc;
    if (ctx->p.unwrap) {
        int64_t maxpx = 0;
        for (const FrameDev& F : plan.frames) maxpx = std::max<int64_t>(maxpx, unwrap_frame_nodes(F.H, F.W));
        if (plan.gamma_elems >= (1ull << 31)) return RMUSIC_EINVAL;
        rc = ensure(ctx, &ctx->d_unwrap, &ctx->unwrap_cap, unwrap_workspace_bytes((int64_t)plan.gamma_elems, maxpx));
        if (rc) return rc;
    }

    // autotune: time the solver variants on this call's work (band-pass first, outside any graph)
    if (ctx->p.precision == RMUSIC_FP32_BATCHED && (force_tune || ctx->p.autotune)) {
        bool need = force_tune;
        for (int L : plan.group_L) need = need || !solver_tuned(ctx, L);
        if (need) {
            RM_CUDA(cudaEventSynchronize(ctx->table_free));
            memcpy(ctx->h_table, plan.frames.data(), plan.frames.size() * sizeof(FrameDev));
            RM_CUDA(cudaMemcpyAsync(ctx->d_table, ctx->h_table, plan.frames.size() * sizeof(FrameDev),
                                    cudaMemcpyHostToDevice, s));
            RM_CUDA(cudaEventRecord(ctx->table_free, s));
            if (!plan.square_direct)
                RM_CUDA(launch_analytic(ctx->d_table, (int)plan.frames.size(), plan.total_lines, plan.max_len,
                                        plan.band_sched, d_frames, ctx->d_gamma, false, s));
            if (plan.cross_groups > 0)
                RM_CUDA(launch_crossband(ctx->d_table, (int)plan.frames.size(), plan.cross_groups, plan.max_kc,
                                         ctx->d_gamma, false, s));
            rc = tune_plan(ctx, plan, d_frames, d_out, d_status, s, force_tune);
            if (rc) return rc;
            for (auto& g : ctx->graphs) drop_graph(ctx, g);  // captured graphs may hold the previous variants
        }
    }

    const bool graph = ctx->p.use_graph && ctx->p.precision == RMUSIC_FP32_BATCHED;
    int launches = 0;
    if (!graph) {
        RM_CUDA(cudaEventSynchronize(ctx->table_free));
        memcpy(ctx->h_table, plan.frames.data(), plan.frames.size() * sizeof(FrameDev));
        RM_CUDA(cudaMemcpyAsync(ctx->d_table, ctx->h_table, plan.frames.size() * sizeof(FrameDev),
                                cudaMemcpyHostToDevice, s));
        RM_CUDA(cudaEventRecord(ctx->table_free, s));
        rc = enqueue(ctx, plan, d_frames, d_out, d_status, s, &launches);
        if (rc) return rc;
        ctx->stats.kernel_launches += launches;
        return RMUSIC_OK;
    }

    // graph path: key = everything the captured work depends on
    std::vector<unsigned char> key;
    auto put = [&](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        key.insert(key.end(), b, b + n);
    };
    put(&d_frames, sizeof(d_frames));
    put(&d_out, sizeof(d_out));
    put(&d_status, sizeof(d_status));
    put(&ctx->p, sizeof(ctx->p));
    put(plan.frames.data(), plan.frames.size() * sizeof(FrameDev));
    for (auto& g : ctx->graphs) {
        if (g.exec && g.key == key) {
            g.stamp = ++ctx->graph_clock;
            ctx->a1_ev.insert(ctx->a1_ev.end(), g.a1_ev.begin(), g.a1_ev.end());
            ctx->solver_ev.insert(ctx->solver_ev.end(), g.solver_ev.begin(), g.solver_ev.end());
            RM_CUDA(cudaGraphLaunch(g.exec, s));
            ctx->stats.kernel_launches += g.launches;
            ctx->stats.graph_replayed = 1;
            return RMUSIC_OK;
        }
    }
    // capture a new graph into the least recently used slot
    GraphEntry* slot = &ctx->graphs[0];
    for (auto& g : ctx->graphs)
        if (!g.exec || g.stamp < slot->stamp) slot = &g;
    drop_graph(ctx, *slot);
    if (cudaMallocHost(&slot->h_table, plan.frames.size() * sizeof(FrameDev)) != cudaSuccess) {
        slot->h_table = nullptr;
        return RMUSIC_ENOMEM;
    }
    memcpy(slot->h_table, plan.frames.data(), plan.frames.size() * sizeof(FrameDev));
    cudaGraph_t graph_def = nullptr;
    const size_t a1_mark = ctx->a1_ev.size(), solver_mark = ctx->solver_ev.size();
    // capture on the context's own stream (the legacy default stream cannot be captured); nothing
    // runs during capture, the graph is launched on the caller's stream below
    cudaStream_t cs = ctx->cap_stream;
    RM_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    ctx->capture_owned = &slot->owned;
    cudaError_t ce = cudaMemcpyAsync(ctx->d_table, slot->h_table, plan.frames.size() * sizeof(FrameDev),
                                     cudaMemcpyHostToDevice, cs);
    int erc = ce == cudaSuccess ? enqueue(ctx, plan, d_frames, d_out, d_status, cs, &launches) : RMUSIC_ECUDA;
    cudaError_t ee = cudaStreamEndCapture(cs, &graph_def);
    ctx->capture_owned = nullptr;
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaMemcpyAsync (capture)");
    if (erc) {
        if (graph_def) cudaGraphDestroy(graph_def);
        return erc;
    }
    if (ee != cudaSuccess) return cuda_fail(ctx, ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&slot->exec, graph_def, 0);
    cudaGraphDestroy(graph_def);
    if (ie != cudaSuccess) {
        slot->exec = nullptr;
        return cuda_fail(ctx, ie, "cudaGraphInstantiate");
    }
    slot->key = std::move(key);
    slot->launches = launches;
    slot->a1_ev.assign(ctx->a1_ev.begin() + a1_mark, ctx->a1_ev.end());
    slot->solver_ev.assign(ctx->solver_ev.begin() + solver_mark, ctx->solver_ev.end());
    slot->stamp = ++ctx->graph_clock;
    RM_CUDA(cudaGraphLaunch(slot->exec, s));
    ctx->stats.kernel_launches += launches;
    return RMUSIC_OK;
}

uint64_t group_bytes(const rmusic_ctx* ctx, const rmusic_frame_desc& d) {
    return (uint64_t)d.height * (uint64_t)d.width * gamma_elem_bytes(ctx);
}

}  // namespace

extern "C" {

int rmusic_create(const rmusic_params* params, int device, size_t hbm_budget_bytes, rmusic_ctx** out) {
    if (!params || !out) return RMUSIC_EINVAL;
    *out = nullptr;
    if (int rc = params_check(*params)) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return ndev == 0 ? RMUSIC_ECUDA : RMUSIC_EINVAL;
    }
    rmusic_ctx* ctx = new (std::nothrow) rmusic_ctx();
    if (!ctx) return RMUSIC_ENOMEM;
    ctx->p = *params;
    ctx->device = device;
    for (int l = 0; l < kKeys; ++l) ctx->variant_by_L[l] = -1;
    ctx->budget = hbm_budget_bytes;
    DeviceGuard guard(device);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = init_analytic();
    if (e == cudaSuccess) e = init_crossband();
    if (e == cudaSuccess) e = init_batched(device);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->table_free, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->call_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_counters, sizeof(unsigned long long) * kCounterSlots);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_counters, 0, sizeof(unsigned long long) * kCounterSlots);
    if (e != cudaSuccess) {
        rmusic_destroy(ctx);
        return RMUSIC_ECUDA;
    }
    ctx->held += sizeof(unsigned long long) * kCounterSlots;
    *out = ctx;
    return RMUSIC_OK;
}

}  // extern "C"

namespace {

int demodulate_impl(rmusic_ctx* ctx, const void* d_frames, const rmusic_frame_desc* descs, int32_t n_frames,
                    float* d_out, uint8_t* d_status, void* cuda_stream, bool force_tune) {
    if (!ctx || n_frames < 0) return RMUSIC_EINVAL;
    ctx->stats.kernel_launches = 0;
    ctx->stats.graph_replayed = 0;
    ctx->a1_ev.clear();
    ctx->solver_ev.clear();
    ctx->ev_used = 0;
    ctx->last_pixels = 0;
    if (n_frames == 0) return RMUSIC_OK;
    if (!d_frames || !descs || !d_out) return RMUSIC_EINVAL;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // validate everything before queueing anything
    uint64_t pixels = 0;
    for (int i = 0; i < n_frames; ++i) {
        FrameDev F;
        int rc = describe(ctx, descs[i], &F);
        if (rc) return rc;
        pixels += (uint64_t)F.H * (uint64_t)F.W;
    }
    RM_CUDA(cudaMemsetAsync(ctx->d_counters + kStatSlot, 0, (kStatSlots + 2) * sizeof(unsigned long long), s));
    // group frames so that each group's analytic signal fits the budget (with room for the frame
    // table when the one held is too small for this call)
    const uint64_t table_reserve =
        ctx->table_cap >= (size_t)n_frames ? 0 : 64 * sizeof(FrameDev) + (uint64_t)n_frames * sizeof(FrameDev);
    uint64_t avail = 0;
    if (ctx->budget) {
        const uint64_t fixed = ctx->held - ctx->gamma_cap + table_reserve;
        avail = ctx->budget > fixed ? ctx->budget - fixed : 0;
    }
    int first = 0;
    while (first < n_frames) {
        int count = 0;
        uint64_t bytes = 0;
        while (first + count < n_frames) {
            const uint64_t b = group_bytes(ctx, descs[first + count]);
            if (ctx->budget && count > 0 && bytes + b > avail) break;
            bytes += b;
            ++count;
        }
        if (ctx->budget && bytes > avail) return RMUSIC_ENOMEM;
        int rc = run_group(ctx, d_frames, descs + first, count, d_out, d_status, s, force_tune);
        if (rc) return rc;
        first += count;
    }
    ctx->stats.workspace_bytes = ctx->held;
    ctx->last_pixels = pixels;
    RM_CUDA(cudaEventRecord(ctx->call_done, s));
    return RMUSIC_OK;
}

}  // namespace

extern "C" {

int rmusic_demodulate_frames(rmusic_ctx* ctx, const void* d_frames, const rmusic_frame_desc* descs,
                             int32_t n_frames, float* d_out, uint8_t* d_status, void* cuda_stream) {
    return demodulate_impl(ctx, d_frames, descs, n_frames, d_out, d_status, cuda_stream, false);
}

int rmusic_autotune(rmusic_ctx* ctx, const void* d_frames, const rmusic_frame_desc* descs, int32_t n_frames,
                    float* d_out, uint8_t* d_status, void* cuda_stream) {
    if (ctx && ctx->p.precision != RMUSIC_FP32_BATCHED) return RMUSIC_EUNSUPPORTED;
    return demodulate_impl(ctx, d_frames, descs, n_frames, d_out, d_status, cuda_stream, true);
}

int rmusic_reserve(rmusic_ctx* ctx, uint64_t max_pixels, int32_t max_frames) {
    if (!ctx || max_frames < 0) return RMUSIC_EINVAL;
    if (ctx->p.unwrap && max_pixels >= (1ull << 31)) return RMUSIC_EINVAL;
    DeviceGuard guard(ctx->device);
    int rc = RMUSIC_OK;
    if (max_frames > 0) rc = ensure_tables(ctx, (size_t)max_frames);
    if (!rc && max_pixels > 0) rc = ensure(ctx, &ctx->d_gamma, &ctx->gamma_cap, max_pixels * gamma_elem_bytes(ctx));
    if (!rc && max_pixels > 0 && ctx->p.unwrap)
        rc = ensure(ctx, &ctx->d_unwrap, &ctx->unwrap_cap,
                    unwrap_workspace_bytes((int64_t)max_pixels, (int64_t)max_pixels));
    ctx->stats.workspace_bytes = ctx->held;
    return rc;
}

}  // extern "C"

namespace {
// Device address of a host buffer the GPU can address directly (pinned, registered or mapped host
// memory: on a Grace-Blackwell node the kernels then read and write it over the coherent
// NVLink-C2C link), or nullptr for pageable memory, which is staged through the device workspace.
void* direct_host_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // an unregistered pointer may report an error: clear it
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

// The host-buffer entries. sync: the maps are complete on return, and pinned frames are read in
// place by the band-pass kernel. Without sync the call only queues the work: the frames are always
// staged by the copy engine, which needs no SM, so a caller alternating two contexts overlaps one
// call's transfer with the other's kernels (reading in place would need the SMs the other call's
// solver holds).
int host_entry(rmusic_ctx* ctx, const void* h_frames, size_t in_bytes, const rmusic_frame_desc* descs,
               int32_t n_frames, float* h_out, uint8_t* h_status, void* cuda_stream, bool sync) {
    if (!ctx || n_frames < 0) return RMUSIC_EINVAL;
    if (n_frames == 0) return RMUSIC_OK;
    if (!h_frames || !descs || !h_out) return RMUSIC_EINVAL;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    uint64_t out_elems = 0, st_elems = 0;
    const int maps = ctx->p.geometry == RMUSIC_GEOM_SQUARE ? 3 + ctx->p.unwrap : 1;  // maps per frame
    for (int i = 0; i < n_frames; ++i) {
        const rmusic_frame_desc& d = descs[i];
        if (d.height < 1 || d.width < 1) return RMUSIC_EINVAL;
        const int esz = d.dtype == RMUSIC_DTYPE_U16 ? 2 : d.dtype == RMUSIC_DTYPE_C64 ? 8 : 4;
        const uint64_t pitch = d.pitch_elems ? (uint64_t)d.pitch_elems : (uint64_t)d.width;
        const uint64_t end = d.offset_bytes + ((uint64_t)(d.height - 1) * pitch + (uint64_t)d.width) * esz;
        if (end > in_bytes) return RMUSIC_EINVAL;
        out_elems = std::max<uint64_t>(out_elems, d.out_offset + (uint64_t)maps * d.height * d.width);
        st_elems = std::max<uint64_t>(st_elems, d.out_offset + (uint64_t)d.height * d.width);
    }
    // Pinned (device-addressable) buffers are used in place: the band-pass reads the frames and the
    // solver writes the maps over the host link while it computes, instead of a copy before and a
    // copy after the kernels. Two solvers' maps are staged on the device instead: the unwrapping
    // pass reads and writes its maps many times (square geometry with phase assembly), and the
    // FP32-batched row solver's lanes each own 16 consecutive pixels, so one of its store
    // instructions writes 32 pixels 64 bytes apart -- merged in the device's L2, but one transaction
    // per pixel over the host link.
    const void* d_in = sync ? direct_host_ptr(h_frames) : nullptr;
    const bool staged_maps = (ctx->p.geometry == RMUSIC_GEOM_SQUARE && ctx->p.unwrap) ||
                             (ctx->p.geometry == RMUSIC_GEOM_ROW && ctx->p.precision == RMUSIC_FP32_BATCHED);
    float* d_out = staged_maps ? nullptr : static_cast<float*>(direct_host_ptr(h_out));
    uint8_t* d_st = nullptr;
    if (d_out && h_status) {
        d_st = static_cast<uint8_t*>(direct_host_ptr(h_status));
        if (!d_st) d_out = nullptr;  // both maps go the same way
    }
    int rc = RMUSIC_OK;
    if (!d_in) rc = ensure(ctx, &ctx->d_in, &ctx->in_cap, std::max<size_t>(in_bytes, 16));
    if (!rc && !d_out) {
        size_t ob = ctx->out_cap;
        void* op = ctx->d_out;
        rc = ensure(ctx, &op, &ob, out_elems * sizeof(float));
        ctx->d_out = (float*)op;
        ctx->out_cap = ob;
    }
    if (!rc && !d_out && h_status) {
        size_t sb = ctx->st_cap;
        void* sp = ctx->d_st;
        rc = ensure(ctx, &sp, &sb, st_elems);
        ctx->d_st = (uint8_t*)sp;
        ctx->st_cap = sb;
    }
    if (rc) return rc;
    if (!d_in) {
        RM_CUDA(cudaMemcpyAsync(ctx->d_in, h_frames, in_bytes, cudaMemcpyHostToDevice, s));
        d_in = ctx->d_in;
    }
    const bool direct_out = d_out != nullptr;
    if (!direct_out) {
        d_out = ctx->d_out;
        d_st = h_status ? ctx->d_st : nullptr;
    }
    rc = rmusic_demodulate_frames(ctx, d_in, descs, n_frames, d_out, d_st, cuda_stream);
    if (rc) return rc;
    if (!direct_out) {
        RM_CUDA(cudaMemcpyAsync(h_out, ctx->d_out, out_elems * sizeof(float), cudaMemcpyDeviceToHost, s));
        if (h_status) RM_CUDA(cudaMemcpyAsync(h_status, ctx->d_st, st_elems, cudaMemcpyDeviceToHost, s));
    }
    if (sync) RM_CUDA(cudaStreamSynchronize(s));
    return RMUSIC_OK;
}

}  // namespace

extern "C" {

int rmusic_demodulate_frames_host(rmusic_ctx* ctx, const void* h_frames, size_t in_bytes,
                                  const rmusic_frame_desc* descs, int32_t n_frames, float* h_out,
                                  uint8_t* h_status, void* cuda_stream) {
    return host_entry(ctx, h_frames, in_bytes, descs, n_frames, h_out, h_status, cuda_stream, true);
}

int rmusic_demodulate_frames_host_async(rmusic_ctx* ctx, const void* h_frames, size_t in_bytes,
                                        const rmusic_frame_desc* descs, int32_t n_frames, float* h_out,
                                        uint8_t* h_status, void* cuda_stream) {
    return host_entry(ctx, h_frames, in_bytes, descs, n_frames, h_out, h_status, cuda_stream, false);
}

int rmusic_set_solver_variant(rmusic_ctx* ctx, int32_t order, int32_t variant) {
    if (!ctx || ctx->p.precision != RMUSIC_FP32_BATCHED) return ctx ? RMUSIC_EUNSUPPORTED : RMUSIC_EINVAL;
    const int key = ctx->p.geometry == RMUSIC_GEOM_SQUARE ? kSquareKey0 + order : row_key(ctx->p, order);
    if (order < 1 || order > kMaxL || key < 0 || key >= kKeys || !solver_supports(key)) return RMUSIC_EINVAL;
    if (variant < -1 || variant >= solver_num_variants(key)) return RMUSIC_EINVAL;
    ctx->variant_by_L[key] = variant;
    for (auto& g : ctx->graphs) drop_graph(ctx, g);  // captured graphs hold the previous variant
    return RMUSIC_OK;
}

int rmusic_unwrap_phase(rmusic_ctx* ctx, const float* d_phase, const rmusic_frame_desc* descs, int32_t n_frames,
                        float* d_out, void* cuda_stream) {
    return rmusic_unwrap_phase_sched(ctx, d_phase, descs, n_frames, d_out, -1, cuda_stream);
}

int rmusic_unwrap_phase_sched(rmusic_ctx* ctx, const float* d_phase, const rmusic_frame_desc* descs, int32_t n_frames,
                              float* d_out, int32_t launched_rounds, void* cuda_stream) {
    if (!ctx || n_frames < 0 || launched_rounds < -1) return RMUSIC_EINVAL;
    if (n_frames == 0) return RMUSIC_OK;
    if (!d_phase || !descs || !d_out) return RMUSIC_EINVAL;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::vector<FrameDev> frames((size_t)n_frames);
    uint64_t npx = 0;
    int64_t maxpx = 0;
    for (int i = 0; i < n_frames; ++i) {
        const rmusic_frame_desc& d = descs[i];
        if (d.height < 1 || d.width < 1) return RMUSIC_EINVAL;
        FrameDev& F = frames[(size_t)i];
        memset(&F, 0, sizeof(F));
        F.H = d.height;
        F.W = d.width;
        F.out_off = d.out_offset;
        F.gam_off = npx;  // first pixel of the frame in the call's pixel numbering
        npx += (uint64_t)d.height * (uint64_t)d.width;
        maxpx = std::max<int64_t>(maxpx, unwrap_frame_nodes(d.height, d.width));
    }
    if (npx >= (1ull << 31)) return RMUSIC_EINVAL;
    int rc = ensure_tables(ctx, frames.size());
    if (!rc) rc = ensure(ctx, &ctx->d_unwrap, &ctx->unwrap_cap, unwrap_workspace_bytes((int64_t)npx, maxpx));
    if (rc) return rc;
    RM_CUDA(cudaEventSynchronize(ctx->table_free));
    memcpy(ctx->h_table, frames.data(), frames.size() * sizeof(FrameDev));
    RM_CUDA(cudaMemcpyAsync(ctx->d_table, ctx->h_table, frames.size() * sizeof(FrameDev), cudaMemcpyHostToDevice, s));
    RM_CUDA(cudaEventRecord(ctx->table_free, s));
    int launches = 0;
    unsigned long long* timeouts = ctx->d_counters + kStatSlot + kWaitSlot;
    RM_CUDA(cudaMemsetAsync(timeouts, 0, sizeof(unsigned long long), s));
    RM_CUDA(launch_unwrap(ctx->d_table, n_frames, (int64_t)npx, maxpx, d_phase, 0, d_out, 0, ctx->d_unwrap,
                          launched_rounds, timeouts, &launches, s));
    ctx->stats.kernel_launches = launches;
    return RMUSIC_OK;
}

void rmusic_destroy(rmusic_ctx* ctx) {
    if (!ctx) return;
    {
        DeviceGuard guard(ctx->device);
        cudaDeviceSynchronize();
        for (auto& g : ctx->graphs) drop_graph(ctx, g);
        for (cudaEvent_t e : ctx->gev_free) cudaEventDestroy(e);
        if (ctx->d_gamma) cudaFree(ctx->d_gamma);
        if (ctx->d_table) cudaFree(ctx->d_table);
        if (ctx->d_counters) cudaFree(ctx->d_counters);
        if (ctx->h_table) cudaFreeHost(ctx->h_table);
        if (ctx->table_free) cudaEventDestroy(ctx->table_free);
        if (ctx->call_done) cudaEventDestroy(ctx->call_done);
        if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
        for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
        if (ctx->d_in) cudaFree(ctx->d_in);
        if (ctx->d_out) cudaFree(ctx->d_out);
        if (ctx->d_st) cudaFree(ctx->d_st);
        if (ctx->d_unwrap) cudaFree(ctx->d_unwrap);
    }
    delete ctx;
}

const char* rmusic_strerror(int code) {
    switch (code) {
        case RMUSIC_OK: return "ok";
        case RMUSIC_EINVAL: return "invalid argument";
        case RMUSIC_ENOMEM: return "out of memory or over the HBM budget";
        case RMUSIC_EUNSUPPORTED: return "unsupported parameters for this path";
        case RMUSIC_ETIMEDOUT: return "device-side wait timed out";
        case RMUSIC_ECUDA: return "CUDA runtime error";
        case RMUSIC_EAGAIN: return "all frame slots of the stream are busy, try again";
        default: return "unknown error";
    }
}

const char* rmusic_last_cuda_error(const rmusic_ctx* ctx) { return ctx ? ctx->last_err : ""; }

int rmusic_checked_build(void) {
#ifdef RMUSIC_CHECKS
    return 1;
#else
    return 0;
#endif
}

int rmusic_get_stats(const rmusic_ctx* ctx_in, rmusic_stats* out) {
    if (!ctx_in || !out) return RMUSIC_EINVAL;
    rmusic_ctx* ctx = const_cast<rmusic_ctx*>(ctx_in);
    DeviceGuard guard(ctx->device);
    *out = ctx->stats;
    out->workspace_bytes = ctx->held;
    out->pixels = ctx->last_pixels;
    RM_CUDA(cudaEventSynchronize(ctx->call_done));
    unsigned long long c[kStatSlots + 2] = {};  // the statistics, the failed index checks, the waits given up
    RM_CUDA(cudaMemcpy(c, ctx->d_counters + kStatSlot, sizeof(c), cudaMemcpyDeviceToHost));
    auto mean = [&](int i) { return c[2] ? (double)c[i] / (double)c[2] : 0.0; };
    out->mean_sweeps = mean(0);
    out->mean_root_iters = mean(1);
    out->mean_root_updates = mean(3);
    out->mean_root_evals = mean(4);
    out->mean_power_steps = mean(5);
    out->eig_fallback_frac = mean(6);
    out->mean_newton_steps = mean(7);
    out->root_fallback_frac = mean(8);
    out->mean_polish_steps = mean(9);
    out->check_violations = c[kCheckSlot];
    out->wait_timeouts = c[kWaitSlot];
    auto sum = [&](const std::vector<cudaEvent_t>& v) {
        float t = 0.f;
        for (size_t i = 0; i + 1 < v.size(); i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, v[i], v[i + 1]) == cudaSuccess) t += ms;
        }
        return t;
    };
    out->bandpass_ms = sum(ctx->a1_ev);
    out->solver_ms = sum(ctx->solver_ev);
    return RMUSIC_OK;
}

}  // extern "C"
