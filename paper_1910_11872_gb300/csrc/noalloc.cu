// noalloc.cu -- rmusic_demodulate_frames_noalloc: the FP32-batched path for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all: code running where the allocator is owned by
// someone else (a host framework with its own memory pool, an audited real-time loop that
// forbids allocation after start-up, a plug-in whose host must account for every byte). The
// regular entry points need a context from rmusic_create, whose workspaces come from
// cudaMalloc. This entry point needs none: every piece of device scratch it uses -- the
// complex64 analytic signal of the frames, the frame table and the work counters -- lives in
// one file-scope __device__ array of fixed size. The caller still passes the frames and the
// output maps.
//
// The array is part of this library's device code: a GPU holds it (about 32 MiB) from the moment
// the library's code for this file is loaded on that GPU -- with CUDA's default lazy loading that
// is the first call of this entry point there -- until the process exits. Its address is looked
// up once per device with cudaGetSymbolAddress; in host code the array's name is only a stand-in
// and must never be handed to a kernel.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/rmusic.h"
#include "rmusic_device.cuh"
#include "rmusic_launch.h"
#include "rmusic_validate.h"

using namespace rmusic;

namespace {

constexpr uint64_t kNaMaxPixels = 4ull << 20;  // 4,194,304 pixels, e.g. four 1024 x 1024 frames
constexpr int kNaMaxFrames = 256;
constexpr int kNaMaxDevices = 64;
constexpr size_t kNaGammaBytes = kNaMaxPixels * sizeof(float2);
constexpr size_t kNaTableOff = kNaGammaBytes;
constexpr size_t kNaTableBytes = ((kNaMaxFrames * sizeof(FrameDev) + 255) / 256) * 256;
constexpr size_t kNaCounterOff = kNaTableOff + kNaTableBytes;
constexpr size_t kNaCounterSlots = 16;
constexpr size_t kNaScratchBytes = kNaCounterOff + kNaCounterSlots * sizeof(unsigned long long);

}  // namespace

// The fixed scratch shared by every call of rmusic_demodulate_frames_noalloc on a device.
static __device__ __align__(256) unsigned char rmusic_noalloc_scratch[kNaScratchBytes];

namespace {

std::mutex g_setup_mu;
void* g_scratch[kNaMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (which must be current), looked up once.
int scratch_address(int device, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, rmusic_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return RMUSIC_ECUDA;
        }
        if (init_analytic() != cudaSuccess) {
            cudaGetLastError();
            return RMUSIC_ECUDA;
        }
        g_scratch[device] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch[device]);
    return RMUSIC_OK;
}

}  // namespace

extern "C" int rmusic_demodulate_frames_noalloc(const rmusic_params* params, int device, const void* d_frames,
                                                const rmusic_frame_desc* descs, int32_t n_frames, float* d_out,
                                                uint8_t* d_status, void* cuda_stream) {
    if (!params || n_frames < 0) return RMUSIC_EINVAL;
    const rmusic_params& p = *params;
    // the checks every entry point makes (the codes rmusic_create returns), then what this entry
    // point adds: only the FP32-batched row-window path with the forward-backward average, without
    // the 2-D band-pass or raw input
    if (int rc = params_check(p)) return rc;
    if (p.precision != RMUSIC_FP32_BATCHED || p.geometry != RMUSIC_GEOM_ROW || p.forward_backward != 1 ||
        p.band_cross != 0.0 || p.raw_input != 0)
        return RMUSIC_EUNSUPPORTED;
    if (n_frames == 0) return RMUSIC_OK;
    if (!d_frames || !descs || !d_out) return RMUSIC_EINVAL;
    if (n_frames > kNaMaxFrames) return RMUSIC_ENOMEM;
    if (device < 0 || device >= kNaMaxDevices) return RMUSIC_EINVAL;

    // frame table on the host stack, grouped by covariance order
    FrameDev table[kNaMaxFrames];
    uint64_t pixels = 0;
    for (int i = 0; i < n_frames; ++i) {
        int rc = describe_frame(p, descs[i], &table[i]);
        if (rc) return rc;
        pixels += (uint64_t)table[i].H * (uint64_t)table[i].W;
    }
    if (pixels > kNaMaxPixels) return RMUSIC_ENOMEM;
    std::stable_sort(table, table + n_frames, [](const FrameDev& a, const FrameDev& b) { return a.L < b.L; });
    int group_L[kMaxL + 1], group_first[kMaxL + 1], group_count[kMaxL + 1];
    int64_t group_items[kMaxL + 1];
    int ngroups = 0;
    uint64_t goff = 0;
    int64_t lines = 0;  // band-pass CTAs
    int band_sched = 0;
    int max_len = 0;
    for (int i = 0; i < n_frames; ++i) {
        FrameDev& F = table[i];
        F.gam_off = goff;
        goff += (uint64_t)F.H * (uint64_t)F.W;
        F.line_start = lines;
        lines += band_assign(&F, false);
        band_sched |= band_schedule_bit(F);
        max_len = std::max(max_len, F.len);
        if (i == 0 || F.L != table[i - 1].L) {
            group_L[ngroups] = F.L;
            group_first[ngroups] = i;
            group_count[ngroups] = 0;
            group_items[ngroups] = 0;
            ++ngroups;
        }
        F.item_start = group_items[ngroups - 1];
        group_items[ngroups - 1] += (int64_t)F.wlines * F.nchunks;
        group_count[ngroups - 1] += 1;
    }

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return RMUSIC_ECUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return RMUSIC_EINVAL;
    int rc = RMUSIC_OK;
    do {
        unsigned char* base = nullptr;
        rc = scratch_address(device, &base);
        if (rc) break;
        float2* gamma = reinterpret_cast<float2*>(base);
        FrameDev* d_table = reinterpret_cast<FrameDev*>(base + kNaTableOff);
        unsigned long long* counters = reinterpret_cast<unsigned long long*>(base + kNaCounterOff);
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        // the table comes from pageable host memory: the copy is staged before the call returns
        if (cudaMemcpyAsync(d_table, table, sizeof(FrameDev) * (size_t)n_frames, cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
            rc = RMUSIC_ECUDA;
            break;
        }
        // the work counters must start at zero; the rest of the scratch is fully overwritten
        if (cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * (size_t)ngroups, s) != cudaSuccess) {
            rc = RMUSIC_ECUDA;
            break;
        }
        if (launch_analytic(d_table, n_frames, lines, max_len, band_sched, d_frames, gamma, false, s) != cudaSuccess) {
            rc = RMUSIC_ECUDA;
            break;
        }
        BatchedArgs a;
        a.max_sweeps = p.max_sweeps ? p.max_sweeps : 6;
        a.max_iters = p.max_root_iters ? p.max_root_iters : 16;
        a.polish64 = p.polish_fp64;
        a.exhaustive = p.exhaustive;
        a.counters = nullptr;
        a.fb = 1;
        for (int g = 0; g < ngroups && rc == RMUSIC_OK; ++g) {
            const int L = group_L[g];
            const int v = batched_default_variant(L);
            if (launch_batched(L, v, d_table + group_first[g], group_count[g], group_items[g], counters + g, gamma,
                               d_out, d_status, a, batched_grid(L, v, device), s) != cudaSuccess)
                rc = RMUSIC_ECUDA;
        }
    } while (0);
    if (prev != device) cudaSetDevice(prev);
    return rc;
}
