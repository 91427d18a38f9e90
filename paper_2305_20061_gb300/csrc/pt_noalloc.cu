// Rendering without device allocation.
//
// pt_render keeps its wavefront scratch (ray queues, escape records,
// per-path radiance) in device memory that the context allocates with
// cudaMalloc on first use.  Some callers cannot let a library allocate
// device memory at render time: a host application that hands out all of
// its GPU memory at start-up from its own pool and forbids further
// cudaMalloc calls, or a real-time loop that must never hit the driver's
// allocator (which can synchronise the device).  pt_render_noalloc serves
// them: it renders the same image as pt_render with the FP32 network, but its
// scratch lives in one fixed array in this file's device memory, sized for
// kMaxSlots paths per wavefront chunk.  It calls no cudaMalloc, cudaFree or
// allocating library routine.
//
// The array exists once per GPU that loads the library and stays until the
// process exits.  Its address is looked up (and the array reserved by the
// driver) when pt_create makes a context on the device, before any render
// call.  Every call shares it, so calls whose GPU work overlaps (on two
// streams, or from two threads) race and corrupt each other's results;
// serialise them on one stream.  The cached address does not survive a
// cudaDeviceReset, after which no object of this library is valid anyway.
#include <algorithm>
#include <mutex>

#include <cuda_runtime.h>

#include "pt_internal.h"

namespace ptk {
namespace {

constexpr uint32_t kMaxSlots = 1u << 18;   // paths per chunk; the frame must have <= this many pixels
constexpr int kMaxDepthNA = 64;
constexpr size_t kHeaderBytes = 2048;      // counters (128 x u32), stats (65 x u64), error word
constexpr size_t kBytesPerSlot = 2 * 4 * sizeof(float4) + kEscapeBytes + sizeof(int2) + 3 * sizeof(float);  // 172
constexpr size_t kScratchBytes = kHeaderBytes + (size_t)kMaxSlots * kBytesPerSlot;            // ~43 MiB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[kMaxDevices] = {};

}  // namespace

// Device address of g_scratch on `device` (which must be current), looked up
// once per device.  pt_create calls this for its device: the lookup is where
// the driver loads this file's module and reserves the array (under lazy
// module loading that would otherwise happen inside the first render call),
// so pt_render_noalloc itself only reads the cached address.
cudaError_t noalloc_setup(int device, unsigned char** out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_dev_ptr[device] = static_cast<unsigned char*>(p);
    }
    if (out) *out = g_dev_ptr[device];
    return cudaSuccess;
}

namespace {
}  // namespace
}  // namespace ptk

using namespace ptk;

extern "C" PT_API pt_status pt_render_noalloc(const pt_scene* scene, const pt_nif* nif, const pt_render_cfg* cfg,
                                              float* d_image, uint32_t* d_err, void* stream)
{
    if (!scene || !cfg || !d_image) return PT_EINVAL;
    int scene_device = 0;
    const DevScene* sv = scene_view(scene, &scene_device);
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return PT_ECUDA;
    if (device != scene_device || device < 0 || device >= kMaxDevices) return PT_EINVAL;
    if (cfg->width < 1 || cfg->height < 1 || cfg->spp < 1 || cfg->max_depth < 1 || cfg->max_depth > kMaxDepthNA ||
        cfg->first_sample < 0 || (cfg->rr && cfg->rr_start < 1))
        return PT_EINVAL;
    const int64_t n_pix = (int64_t)cfg->width * cfg->height;
    if (n_pix > (int64_t)kMaxSlots) return PT_EINVAL;   // one sample of the frame must fit the fixed scratch
    if (sv->env_is_nif && !nif) return PT_EINVAL;
    if (sv->env_is_nif && cfg->precision != PT_FP32) return PT_EUNSUPPORTED;
    if (cfg->cache_vertex != 0) return PT_EUNSUPPORTED;   // no radiance cache on this path
    const int64_t n_slots = n_pix * (int64_t)cfg->spp;
    if (n_slots > 0xFFFFFFFFll) return PT_EINVAL;

    unsigned char* base = nullptr;
    if (noalloc_setup(device, &base) != cudaSuccess) return PT_ECUDA;
    uint32_t* counters = reinterpret_cast<uint32_t*>(base);
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(base + 512);
    uint32_t* err = d_err ? d_err : reinterpret_cast<uint32_t*>(base + 1536);
    unsigned char* p = base + kHeaderBytes;
    RayQueue q[2];
    for (auto& qq : q) {
        qq.o = reinterpret_cast<float4*>(p); p += (size_t)kMaxSlots * sizeof(float4);
        qq.d = reinterpret_cast<float4*>(p); p += (size_t)kMaxSlots * sizeof(float4);
        qq.tp = reinterpret_cast<float4*>(p); p += (size_t)kMaxSlots * sizeof(float4);
        qq.L = reinterpret_cast<float4*>(p); p += (size_t)kMaxSlots * sizeof(float4);
    }
    EscapeQueue esc;
    esc.uv = reinterpret_cast<float2*>(p); p += (size_t)kMaxSlots * sizeof(float2);
    esc.tp = reinterpret_cast<float4*>(p); p += (size_t)kMaxSlots * sizeof(float4);
    int2* hits = reinterpret_cast<int2*>(p); p += (size_t)kMaxSlots * sizeof(int2);
    float* slot_L = reinterpret_cast<float*>(p);

    int sm_count = 0;
    if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PT_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // whole samples per chunk
    const int64_t chunk = std::min<int64_t>(n_slots, ((int64_t)kMaxSlots / n_pix) * n_pix);

    BounceParams bp = {};
    bp.sc = *sv;
    bp.sc.aspect = (float)((double)cfg->width / (double)cfg->height);
    bp.max_depth = cfg->max_depth;
    bp.rr = cfg->rr;
    bp.rr_start = cfg->rr_start;
    bp.seed = cfg->seed;
    bp.first_sample = (uint32_t)cfg->first_sample;
    bp.n_pix = (uint32_t)n_pix;
    bp.pixels = nullptr;
    bp.W = cfg->width;
    bp.H = cfg->height;
    bp.esc = esc;
    bp.esc_count = counters + kMaxDepthNA + 2;
    bp.slot_L = slot_L;
    bp.hit_ids = nullptr;
    bp.err = err;
    bp.stats = stats;
    bp.cap = (uint32_t)chunk;
    bp.hits = hits;
    bp.fetch = counters + kMaxDepthNA + 4;
    const int64_t n_chunks = (n_slots + chunk - 1) / chunk;
    for (int64_t c = 0; c < n_chunks; ++c) {
        const int64_t first = c * chunk;
        const int64_t n = std::min(chunk, n_slots - first);
        // the array keeps the previous call's contents: queue counters must start at zero
        if (cudaMemsetAsync(counters, 0, 128 * sizeof(uint32_t), s) != cudaSuccess) return PT_ECUDA;
        bp.chunk_first = (uint64_t)first;
        bp.n_chunk = (uint32_t)n;
        for (int k = 1; k <= cfg->max_depth; ++k) {
            bp.k = k;
            bp.qin = q[(k + 1) & 1];
            bp.qout = q[k & 1];
            bp.count_in = counters + (k - 1);
            bp.count_out = counters + k;
            if (launch_bounce(bp, sm_count, s) != cudaSuccess) return PT_ECUDA;
        }
        if (sv->env_is_nif) {
            NifEvalParams np = {};
            np.nif = *nif_view(nif);
            np.esc = esc;
            np.esc_count = counters + kMaxDepthNA + 2;
            np.esc_cap = (uint32_t)chunk;
            np.accumulate = sv->has_emission;
            np.slot_L = slot_L;
            np.err = err;
            np.stats = stats + cfg->max_depth;
            if (launch_nif_fp32(np, 1, sm_count, s) != cudaSuccess) return PT_ECUDA;
        }
        const float scale = (c == n_chunks - 1) ? (float)(1.0 / cfg->spp) : 1.f;
        if (launch_reduce(slot_L, d_image, (uint32_t)n_pix, (uint32_t)(n / n_pix), c == 0, scale, s) != cudaSuccess)
            return PT_ECUDA;
    }
    return PT_OK;
}
