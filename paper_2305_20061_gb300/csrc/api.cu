// C ABI of the path tracer (include/pt.h): argument checking, device
// memory of scenes / networks / wavefront scratch, and the render loop that
// alternates traversal-and-shading steps with batched NIF evaluation
// (Section 3.3).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "pt_internal.h"

using namespace ptk;

struct pt_ctx {
    int device = 0;
    int sm_count = 0;
    int paths_threads[3] = {0, 0, 0};   // resident threads of the path kernel (packed, decoded, quantised nodes)
    std::string last_error;
    uint32_t* d_err = nullptr;
    // wavefront scratch
    uint32_t chunk_cap = 0;
    RayQueue q[2] = {};
    EscapeQueue esc = {};
    float* slot_L = nullptr;
    uint32_t* counters = nullptr;          // [kCounters]
    unsigned long long* stats = nullptr;   // [kMaxDepth + 1]
    int2* hits = nullptr;                  // traversal results [chunk_cap]
    float* cache_rows = nullptr;           // radiance-cache query rows [cache_cap][16]
    uint32_t cache_cap = 0;
    int last_depth = 0;
    int last_schedule = PT_SCHED_AUTO;    // schedule the last render's last chunk ran with
    // non-blocking stream of the host-array uploads (scene, weights, cache): an upload does not wait for
    // renders queued on the caller's streams, so the next scene can be built while the GPU renders
    cudaStream_t upload = nullptr;
    // kernel timing (pt_profile_enable)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;      // pairs: start, stop
    std::vector<int> prof_kind;
    size_t prof_used = 0;
    // CUDA graphs of render launch sequences (replayed when a render repeats with the same buffers)
    uint64_t scratch_gen = 0;              // bumped whenever a scratch buffer moves
    uint32_t* d_first_sample = nullptr;    // the sample offset the bounce kernels read
    cudaStream_t cap_stream = nullptr;     // capture stream (captures record, nothing runs on it)
    struct CachedGraph {
        std::vector<unsigned char> key;
        cudaGraphExec_t exec;
        unsigned long long kernels;   // kernels one replay launches
    };
    std::vector<CachedGraph> graphs;
    size_t graph_next = 0;
    std::vector<std::vector<unsigned char>> graph_seen;   // keys seen once (captured on their second use)
    size_t seen_next = 0;
};

namespace ptk {
std::atomic<unsigned long long> g_kernels_launched{0};
thread_local unsigned long long t_kernels_launched = 0;
}  // namespace ptk

// identities that are never reused (a graph key must not match a new object at a recycled address)
std::atomic<uint64_t> g_next_uid{1};

struct pt_scene {
    pt_ctx* ctx = nullptr;
    uint64_t uid = g_next_uid++;
    DevScene dev = {};
    pt_scene_info info = {};
    std::vector<void*> allocs;
};

struct pt_nif {
    pt_ctx* ctx = nullptr;
    uint64_t uid = g_next_uid++;
    uint64_t version = 0;        // bumped when host-side copies (colour matrix) change
    int32_t F = 0, H = 0, L = 0;
    int32_t skip = 0;             // hidden layer joined with the features (1-based), 0: none
    int64_t n_params = 0;
    unsigned char* d_arena = nullptr;   // one allocation holding d_params, d_fp32 and d_tc
    float* d_params = nullptr;   // flat FP32 master weights
    float* d_fp32 = nullptr;     // packed FP32 layout (Wt, bias, Wout, bout)
    unsigned char* d_tc = nullptr;  // BF16 shared-memory image of the tensor-core kernel (F=64, H=128, L=1..5)
    // FP8 E4M3 image of the same shape, built on first use (its calibration runs on the host) and
    // rebuilt on the next use after the weights change
    bool fp8_ok = false;
    mutable unsigned char* d_fp8 = nullptr;
    mutable bool fp8_stale = true;
    mutable float fp8_scales[4] = {0, 0, 0, 0};
    DevNif dev = {};
    // training state (allocated by the first training call)
    int64_t n_trainable = 0;
    float* d_grad = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    int64_t adam_t = 0;             // Adam steps taken; also the Philox step counter of the samples
    int64_t work_cap = 0;           // batch rows the work buffers hold
    void* d_work = nullptr;         // activations, gradients, partials
    TrainWork work = {};
    float* d_batch = nullptr;       // uv [cap][2] + target [cap][3] for pt_train_nif
    double* d_loss = nullptr;
};

struct pt_cache {
    pt_ctx* ctx = nullptr;
    uint64_t uid = g_next_uid++;
    int32_t J = 0, H = 0, L = 0, in0 = 0;
    int64_t n_params = 0;
    float* d_params = nullptr;      // flat FP32 weights (pt_cache_desc layout)
    unsigned char* d_tc = nullptr;  // BF16 tensor-core image (J = 12, H = 64, L = 5 only), follows d_params
    CacheBox box = {};
    float box_lo[3] = {0, 0, 0}, box_hi[3] = {0, 0, 0};   // the box as given (checkpoints)
    // online training state
    float* d_grad = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    int64_t adam_t = 0;
    int64_t work_cap = 0;
    void* d_work = nullptr;
    TrainWork work = {};
    int64_t train_cap = 0;          // training paths the buffers below hold
    void* d_train = nullptr;        // one allocation: pixels, records, radiance, targets, mask
    int64_t* d_pixels = nullptr;
    float* d_rec = nullptr;         // [n][16]
    float* d_Lpath = nullptr;       // [n][3]
    float* d_target = nullptr;      // [n][3]
    int32_t* d_mask = nullptr;      // [n]
    double* d_loss = nullptr;
};

namespace {

constexpr int kMaxDepth = 64;
constexpr int kCounters = kMaxDepth + 8;
constexpr int kEscCounter = kMaxDepth + 2;
constexpr int kCacheCounter = kMaxDepth + 3;
constexpr int kFetchCounter = kMaxDepth + 4;
constexpr int kStats = kMaxDepth + 1 + 4 + 1; // rays per vertex, NIF evaluations, traversal work [4], cache queries
constexpr int kCacheStat = kMaxDepth + 5;
constexpr int kWorkBase = kMaxDepth + 1;

pt_status fail(pt_ctx* ctx, pt_status st, const std::string& msg)
{
    if (ctx) ctx->last_error = msg;
    // a failed allocation leaves its (non-sticky) error pending in the runtime, where the next call's launch
    // check would report it: consume it here
    if (st == PT_ENOMEM) (void)cudaGetLastError();
    return st;
}

// Copies host memory to the device on the context's upload stream and waits
// for it: the copy is complete on return, and it does not wait for work queued
// on the legacy default stream or the caller's streams.
cudaError_t upload_host(pt_ctx* ctx, void* dst, const void* src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->upload);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->upload);
    return e;
}

// Runs the body of an entry point that builds large host arrays or starts host
// threads: a failed host allocation or thread start becomes PT_ENOMEM instead
// of an exception crossing the C ABI.
template <class F>
pt_status no_throw(pt_ctx* ctx, F&& body)
{
    try {
        return body();
    } catch (const std::bad_alloc&) {
        return fail(ctx, PT_ENOMEM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(ctx, PT_ENOMEM, std::string("host resources exhausted: ") + e.what());
    }
}

pt_status cuda_fail(pt_ctx* ctx, cudaError_t e, const char* what)
{
    (void)cudaGetLastError();   // consume a non-sticky error so that it is not reported again by the next call
    return fail(ctx, e == cudaErrorMemoryAllocation ? PT_ENOMEM : PT_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define PT_CUDA(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

void free_scratch(pt_ctx* ctx)
{
    for (auto& q : ctx->q) {
        cudaFree(q.o); cudaFree(q.d); cudaFree(q.tp); cudaFree(q.L);
        q = RayQueue{};
    }
    cudaFree(ctx->esc.uv); cudaFree(ctx->esc.tp); ctx->esc = EscapeQueue{};
    cudaFree(ctx->slot_L); ctx->slot_L = nullptr;
    cudaFree(ctx->hits); ctx->hits = nullptr;
    ctx->chunk_cap = 0;
    cudaFree(ctx->cache_rows); ctx->cache_rows = nullptr;
    ctx->cache_cap = 0;
}

pt_status ensure_scratch(pt_ctx* ctx, uint32_t chunk)
{
    if (ctx->chunk_cap >= chunk) return PT_OK;
    free_scratch(ctx);
    for (auto& q : ctx->q) {
        if (dalloc(&q.o, chunk) || dalloc(&q.d, chunk) || dalloc(&q.tp, chunk) || dalloc(&q.L, chunk)) {
            free_scratch(ctx);
            return fail(ctx, PT_ENOMEM, "wavefront queue allocation failed");
        }
    }
    if (dalloc(&ctx->esc.uv, chunk) || dalloc(&ctx->esc.tp, chunk) || dalloc(&ctx->slot_L, (size_t)chunk * 3) ||
        dalloc(&ctx->hits, chunk)) {
        free_scratch(ctx);
        return fail(ctx, PT_ENOMEM, "escape queue allocation failed");
    }
    ctx->chunk_cap = chunk;
    ++ctx->scratch_gen;
    return PT_OK;
}

bool finite3(const float* p, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

void camera_basis(const float cam[10], DevScene& d)
{
    const double eye[3] = {cam[0], cam[1], cam[2]};
    double f[3] = {cam[3] - eye[0], cam[4] - eye[1], cam[5] - eye[2]};
    const double up[3] = {cam[6], cam[7], cam[8]};
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (double& x : f) x /= fl;
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (double& x : r) x /= rl;
    const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    for (int a = 0; a < 3; ++a) {
        d.eye[a] = (float)eye[a];
        d.fwd[a] = (float)f[a];
        d.right[a] = (float)r[a];
        d.up[a] = (float)u[a];
    }
    d.tan_half = (float)std::tan(0.5 * (double)cam[9] * 3.14159265358979323846 / 180.0);
    d.aspect = 1.f;
}

// Run one kernel launch, bracketed by a CUDA event pair on its stream when
// profiling is enabled.
template <typename F>
cudaError_t timed(pt_ctx* ctx, int kind, cudaStream_t s, F&& launch)
{
    if (!ctx->prof_on) return launch();
    if (ctx->prof_used * 2 + 2 > ctx->prof_ev.size()) {
        for (int i = 0; i < 2; ++i) {
            cudaEvent_t e;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
            ctx->prof_ev.push_back(e);
        }
        ctx->prof_kind.push_back(0);
    }
    const size_t i = ctx->prof_used++;
    ctx->prof_kind[i] = kind;
    cudaError_t r = cudaEventRecord(ctx->prof_ev[2 * i], s);
    if (r != cudaSuccess) return r;
    r = launch();
    if (r != cudaSuccess) return r;
    return cudaEventRecord(ctx->prof_ev[2 * i + 1], s);
}

pt_status check_cfg(pt_ctx* ctx, const pt_scene* scene, const pt_nif* nif, const pt_render_cfg* cfg)
{
    if (!ctx || !scene || !cfg) return fail(ctx, PT_EINVAL, "null argument");
    if (cfg->width < 1 || cfg->height < 1 || cfg->spp < 1) return fail(ctx, PT_EINVAL, "image size and spp must be >= 1");
    if (cfg->max_depth < 1 || cfg->max_depth > kMaxDepth) return fail(ctx, PT_EINVAL, "max_depth must be in [1, 64]");
    if ((int64_t)cfg->width * cfg->height > (1ll << 31)) return fail(ctx, PT_EINVAL, "image too large");
    if (cfg->rr && cfg->rr_start < 1) return fail(ctx, PT_EINVAL, "rr_start must be >= 1");
    if (cfg->first_sample < 0) return fail(ctx, PT_EINVAL, "first_sample must be >= 0");
    if (cfg->schedule < PT_SCHED_AUTO || cfg->schedule > PT_SCHED_PATHS) return fail(ctx, PT_EINVAL, "unknown schedule");
    if (scene->dev.env_is_nif && !nif) return fail(ctx, PT_EINVAL, "scene environment is a NIF but no NIF was given");
    if (cfg->precision != PT_FP32 && cfg->precision != PT_BF16 && cfg->precision != PT_FP8E4M3)
        return fail(ctx, PT_EINVAL, "unknown precision");
    return PT_OK;
}

// Builds (or rebuilds after a weight change) the FP8 image: the calibration of
// its activation scales runs on the host, so the master weights round-trip.
pt_status ensure_fp8(pt_ctx* ctx, const pt_nif* nf, cudaStream_t s)
{
    if (!nf->fp8_ok) return fail(ctx, PT_EUNSUPPORTED, "the FP8 NIF needs F = 64, H = 128, L = 3");
    if (nf->d_fp8 && !nf->fp8_stale) return PT_OK;
    std::vector<float> host(nf->n_params);
    std::vector<unsigned char> img;
    PT_CUDA(cudaMemcpyAsync(host.data(), nf->d_params, host.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    PT_CUDA(cudaStreamSynchronize(s));
    if (!pack_nif_fp8_image(host.data(), nf->F, nf->H, nf->L, img, nf->fp8_scales))
        return fail(ctx, PT_EINVAL, "FP8 packing failed");
    if (!nf->d_fp8 && cudaMalloc((void**)&nf->d_fp8, img.size()) != cudaSuccess)
        return fail(ctx, PT_ENOMEM, "NIF FP8 image allocation failed");
    PT_CUDA(cudaMemcpyAsync(nf->d_fp8, img.data(), img.size(), cudaMemcpyHostToDevice, s));
    PT_CUDA(cudaStreamSynchronize(s));
    nf->fp8_stale = false;
    return PT_OK;
}

pt_status eval_nif_escapes(pt_ctx* ctx, const pt_nif* nif, int precision, int accumulate, cudaStream_t s)
{
    NifEvalParams p = {};
    p.nif = nif->dev;
    p.esc = ctx->esc;
    p.esc_count = ctx->counters + kEscCounter;
    p.esc_cap = ctx->chunk_cap;
    p.accumulate = accumulate;
    p.slot_L = ctx->slot_L;
    p.err = ctx->d_err;
    p.stats = ctx->stats + ctx->last_depth;
    if (precision == PT_FP32) {
        PT_CUDA(timed(ctx, PT_KIND_NIF, s, [&] { return launch_nif_fp32(p, 1, ctx->sm_count, s); }));
        return PT_OK;
    }
    if (precision == PT_BF16 && nif->d_tc) {
        PT_CUDA(timed(ctx, PT_KIND_NIF, s, [&] { return launch_nif_tc(nif->d_tc, nif->F, nif->H, nif->L, nif->skip, p, 1, ctx->sm_count, s); }));
        return PT_OK;
    }
    if (precision == PT_FP8E4M3 && nif->fp8_ok) {
        const pt_status st = ensure_fp8(ctx, nif, s);
        if (st != PT_OK) return st;
        PT_CUDA(timed(ctx, PT_KIND_NIF, s, [&] { return launch_nif_fp8(nif->d_fp8, p, 1, ctx->sm_count, s); }));
        return PT_OK;
    }
    return fail(ctx, PT_EUNSUPPORTED, "no BF16 kernel for this NIF shape (F = 64 with H = 128 and L <= 5, H = 64 or 32 and L <= 8, H = 256 and L = 1; the paper's F = 20 skip network); FP8: F = 64, H = 128, L = 3");
}

}  // namespace

// Read-only views of the opaque handles for other translation units.
namespace ptk {
const DevScene* scene_view(const pt_scene* s, int* device) { if (device) *device = s->ctx->device; return &s->dev; }
const DevNif* nif_view(const pt_nif* n) { return &n->dev; }
}  // namespace ptk

// ---------------------------------------------------------------------------
extern "C" {

PT_API pt_status pt_create(pt_ctx** out, int device)
{
    if (!out) return PT_EINVAL;
    *out = nullptr;
    pt_ctx* ctx = new pt_ctx();
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_err, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->counters, kCounters * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->stats, kStats * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->stats, 0, kStats * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_first_sample, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->upload, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        for (int f = 0; f < 3; ++f) ctx->paths_threads[f] = paths_resident_threads(f, ctx->sm_count);
    }
    // the no-allocation render path's fixed scratch: resolved here so that the driver reserves it now,
    // not inside a later pt_render_noalloc call
    if (e == cudaSuccess) e = noalloc_setup(device, nullptr);
    if (e != cudaSuccess) {
        cudaFree(ctx->d_err);
        cudaFree(ctx->counters);
        cudaFree(ctx->stats);
        cudaFree(ctx->d_first_sample);
        if (ctx->upload) cudaStreamDestroy(ctx->upload);
        delete ctx;
        return PT_ECUDA;
    }
    *out = ctx;
    return PT_OK;
}

PT_API void pt_destroy(pt_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    free_scratch(ctx);
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->upload) cudaStreamDestroy(ctx->upload);
    cudaFree(ctx->d_err);
    cudaFree(ctx->counters);
    cudaFree(ctx->stats);
    cudaFree(ctx->d_first_sample);
    delete ctx;
}

PT_API const char* pt_last_error(const pt_ctx* ctx)
{
    if (!ctx) return "no context (pt_create failed or was not called)";
    return ctx->last_error.c_str();
}

PT_API pt_status pt_check(pt_ctx* ctx, void* stream, uint32_t* bits)
{
    if (!ctx) return PT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    PT_CUDA(cudaStreamSynchronize(s));
    PT_CUDA(cudaGetLastError());
    uint32_t h = 0;
    PT_CUDA(cudaMemcpy(&h, ctx->d_err, sizeof(h), cudaMemcpyDeviceToHost));
    PT_CUDA(cudaMemset(ctx->d_err, 0, sizeof(uint32_t)));
    if (bits) *bits = h;
    if (h) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "device error word 0x%x", h);
        return fail(ctx, PT_EDEVICE, buf);
    }
    return PT_OK;
}

PT_API uint32_t pt_device_error_bits(pt_ctx* ctx)
{
    if (!ctx) return PT_ERR_UNREADABLE;
    uint32_t h = 0;
    if (cudaSetDevice(ctx->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&h, ctx->d_err, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
        (void)cudaGetLastError();
        return PT_ERR_UNREADABLE;
    }
    return h;
}

// ---------------------------------------------------------------------------
static pt_status create_scene(pt_ctx* ctx, const pt_scene_desc* d, pt_scene** out)
{
    if (!ctx || !d || !out) return fail(ctx, PT_EINVAL, "null argument");
    *out = nullptr;
    if (d->n_spheres < 0 || d->n_quads < 0 || d->n_tris < 0 || d->n_verts < 0 || d->n_mats < 1)
        return fail(ctx, PT_EINVAL, "negative counts or no materials");
    const int64_t nS = d->n_spheres, nQ = d->n_quads, nT = d->n_tris, nP = nS + nQ + nT;
    if (nP >= (int64_t)kLeafBit - 1) return fail(ctx, PT_EINVAL, "too many primitives");
    if ((nS && (!d->spheres || !d->sphere_mat)) || (nQ && (!d->quads || !d->quad_axis || !d->quad_mat)) ||
        (nT && (!d->tris || !d->tri_mat || !d->verts)) || !d->mat_type || !d->mats)
        return fail(ctx, PT_EINVAL, "missing primitive arrays");
    if (!finite3(d->spheres, 4 * nS) || !finite3(d->quads, 5 * nQ) || !finite3(d->verts, 3 * d->n_verts) ||
        !finite3(d->mats, 8 * d->n_mats) || !finite3(d->camera, 10))
        return fail(ctx, PT_EINVAL, "non-finite scene values");
    for (int64_t i = 0; i < d->n_mats; ++i)
        if (d->mat_type[i] < 0 || d->mat_type[i] > 2) return fail(ctx, PT_EINVAL, "unknown material type");
    auto bad_mat = [&](const int32_t* m, int64_t n) {
        for (int64_t i = 0; i < n; ++i)
            if (m[i] < 0 || m[i] >= d->n_mats) return true;
        return false;
    };
    if (bad_mat(d->sphere_mat, nS) || bad_mat(d->quad_mat, nQ) || bad_mat(d->tri_mat, nT))
        return fail(ctx, PT_EINVAL, "material index out of range");
    for (int64_t i = 0; i < nQ; ++i)
        if (d->quad_axis[i] < 0 || d->quad_axis[i] > 2) return fail(ctx, PT_EINVAL, "quad axis out of range");
    for (int64_t i = 0; i < 3 * nT; ++i)
        if (d->tris[i] < 0 || d->tris[i] >= d->n_verts) return fail(ctx, PT_EINVAL, "triangle vertex index out of range");
    for (int64_t i = 0; i < nS; ++i)
        if (!(d->spheres[4 * i + 3] > 0.f)) return fail(ctx, PT_EINVAL, "sphere radius must be > 0");

    // primitive bounds, centroids, device records
    BuildInput bin;
    bin.n_prims = nP;
    bin.lo.resize(3 * nP);
    bin.hi.resize(3 * nP);
    std::vector<float4> sph(nS), quad(2 * nQ), tri(3 * nT);
    std::vector<int32_t> pmat(nP);
    for (int64_t i = 0; i < nS; ++i) {
        const float* s = d->spheres + 4 * i;
        sph[i] = make_float4(s[0], s[1], s[2], s[3]);
        for (int a = 0; a < 3; ++a) {
            // float bounds that contain the exact sphere
            bin.lo[3 * i + a] = std::nextafter(s[a] - s[3], -INFINITY);
            bin.hi[3 * i + a] = std::nextafter(s[a] + s[3], INFINITY);
        }
        pmat[i] = d->sphere_mat[i];
    }
    for (int64_t i = 0; i < nQ; ++i) {
        const float* q = d->quads + 5 * i;
        const int a = d->quad_axis[i], u = (a + 1) % 3, v = (a + 2) % 3;
        int32_t ab = a;
        float abf;
        std::memcpy(&abf, &ab, 4);
        quad[2 * i] = make_float4(q[0], q[1], q[2], q[3]);
        quad[2 * i + 1] = make_float4(q[4], abf, 0.f, 0.f);
        const int64_t g = nS + i;
        bin.lo[3 * g + a] = bin.hi[3 * g + a] = q[0];
        bin.lo[3 * g + u] = q[1]; bin.hi[3 * g + u] = q[2];
        bin.lo[3 * g + v] = q[3]; bin.hi[3 * g + v] = q[4];
        pmat[g] = d->quad_mat[i];
    }
    for_chunks(0, nT, host_pass_threads(nT), [&](int, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            const int64_t g = nS + nQ + i;
            for (int k = 0; k < 3; ++k) {
                const float* p = d->verts + 3 * (int64_t)d->tris[3 * i + k];
                tri[3 * i + k] = make_float4(p[0], p[1], p[2], 0.f);
                for (int a = 0; a < 3; ++a) {
                    if (k == 0) { bin.lo[3 * g + a] = p[a]; bin.hi[3 * g + a] = p[a]; }
                    bin.lo[3 * g + a] = std::min(bin.lo[3 * g + a], p[a]);
                    bin.hi[3 * g + a] = std::max(bin.hi[3 * g + a], p[a]);
                }
            }
            pmat[g] = d->tri_mat[i];
        }
    });
    BuildOutput bo;
    if (!build_bvh(bin, bo)) return fail(ctx, PT_EINVAL, bo.error);
    if (bo.depth > kStackSize) return fail(ctx, PT_EUNSUPPORTED, "BVH deeper than the traversal stack");

    std::vector<float4> mat(2 * d->n_mats);
    int has_em = 0;
    for (int64_t i = 0; i < d->n_mats; ++i) {
        const float* m = d->mats + 8 * i;
        mat[2 * i] = make_float4(m[0], m[1], m[2], m[3]);
        mat[2 * i + 1] = make_float4(m[4], m[5], m[6], m[7]);
        if (m[5] != 0.f || m[6] != 0.f || m[7] != 0.f) has_em = 1;
    }

    // The node form the traversal reads: automatic = the decoded 64-byte form for BVHs that fit
    // comfortably in L2, else the packed 48-byte form; or the form the descriptor asks for.
    constexpr size_t kWideLimit = 48u << 20;
    const int32_t form_req = d->node_format;
    if (form_req < PT_NODES_AUTO || form_req > PT_NODES_QUANT8) return fail(ctx, PT_EINVAL, "unknown node_format");
    const bool want_wide = form_req == PT_NODES_DECODED ||
                           (form_req == PT_NODES_AUTO && bo.nodes.size() * 64 <= kWideLimit);
    QuantVec qn;
    if (form_req == PT_NODES_QUANT8 && !bo.nodes.empty()) {
        std::string qerr;
        if (!quantize_bvh(bo.nodes.data(), bo.nodes.size(), qn, &qerr)) return fail(ctx, PT_EUNSUPPORTED, qerr);
    }
    std::vector<float> wide;
    if (!bo.nodes.empty() && want_wide) {
        wide.assign(bo.nodes.size() * 16, 0.f);
        const int64_t n_nodes = (int64_t)bo.nodes.size();
        for_chunks(0, n_nodes, host_pass_threads(n_nodes), [&](int, int64_t i0, int64_t i1) {
            for (int64_t i = i0; i < i1; ++i) {
                const uint32_t* w = bo.nodes[(size_t)i].w;
                float lo[6], hi[6];
                for (int a = 0; a < 6; ++a) std::memcpy(&lo[a], &w[a], 4);
                const uint16_t ext[6] = {(uint16_t)(w[6] & 0xFFFFu), (uint16_t)(w[6] >> 16),
                                         (uint16_t)(w[7] & 0xFFFFu), (uint16_t)(w[7] >> 16),
                                         (uint16_t)(w[8] & 0xFFFFu), (uint16_t)(w[8] >> 16)};
                for (int a = 0; a < 6; ++a) hi[a] = lo[a] + half_bits_to_float(ext[a]);   // FP32 add, as the device does
                float* o = &wide[16 * (size_t)i];
                o[0] = lo[0]; o[1] = lo[1]; o[2] = lo[2]; o[3] = hi[0];
                o[4] = hi[1]; o[5] = hi[2]; o[6] = lo[3]; o[7] = lo[4];
                o[8] = lo[5]; o[9] = hi[3]; o[10] = hi[4]; o[11] = hi[5];
                std::memcpy(&o[12], &w[9], 4);
                std::memcpy(&o[13], &w[10], 4);
            }
        });
    }

    // one device arena per scene (one allocation; small scenes also one copy)
    struct Segment { const void* src; size_t bytes; size_t off; };
    Segment seg[9] = {{bo.nodes.data(), bo.nodes.size() * sizeof(PackedNode), 0},
                      {sph.data(), sph.size() * sizeof(float4), 0},
                      {quad.data(), quad.size() * sizeof(float4), 0},
                      {tri.data(), tri.size() * sizeof(float4), 0},
                      {pmat.data(), pmat.size() * sizeof(int32_t), 0},
                      {mat.data(), mat.size() * sizeof(float4), 0},
                      {d->mat_type, (size_t)d->n_mats * sizeof(int32_t), 0},
                      {wide.data(), wide.size() * sizeof(float), 0},
                      {qn.data(), qn.size() * sizeof(QuantNode), 0}};
    size_t total = 0;
    for (Segment& g : seg) {
        g.off = total;
        total += (g.bytes + 255) & ~(size_t)255;
    }
    pt_scene* sc = new pt_scene();
    sc->ctx = ctx;
    unsigned char* arena = nullptr;
    if (cudaMalloc((void**)&arena, std::max<size_t>(total, 256)) != cudaSuccess) {
        cudaGetLastError();
        pt_destroy_scene(sc);
        return fail(ctx, PT_ENOMEM, "scene upload failed");
    }
    sc->allocs.push_back(arena);
    bool ok = true;
    constexpr size_t kStageLimit = 4u << 20;   // small scenes: one copy; large: no extra host copy
    if (total <= kStageLimit) {
        std::vector<unsigned char> stage(total);
        for (const Segment& g : seg)
            if (g.bytes) std::memcpy(stage.data() + g.off, g.src, g.bytes);
        ok = upload_host(ctx, arena, stage.data(), total) == cudaSuccess;
    } else {
        for (const Segment& g : seg)
            if (ok && g.bytes) ok = upload_host(ctx, arena + g.off, g.src, g.bytes) == cudaSuccess;
    }
    if (!ok) {
        pt_destroy_scene(sc);
        return fail(ctx, PT_ECUDA, "scene upload failed");
    }
    void* dn = arena + seg[0].off;
    void* ds = arena + seg[1].off;
    void* dq = arena + seg[2].off;
    void* dt = arena + seg[3].off;
    void* dpm = arena + seg[4].off;
    void* dm = arena + seg[5].off;
    void* dmt = arena + seg[6].off;
    if (!wide.empty()) sc->dev.wnodes = (const uint4*)(arena + seg[7].off);
    if (!qn.empty()) sc->dev.qnodes = (const uint4*)(arena + seg[8].off);
    DevScene& v = sc->dev;
    v.nodes = (const uint4*)dn;
    v.root = bo.root;
    v.n_nodes = (uint32_t)bo.nodes.size();
    v.nS = (uint32_t)nS; v.nQ = (uint32_t)nQ; v.nT = (uint32_t)nT;
    v.sph = (const float4*)ds; v.quad = (const float4*)dq; v.tri = (const float4*)dt;
    v.prim_mat = (const int32_t*)dpm; v.mat = (const float4*)dm; v.mat_type = (const int32_t*)dmt;
    camera_basis(d->camera, v);
    v.env_is_nif = d->env_is_nif ? 1 : 0;
    for (int a = 0; a < 3; ++a) v.env[a] = d->env_rgb[a];
    v.has_emission = has_em;
    sc->info.n_prims = nP;
    sc->info.n_nodes = (int64_t)bo.nodes.size();
    sc->info.node_bytes = (int64_t)(bo.nodes.size() * sizeof(PackedNode));
    sc->info.node_format = !qn.empty() ? PT_NODES_QUANT8 : (!wide.empty() ? PT_NODES_DECODED : PT_NODES_PACKED);
    sc->info.traversed_node_bytes = (int64_t)bo.nodes.size() * (!qn.empty() ? 32 : (!wide.empty() ? 64 : 48));
    sc->info.prim_bytes = (int64_t)((sph.size() + quad.size() + tri.size()) * sizeof(float4) + pmat.size() * 4);
    sc->info.bvh_depth = bo.depth;
    sc->info.has_emission = has_em;
    *out = sc;
    return PT_OK;
}

PT_API pt_status pt_create_scene(pt_ctx* ctx, const pt_scene_desc* d, pt_scene** out)
{
    return no_throw(ctx, [&] { return create_scene(ctx, d, out); });
}

PT_API void pt_destroy_scene(pt_scene* sc)
{
    if (!sc) return;
    for (void* p : sc->allocs) cudaFree(p);
    delete sc;
}

PT_API pt_status pt_scene_get_info(const pt_scene* sc, pt_scene_info* info)
{
    if (!sc || !info) return PT_EINVAL;
    *info = sc->info;
    return PT_OK;
}

static pt_status build_bvh_host(int64_t n, const float* lo, const float* hi, uint32_t* nodes, int64_t cap,
                                   int64_t* n_nodes, uint32_t* root, int32_t* depth)
{
    if (n < 0 || !n_nodes || !root || !depth || (n > 0 && (!lo || !hi))) return PT_EINVAL;
    if (n >= (int64_t)kLeafBit - 1) return PT_EINVAL;
    if (!finite3(lo, 3 * n) || !finite3(hi, 3 * n)) return PT_EINVAL;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (lo[i] > hi[i]) return PT_EINVAL;   // an inverted box would give negative extents
    if (n > 1 && (!nodes || cap < n - 1)) return PT_EINVAL;
    BuildInput bin;
    bin.n_prims = n;
    bin.lo.assign(lo, lo + 3 * n);
    bin.hi.assign(hi, hi + 3 * n);
    BuildOutput bo;
    if (!build_bvh(bin, bo)) return PT_EUNSUPPORTED;
    if ((int64_t)bo.nodes.size() > cap && !bo.nodes.empty()) return PT_EINVAL;
    if (!bo.nodes.empty()) std::memcpy(nodes, bo.nodes.data(), bo.nodes.size() * sizeof(PackedNode));
    *n_nodes = (int64_t)bo.nodes.size();
    *root = bo.root;
    *depth = bo.depth;
    return PT_OK;
}

PT_API pt_status pt_build_bvh_host(int64_t n, const float* lo, const float* hi, uint32_t* nodes, int64_t cap,
                                   int64_t* n_nodes, uint32_t* root, int32_t* depth)
{
    return no_throw(nullptr, [&] { return build_bvh_host(n, lo, hi, nodes, cap, n_nodes, root, depth); });
}

static pt_status quantize_bvh_host(int64_t n_nodes, const uint32_t* nodes, uint32_t* out)
{
    if (n_nodes < 0 || (n_nodes > 0 && (!nodes || !out))) return PT_EINVAL;
    NodeVec in((size_t)n_nodes);
    if (n_nodes) std::memcpy(in.data(), nodes, (size_t)n_nodes * sizeof(PackedNode));
    QuantVec q;
    std::string err;
    if (!quantize_bvh(in.data(), in.size(), q, &err)) return PT_EUNSUPPORTED;
    if (n_nodes) std::memcpy(out, q.data(), (size_t)n_nodes * sizeof(QuantNode));
    return PT_OK;
}

PT_API pt_status pt_quantize_bvh_host(int64_t n_nodes, const uint32_t* nodes, uint32_t* out)
{
    return no_throw(nullptr, [&] { return quantize_bvh_host(n_nodes, nodes, out); });
}

PT_API pt_status pt_scene_download_bvh(pt_ctx* ctx, const pt_scene* sc, uint32_t* nodes, uint32_t* root)
{
    if (!ctx || !sc) return fail(ctx, PT_EINVAL, "null argument");
    if (root) *root = sc->dev.root;
    if (nodes && sc->info.n_nodes)
        PT_CUDA(cudaMemcpy(nodes, sc->dev.nodes, sc->info.node_bytes, cudaMemcpyDeviceToHost));
    return PT_OK;
}

// ---------------------------------------------------------------------------
static pt_status load_nif(pt_ctx* ctx, const pt_nif_desc* d, pt_nif** out)
{
    if (!ctx || !d || !out || !d->params) return fail(ctx, PT_EINVAL, "null argument");
    *out = nullptr;
    const int F = d->n_freq, H = d->hidden, L = d->n_hidden_layers, S = d->skip_after;
    if (F < 1 || 2 * F > 128 || H < 1 || H > 256 || L < 1 || L > 8)
        return fail(ctx, PT_EUNSUPPORTED, "NIF shape outside 2F <= 128, H <= 256, 1 <= L <= 8");
    if (S < 0 || S >= L || (S > 0 && H <= 2 * F))
        return fail(ctx, PT_EINVAL, "skip_after must be 0 or in [1, L - 1] with H > 2F");
    int64_t n = 2 * F;
    for (int l = 0; l <= L; ++l) {
        int in, o;
        nif_layer_dims(F, H, L, S, l, &in, &o);
        n += (int64_t)in * o + o;
    }
    n += 9;
    if (!finite3(d->params, n)) return fail(ctx, PT_EINVAL, "non-finite NIF parameters");
    // FP32 packed layout, each layer padded to D x D
    const int D = nif_fp32_width(H);
    const size_t fp32_floats = (size_t)L * D * D + (size_t)L * D + 3 * (size_t)D + 3 + 2 * F;
    std::vector<float> pk(fp32_floats, 0.f);
    float* Wt = pk.data();
    float* bias = Wt + (size_t)L * D * D;
    float* Wout = bias + (size_t)L * D;
    float* bout = Wout + 3 * D;
    float* Bc = bout + 3;
    const float* p = d->params;
    for (int i = 0; i < 2 * F; ++i) Bc[i] = *p++;
    for (int l = 0; l <= L; ++l) {
        int in, o;
        nif_layer_dims(F, H, L, S, l, &in, &o);
        if (l < L) {
            for (int j = 0; j < o; ++j)
                for (int k = 0; k < in; ++k) Wt[(size_t)l * D * D + (size_t)k * D + j] = p[(size_t)j * in + k];
            p += (size_t)in * o;
            for (int j = 0; j < o; ++j) bias[l * D + j] = p[j];
            p += o;
        } else {
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < in; ++k) Wout[j * D + k] = p[(size_t)j * in + k];
            p += (size_t)in * 3;
            for (int j = 0; j < 3; ++j) bout[j] = p[j];
            p += 3;
        }
    }
    pt_nif* nf = new pt_nif();
    nf->ctx = ctx;
    nf->F = F; nf->H = H; nf->L = L; nf->skip = S; nf->n_params = n;
    std::vector<unsigned char> img;
    const bool tc = pack_nif_tc_image(d->params, F, H, L, S, img);
    // one allocation and one copy: master weights | FP32 layout | tensor-core image
    const size_t b_params = ((size_t)n * sizeof(float) + 255) & ~(size_t)255;
    const size_t b_fp32 = (fp32_floats * sizeof(float) + 255) & ~(size_t)255;
    const size_t total = b_params + b_fp32 + (tc ? img.size() : 0);
    if (cudaMalloc((void**)&nf->d_arena, total) != cudaSuccess) {
        cudaGetLastError();
        pt_destroy_nif(nf);
        return fail(ctx, PT_ENOMEM, "NIF allocation failed");
    }
    nf->d_params = reinterpret_cast<float*>(nf->d_arena);
    nf->d_fp32 = reinterpret_cast<float*>(nf->d_arena + b_params);
    if (tc) nf->d_tc = nf->d_arena + b_params + b_fp32;
    {
        std::vector<unsigned char> stage(total, 0);
        std::memcpy(stage.data(), d->params, (size_t)n * sizeof(float));
        std::memcpy(stage.data() + b_params, pk.data(), fp32_floats * sizeof(float));
        if (tc) std::memcpy(stage.data() + b_params + b_fp32, img.data(), img.size());
        if (upload_host(ctx, nf->d_arena, stage.data(), total) != cudaSuccess) {
            pt_destroy_nif(nf);
            return fail(ctx, PT_ECUDA, "NIF upload failed");
        }
    }
    DevNif& v = nf->dev;
    v.F = F; v.H = H; v.L = L; v.skip = S; v.D = D;
    v.Wt = nf->d_fp32;
    v.bias = nf->d_fp32 + (size_t)L * D * D;
    v.Wout = v.bias + (size_t)L * D;
    v.bout = v.Wout + 3 * D;
    v.B = v.bout + 3;
    for (int i = 0; i < 9; ++i) v.M[i] = d->params[n - 9 + i];
    nf->fp8_ok = F == 64 && H == 128 && L == 3 && S == 0;
    *out = nf;
    return PT_OK;
}

PT_API pt_status pt_load_nif(pt_ctx* ctx, const pt_nif_desc* d, pt_nif** out)
{
    return no_throw(ctx, [&] { return load_nif(ctx, d, out); });
}

PT_API void pt_destroy_nif(pt_nif* nf)
{
    if (!nf) return;
    cudaFree(nf->d_arena);   // d_params, d_fp32 and d_tc live in it
    cudaFree(nf->d_fp8);
    cudaFree(nf->d_grad);
    cudaFree(nf->d_m);
    cudaFree(nf->d_v);
    cudaFree(nf->d_work);
    cudaFree(nf->d_batch);
    cudaFree(nf->d_loss);
    delete nf;
}

PT_API int64_t pt_nif_param_count(const pt_nif* nf) { return nf ? nf->n_params : 0; }

PT_API pt_status pt_nif_get_params(pt_ctx* ctx, const pt_nif* nf, float* params)
{
    if (!ctx || !nf || !params) return fail(ctx, PT_EINVAL, "null argument");
    PT_CUDA(cudaDeviceSynchronize());
    PT_CUDA(cudaMemcpy(params, nf->d_params, nf->n_params * sizeof(float), cudaMemcpyDeviceToHost));
    return PT_OK;
}

PT_API pt_status pt_nif_eval(pt_ctx* ctx, const pt_nif* nf, int32_t precision, int64_t n, const float* d_uv,
                             float* d_rgb, void* stream)
{
    if (!ctx || !nf || n < 0 || (n > 0 && (!d_uv || !d_rgb))) return fail(ctx, PT_EINVAL, "bad argument");
    if (n == 0) return PT_OK;
    NifEvalParams p = {};
    p.nif = nf->dev;
    p.uv = d_uv;
    p.rgb = d_rgb;
    p.n = n;
    p.err = ctx->d_err;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == PT_FP32) {
        PT_CUDA(timed(ctx, PT_KIND_NIF, s, [&] { return launch_nif_fp32(p, 0, ctx->sm_count, s); }));
        return PT_OK;
    }
    if (precision == PT_BF16 && nf->d_tc) {
        PT_CUDA(timed(ctx, PT_KIND_NIF, s, [&] { return launch_nif_tc(nf->d_tc, nf->F, nf->H, nf->L, nf->skip, p, 0, ctx->sm_count, s); }));
        return PT_OK;
    }
    if (precision == PT_FP8E4M3 && nf->fp8_ok) {
        const pt_status st = ensure_fp8(ctx, nf, s);
        if (st != PT_OK) return st;
        PT_CUDA(timed(ctx, PT_KIND_NIF, s, [&] { return launch_nif_fp8(nf->d_fp8, p, 0, ctx->sm_count, s); }));
        return PT_OK;
    }
    if (precision == PT_BF16 || precision == PT_FP8E4M3)
        return fail(ctx, PT_EUNSUPPORTED, "no BF16 kernel for this NIF shape (F = 64 with H = 128 and L <= 5, H = 64 or 32 and L <= 8, H = 256 and L = 1; the paper's F = 20 skip network); FP8: F = 64, H = 128, L = 3");
    return fail(ctx, PT_EINVAL, "unknown precision");
}

// ---------------------------------------------------------------------------
// NIF training (Section 3.2.1)
namespace {

// training GEMM precision: PT_FP32, or PT_BF16 where the tensor-core kernels take the shape
pt_status check_train_precision(pt_ctx* ctx, int L, int H, int in0, int32_t precision, int skip = 0)
{
    if (H > 128) return fail(ctx, PT_EUNSUPPORTED, "training takes hidden widths up to 128");
    if (precision == PT_FP32) return PT_OK;
    if (precision != PT_BF16) return fail(ctx, PT_EINVAL, "training precision is PT_FP32 or PT_BF16");
    if (skip > 0) return fail(ctx, PT_EUNSUPPORTED, "the skip-concatenated NIF trains with FP32 GEMMs");
    TrainNet t = {};
    t.L = L;
    t.H = H;
    t.in0 = in0;
    if (!train_tc_supported(t))
        return fail(ctx, PT_EUNSUPPORTED,
                    "BF16 training needs inputs and width <= 128 and every hidden layer's weights resident in shared "
                    "memory (width 128: at most 5 layers)");
    return PT_OK;
}

TrainNet make_train_net(pt_nif* nf)
{
    TrainNet t = {};
    t.F = nf->F; t.H = nf->H; t.L = nf->L;
    t.in0 = 2 * nf->F;
    t.skip = nf->skip;
    const float* p = nf->d_params;
    float* g = nf->d_grad;
    t.B = p;
    p += 2 * nf->F;
    for (int l = 0; l <= nf->L; ++l) {
        int in, o;
        nif_layer_dims(nf->F, nf->H, nf->L, nf->skip, l, &in, &o);
        t.in[l] = in;
        t.out[l] = o;
        t.W[l] = p; t.gW[l] = g;
        p += (size_t)in * o; g += (size_t)in * o;
        t.b[l] = p; t.gb[l] = g;
        p += o; g += o;
    }
    t.M = p;
    return t;
}

pt_status ensure_train(pt_ctx* ctx, pt_nif* nf, int64_t B)
{
    if (!nf->d_grad) {
        nf->n_trainable = nf->n_params - 2 * nf->F - 9;
        if (cudaMalloc((void**)&nf->d_grad, nf->n_trainable * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&nf->d_m, nf->n_trainable * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&nf->d_v, nf->n_trainable * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&nf->d_loss, sizeof(double)) != cudaSuccess)
            return fail(ctx, PT_ENOMEM, "training state allocation failed");
        if (cudaMemset(nf->d_m, 0, nf->n_trainable * sizeof(float)) != cudaSuccess ||
            cudaMemset(nf->d_v, 0, nf->n_trainable * sizeof(float)) != cudaSuccess)
            return fail(ctx, PT_ECUDA, "training state initialisation failed");
    }
    if (nf->work_cap >= B) return PT_OK;
    cudaFree(nf->d_work);
    cudaFree(nf->d_batch);
    nf->d_work = nullptr;
    nf->d_batch = nullptr;
    const int G = 4 * ctx->sm_count;   // partial slots: up to four GEMM CTAs per SM
    const size_t rows = (size_t)((B + 127) / 128) * 128 * 128;   // whole 128-row tiles (tiled layouts)
    // X[0 .. L], dX[2], BF16 operand tiles Xb[0 .. L-1] and Gb[0 .. L-1], partials, loss partials
    const size_t tiles = (size_t)((B + 127) / 128) * 128 * 128 * 2;
    const size_t bytes = (size_t)(nf->L + 3) * rows * sizeof(float) + 2 * (size_t)nf->L * tiles +
                         (size_t)G * (128 * 128 + 128) * sizeof(float) +
                         (size_t)G * sizeof(double) + 4096;
    if (cudaMalloc(&nf->d_work, bytes) != cudaSuccess || cudaMalloc((void**)&nf->d_batch, (size_t)B * 5 * sizeof(float)) != cudaSuccess) {
        nf->work_cap = 0;
        return fail(ctx, PT_ENOMEM, "training work buffers allocation failed");
    }
    char* w = static_cast<char*>(nf->d_work);
    nf->work = TrainWork{};
    nf->work.n_blocks = G;
    nf->work.sm_count = ctx->sm_count;
    for (int l = 0; l <= nf->L; ++l) { nf->work.X[l] = reinterpret_cast<float*>(w); w += rows * sizeof(float); }
    for (int i = 0; i < 2; ++i) { nf->work.dX[i] = reinterpret_cast<float*>(w); w += rows * sizeof(float); }
    for (int l = 0; l < nf->L; ++l) {
        nf->work.Xb[l] = reinterpret_cast<unsigned char*>(w);
        w += tiles;
        nf->work.Gb[l] = reinterpret_cast<unsigned char*>(w);
        w += tiles;
    }
    nf->work.err = ctx->d_err;
    nf->work.partial = reinterpret_cast<float*>(w);
    w += (size_t)G * (128 * 128 + 128) * sizeof(float);
    nf->work.loss_partial = reinterpret_cast<double*>(w);
    nf->work_cap = B;
    return PT_OK;
}

// FP32 packed layout and tensor-core image follow the master weights
pt_status refresh_layouts(pt_ctx* ctx, pt_nif* nf, cudaStream_t s)
{
    PT_CUDA(repack_nif_fp32(nf->d_params, nf->F, nf->H, nf->L, nf->skip, nf->d_fp32, s));
    if (nf->d_tc) PT_CUDA(repack_nif_tc_image(nf->d_params, nf->F, nf->H, nf->L, nf->skip, nf->d_tc, s));
    nf->fp8_stale = true;   // rebuilt on its next use
    return PT_OK;
}

}  // namespace

PT_API pt_status pt_nif_loss_grad(pt_ctx* ctx, pt_nif* nf, int64_t n, const float* d_uv, const float* d_target,
                                  float delta, int32_t precision, float* d_grad, double* d_loss, void* stream)
{
    if (!ctx || !nf || n < 1 || !d_uv || !d_target || !(delta > 0.f)) return fail(ctx, PT_EINVAL, "bad argument");
    pt_status st = check_train_precision(ctx, nf->L, nf->H, 2 * nf->F, precision, nf->skip);
    if (st != PT_OK) return st;
    st = ensure_train(ctx, nf, n);
    if (st != PT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    TrainNet net = make_train_net(nf);
    PT_CUDA(timed(ctx, PT_KIND_OTHER, s, [&] {
        return nif_loss_grad(net, n, d_uv, d_target, delta, precision, nf->work, d_loss ? d_loss : nf->d_loss, nullptr,
                             s);
    }));
    if (d_grad)
        PT_CUDA(cudaMemcpyAsync(d_grad, nf->d_grad, nf->n_trainable * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return PT_OK;
}

PT_API pt_status pt_train_nif(pt_ctx* ctx, pt_nif* nf, const float* d_sky, int32_t w, int32_t h, const pt_train_cfg* cfg,
                              float* d_losses, void* stream)
{
    if (!ctx || !nf || !d_sky || !cfg || w < 1 || h < 1) return fail(ctx, PT_EINVAL, "bad argument");
    if (cfg->steps < 0 || cfg->batch < 1 || !(cfg->lr > 0.f) || !(cfg->huber_delta > 0.f) || !(cfg->beta1 >= 0.f) ||
        !(cfg->beta1 < 1.f) || !(cfg->beta2 >= 0.f) || !(cfg->beta2 < 1.f) || !(cfg->eps > 0.f))
        return fail(ctx, PT_EINVAL, "bad training configuration");
    pt_status st = check_train_precision(ctx, nf->L, nf->H, 2 * nf->F, cfg->precision, nf->skip);
    if (st != PT_OK) return st;
    st = ensure_train(ctx, nf, cfg->batch);
    if (st != PT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    TrainNet net = make_train_net(nf);
    float* uv = nf->d_batch;
    float* target = uv + 2 * cfg->batch;
    for (int64_t i = 0; i < cfg->steps; ++i) {
        const int64_t t = nf->adam_t;  // global step index: Philox counter word 1 and Adam's t - 1
        PT_CUDA(timed(ctx, PT_KIND_OTHER, s, [&] {
            return train_inputs(cfg->seed, (uint32_t)t, cfg->batch, d_sky, w, h, uv, target, s);
        }));
        PT_CUDA(timed(ctx, PT_KIND_OTHER, s, [&] {
            return nif_loss_grad(net, cfg->batch, uv, target, cfg->huber_delta, cfg->precision, nf->work, nullptr,
                                 d_losses ? d_losses + i : nullptr, s);
        }));
        const double c1 = 1.0 - std::pow((double)cfg->beta1, (double)(t + 1));
        const double c2 = 1.0 - std::pow((double)cfg->beta2, (double)(t + 1));
        float* wts = nf->d_params + 2 * nf->F;
        PT_CUDA(timed(ctx, PT_KIND_OTHER, s, [&] {
            return adam_step(nf->n_trainable, wts, nf->d_grad, nf->d_m, nf->d_v, cfg->lr, cfg->beta1, cfg->beta2, cfg->eps,
                             (float)c1, (float)c2, s);
        }));
        nf->adam_t = t + 1;
    }
    return refresh_layouts(ctx, nf, s);
}

PT_API pt_status pt_nif_fp8_scales(const pt_nif* nf, float* scales)
{
    if (!nf || !scales) return PT_EINVAL;
    if (!nf->fp8_ok) return PT_EUNSUPPORTED;
    const pt_status st = ensure_fp8(nf->ctx, nf, 0);
    if (st != PT_OK) return st;
    for (int i = 0; i < 4; ++i) scales[i] = nf->fp8_scales[i];
    return PT_OK;
}

PT_API pt_status pt_nif_set_params(pt_ctx* ctx, pt_nif* nf, const float* params, void* stream)
{
    if (nf) ++nf->version;   // host-side copies (the colour matrix) may change
    if (!ctx || !nf || !params) return fail(ctx, PT_EINVAL, "bad argument");
    if (!finite3(params, nf->n_params)) return fail(ctx, PT_EINVAL, "non-finite NIF parameters");
    cudaStream_t s = (cudaStream_t)stream;
    PT_CUDA(cudaMemcpyAsync(nf->d_params, params, nf->n_params * sizeof(float), cudaMemcpyHostToDevice, s));
    PT_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < 9; ++i) nf->dev.M[i] = params[nf->n_params - 9 + i];
    return refresh_layouts(ctx, nf, s);
}

// ---------------------------------------------------------------------------
// Neural radiance cache (Mueller et al. 2021, cited in Section 2.1)
static pt_status render_impl(pt_ctx* ctx, const pt_scene* sc, const pt_nif* nf, const pt_render_cfg* cfg,
                             uint32_t first_sample, const pt_cache* cache, int cache_vertex, int rec_vertex, float* d_rec,
                             int64_t n_pix, const int64_t* d_pixels, float* d_pixel_rgb, float* d_slot_rgb,
                             int32_t* d_hit_ids, cudaStream_t s);
namespace {

TrainNet make_cache_net(pt_cache* c)
{
    TrainNet t = {};
    t.F = 0; t.H = c->H; t.L = c->L;
    t.in0 = c->in0;
    const float* p = c->d_params;
    float* g = c->d_grad;
    for (int l = 0; l <= c->L; ++l) {
        const int in = l == 0 ? c->in0 : c->H, o = l == c->L ? 3 : c->H;
        t.in[l] = in;
        t.out[l] = o;
        t.W[l] = p; t.gW[l] = g;
        p += (size_t)in * o; g += (size_t)in * o;
        t.b[l] = p; t.gb[l] = g;
        p += o; g += o;
    }
    return t;
}

pt_status ensure_cache_train(pt_ctx* ctx, pt_cache* c, int64_t B)
{
    if (!c->d_grad) {
        if (cudaMalloc((void**)&c->d_grad, c->n_params * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&c->d_m, c->n_params * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&c->d_v, c->n_params * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&c->d_loss, sizeof(double)) != cudaSuccess)
            return fail(ctx, PT_ENOMEM, "cache training state allocation failed");
        if (cudaMemset(c->d_m, 0, c->n_params * sizeof(float)) != cudaSuccess ||
            cudaMemset(c->d_v, 0, c->n_params * sizeof(float)) != cudaSuccess)
            return fail(ctx, PT_ECUDA, "cache training state initialisation failed");
    }
    if (c->work_cap >= B) return PT_OK;
    cudaFree(c->d_work);
    c->d_work = nullptr;
    c->work_cap = 0;
    const int G = 4 * ctx->sm_count;   // partial slots: up to four GEMM CTAs per SM
    const size_t rows = (size_t)((B + 127) / 128) * 128 * 128;   // whole 128-row tiles (tiled layouts)
    // X[0 .. L], dX[2], BF16 operand tiles Xb[0 .. L-1] and Gb[0 .. L-1], partials, loss partials
    const size_t tiles = (size_t)((B + 127) / 128) * 128 * 128 * 2;
    const size_t bytes = (size_t)(c->L + 3) * rows * sizeof(float) + 2 * (size_t)c->L * tiles +
                         (size_t)G * (128 * 128 + 128) * sizeof(float) +
                         (size_t)G * sizeof(double) + 4096;
    if (cudaMalloc(&c->d_work, bytes) != cudaSuccess) return fail(ctx, PT_ENOMEM, "cache work buffers allocation failed");
    char* w = static_cast<char*>(c->d_work);
    c->work = TrainWork{};
    c->work.n_blocks = G;
    c->work.sm_count = ctx->sm_count;
    for (int l = 0; l <= c->L; ++l) { c->work.X[l] = reinterpret_cast<float*>(w); w += rows * sizeof(float); }
    for (int i = 0; i < 2; ++i) { c->work.dX[i] = reinterpret_cast<float*>(w); w += rows * sizeof(float); }
    for (int l = 0; l < c->L; ++l) {
        c->work.Xb[l] = reinterpret_cast<unsigned char*>(w);
        w += tiles;
        c->work.Gb[l] = reinterpret_cast<unsigned char*>(w);
        w += tiles;
    }
    c->work.err = ctx->d_err;
    c->work.partial = reinterpret_cast<float*>(w);
    w += (size_t)G * (128 * 128 + 128) * sizeof(float);
    c->work.loss_partial = reinterpret_cast<double*>(w);
    c->work_cap = B;
    return PT_OK;
}

pt_status ensure_cache_paths(pt_ctx* ctx, pt_cache* c, int64_t n)
{
    if (c->train_cap >= n) return PT_OK;
    cudaFree(c->d_train);
    c->d_train = nullptr;
    c->train_cap = 0;
    const size_t bytes = (size_t)n * (8 + 16 * 4 + 3 * 4 + 3 * 4 + 4) + 1024;
    if (cudaMalloc(&c->d_train, bytes) != cudaSuccess) return fail(ctx, PT_ENOMEM, "cache training paths allocation failed");
    char* w = static_cast<char*>(c->d_train);
    c->d_pixels = reinterpret_cast<int64_t*>(w); w += (size_t)n * 8;
    c->d_rec = reinterpret_cast<float*>(w); w += (size_t)n * 64;
    c->d_Lpath = reinterpret_cast<float*>(w); w += (size_t)n * 12;
    c->d_target = reinterpret_cast<float*>(w); w += (size_t)n * 12;
    c->d_mask = reinterpret_cast<int32_t*>(w);
    c->train_cap = n;
    return PT_OK;
}

bool adam_cfg_ok(float lr, float b1, float b2, float eps)
{
    return lr > 0.f && b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps > 0.f;
}

}  // namespace

static pt_status create_cache(pt_ctx* ctx, const pt_cache_desc* d, pt_cache** out)
{
    if (!ctx || !d || !out || !d->params) return fail(ctx, PT_EINVAL, "null argument");
    *out = nullptr;
    if (d->hidden != 64) return fail(ctx, PT_EUNSUPPORTED, "the cache kernels need hidden = 64");
    if (d->n_freq < 1 || d->n_freq > 15 || d->n_hidden_layers < 1 || d->n_hidden_layers > 7)
        return fail(ctx, PT_EINVAL, "n_freq must be in [1, 15] and n_hidden_layers in [1, 7]");
    const int J = d->n_freq, H = d->hidden, L = d->n_hidden_layers, in0 = 6 * J + 6;
    if (cache_eval_smem_bytes(in0, L) > 227 * 1024) return fail(ctx, PT_EUNSUPPORTED, "cache too large for shared memory");
    const int64_t np = (int64_t)in0 * H + H + (int64_t)(L - 1) * (H * H + H) + 3 * H + 3;
    if (!finite3(d->params, np)) return fail(ctx, PT_EINVAL, "non-finite cache parameters");
    CacheBox box = {};
    box.J = J;
    for (int a = 0; a < 3; ++a) {
        if (!(std::isfinite(d->lo[a]) && std::isfinite(d->hi[a]) && d->hi[a] > d->lo[a]))
            return fail(ctx, PT_EINVAL, "cache box needs finite hi > lo");
        const double ext = (double)d->hi[a] - (double)d->lo[a];
        box.lo[a] = d->lo[a];
        box.eh[a] = (float)ext;
        box.el[a] = (float)(ext - (double)box.eh[a]);
    }
    PT_CUDA(cudaSetDevice(ctx->device));
    pt_cache* c = new pt_cache;
    c->ctx = ctx;
    c->J = J; c->H = H; c->L = L; c->in0 = in0;
    c->n_params = np;
    c->box = box;
    for (int a = 0; a < 3; ++a) {
        c->box_lo[a] = d->lo[a];
        c->box_hi[a] = d->hi[a];
    }
    if (cudaMalloc((void**)&c->d_params, np * sizeof(float)) != cudaSuccess ||
        upload_host(ctx, c->d_params, d->params, np * sizeof(float)) != cudaSuccess) {
        pt_destroy_cache(c);
        return fail(ctx, PT_ENOMEM, "cache parameter upload failed");
    }
    if (cache_tc_supported(J, H, L)) {
        if (cudaMalloc((void**)&c->d_tc, cache_tc_image_bytes()) != cudaSuccess ||
            cudaMemset(c->d_tc, 0, cache_tc_image_bytes()) != cudaSuccess ||
            repack_cache_tc(c->d_params, c->d_tc, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            pt_destroy_cache(c);
            return fail(ctx, PT_ENOMEM, "cache tensor-core image failed");
        }
    }
    *out = c;
    return PT_OK;
}

PT_API pt_status pt_create_cache(pt_ctx* ctx, const pt_cache_desc* d, pt_cache** out)
{
    return no_throw(ctx, [&] { return create_cache(ctx, d, out); });
}

PT_API void pt_destroy_cache(pt_cache* c)
{
    if (!c) return;
    cudaSetDevice(c->ctx->device);
    cudaFree(c->d_params);
    cudaFree(c->d_tc);
    cudaFree(c->d_grad);
    cudaFree(c->d_m);
    cudaFree(c->d_v);
    cudaFree(c->d_work);
    cudaFree(c->d_train);
    cudaFree(c->d_loss);
    delete c;
}

PT_API int64_t pt_cache_param_count(const pt_cache* c) { return c ? c->n_params : 0; }

PT_API pt_status pt_cache_get_params(pt_ctx* ctx, const pt_cache* c, float* params)
{
    if (!ctx || !c || !params) return fail(ctx, PT_EINVAL, "null argument");
    PT_CUDA(cudaDeviceSynchronize());
    PT_CUDA(cudaMemcpy(params, c->d_params, c->n_params * sizeof(float), cudaMemcpyDeviceToHost));
    return PT_OK;
}

PT_API pt_status pt_cache_set_params(pt_ctx* ctx, pt_cache* c, const float* params, void* stream)
{
    if (!ctx || !c || !params) return fail(ctx, PT_EINVAL, "null argument");
    if (!finite3(params, c->n_params)) return fail(ctx, PT_EINVAL, "non-finite cache parameters");
    cudaStream_t s = (cudaStream_t)stream;
    PT_CUDA(cudaMemcpyAsync(c->d_params, params, c->n_params * sizeof(float), cudaMemcpyHostToDevice, s));
    if (c->d_m) {
        PT_CUDA(cudaMemsetAsync(c->d_m, 0, c->n_params * sizeof(float), s));
        PT_CUDA(cudaMemsetAsync(c->d_v, 0, c->n_params * sizeof(float), s));
    }
    if (c->d_tc) PT_CUDA(repack_cache_tc(c->d_params, c->d_tc, s));
    c->adam_t = 0;
    PT_CUDA(cudaStreamSynchronize(s));
    return PT_OK;
}

PT_API pt_status pt_cache_eval(pt_ctx* ctx, const pt_cache* c, int32_t precision, int64_t n, const float* d_q,
                               float* d_out, void* stream)
{
    if (!ctx || !c || n < 0 || (n > 0 && (!d_q || !d_out))) return fail(ctx, PT_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == PT_FP32) {
        PT_CUDA(timed(ctx, PT_KIND_CACHE, s, [&] {
            return cache_eval(c->d_params, c->J, c->L, c->box, n, d_q, d_out, ctx->sm_count, s);
        }));
        return PT_OK;
    }
    if (precision != PT_BF16) return fail(ctx, PT_EINVAL, "cache precision is PT_FP32 or PT_BF16");
    if (!c->d_tc) return fail(ctx, PT_EUNSUPPORTED, "the BF16 cache needs n_freq = 12, hidden = 64, 5 hidden layers");
    PT_CUDA(timed(ctx, PT_KIND_CACHE, s, [&] {
        return cache_eval_tc(c->d_tc, c->box, n, d_q, d_out, ctx->d_err, ctx->sm_count, s);
    }));
    return PT_OK;
}

PT_API pt_status pt_cache_loss_grad(pt_ctx* ctx, pt_cache* c, int64_t n, const float* d_q, const float* d_target,
                                    const int32_t* d_mask, int32_t precision, float* d_grad, double* d_loss,
                                    void* stream)
{
    if (!ctx || !c || n < 1 || !d_q || !d_target) return fail(ctx, PT_EINVAL, "bad argument");
    pt_status st = check_train_precision(ctx, c->L, c->H, c->in0, precision);
    if (st != PT_OK) return st;
    st = ensure_cache_train(ctx, c, n);
    if (st != PT_OK) return st;
    st = ensure_cache_paths(ctx, c, n);
    if (st != PT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // queries -> 16-float record rows (valid = 1) so that the training feature kernel reads them
    PT_CUDA(cudaMemsetAsync(c->d_rec, 0, (size_t)n * 64, s));
    PT_CUDA(cudaMemcpy2DAsync(c->d_rec, 64, d_q, 36, 36, (size_t)n, cudaMemcpyDeviceToDevice, s));
    TrainNet net = make_cache_net(c);
    PT_CUDA(timed(ctx, PT_KIND_OTHER, s, [&] {
        cudaError_t e = cache_train_inputs(n, c->d_rec, nullptr, c->box, c->work.X[0], nullptr, nullptr, s);
        if (e != cudaSuccess) return e;
        return mlp_loss_grad(net, n, d_target, 0.f, 1, d_mask, precision, c->work, d_loss ? d_loss : c->d_loss,
                             nullptr, s);
    }));
    if (d_grad) PT_CUDA(cudaMemcpyAsync(d_grad, c->d_grad, c->n_params * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return PT_OK;
}

PT_API pt_status pt_train_cache(pt_ctx* ctx, const pt_scene* sc, const pt_nif* nf, pt_cache* c,
                                const pt_cache_train_cfg* cfg, float* d_loss, void* stream)
{
    if (!ctx || !sc || !c || !cfg) return fail(ctx, PT_EINVAL, "null argument");
    if (cfg->n_train < 1 || cfg->max_depth < 1 || cfg->max_depth > kMaxDepth || cfg->rec_vertex < 1 ||
        cfg->rec_vertex > cfg->max_depth || !adam_cfg_ok(cfg->lr, cfg->beta1, cfg->beta2, cfg->eps))
        return fail(ctx, PT_EINVAL, "bad cache training configuration");
    pt_render_cfg rc = {};
    rc.width = cfg->width;
    rc.height = cfg->height;
    rc.spp = 1;
    rc.max_depth = cfg->max_depth;
    rc.seed = cfg->seed;
    rc.precision = cfg->precision;
    pt_status st = check_cfg(ctx, sc, nf, &rc);
    if (st != PT_OK) return st;
    st = check_train_precision(ctx, c->L, c->H, c->in0, cfg->train_precision);
    if (st != PT_OK) return st;
    const int64_t n = cfg->n_train;
    st = ensure_cache_train(ctx, c, n);
    if (st != PT_OK) return st;
    st = ensure_cache_paths(ctx, c, n);
    if (st != PT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n_pix = (uint32_t)((int64_t)cfg->width * cfg->height);
    PT_CUDA(timed(ctx, PT_KIND_OTHER, s, [&] { return cache_train_pixels(cfg->seed, cfg->frame, n, n_pix, c->d_pixels, s); }));
    // plain training paths with records at rec_vertex; spp 1, so the pixel means are the path radiances
    st = render_impl(ctx, sc, nf, &rc, 0x40000000u + cfg->frame, nullptr, 0, cfg->rec_vertex, c->d_rec, n, c->d_pixels,
                     c->d_Lpath, nullptr, nullptr, s);
    if (st != PT_OK) return st;
    TrainNet net = make_cache_net(c);
    PT_CUDA(timed(ctx, PT_KIND_OTHER, s, [&] {
        cudaError_t e = cache_train_inputs(n, c->d_rec, c->d_Lpath, c->box, c->work.X[0], c->d_target, c->d_mask, s);
        if (e != cudaSuccess) return e;
        return mlp_loss_grad(net, n, c->d_target, 0.f, 1, c->d_mask, cfg->train_precision, c->work, c->d_loss, d_loss,
                             s);
    }));
    const int64_t t = c->adam_t;
    const double c1 = 1.0 - std::pow((double)cfg->beta1, (double)(t + 1));
    const double c2 = 1.0 - std::pow((double)cfg->beta2, (double)(t + 1));
    PT_CUDA(timed(ctx, PT_KIND_OTHER, s, [&] {
        cudaError_t e = adam_step(c->n_params, c->d_params, c->d_grad, c->d_m, c->d_v, cfg->lr, cfg->beta1, cfg->beta2,
                                  cfg->eps, (float)c1, (float)c2, s);
        if (e != cudaSuccess || !c->d_tc) return e;
        return repack_cache_tc(c->d_params, c->d_tc, s);   // the BF16 image follows the master weights
    }));
    c->adam_t = t + 1;
    return PT_OK;
}

// ---------------------------------------------------------------------------
// The render loop behind pt_render / pt_render_pixels / pt_render_cached and
// the training paths of pt_train_cache.  first_sample is the Philox sample
// index of the first path per pixel; cache (nullable) ends paths at
// cache_vertex; rec_vertex > 0 writes vertex records to d_rec.
// The launch sequence of one render (no host synchronisation, no allocation):
// recorded once into a CUDA graph and replayed when the same render repeats.
// Schedule of a chunk of n paths: the path-per-thread kernel when asked for,
// or (automatic) when the chunk fits in one resident wave of it.
static bool use_paths(const pt_ctx* ctx, const pt_scene* sc, const pt_render_cfg* cfg, int64_t n)
{
    const int resident = ctx->paths_threads[sc->dev.qnodes ? 2 : (sc->dev.wnodes ? 1 : 0)];
    return cfg->schedule == PT_SCHED_PATHS || (cfg->schedule == PT_SCHED_AUTO && resident > 0 && n <= resident);
}

static pt_status render_launches(pt_ctx* ctx, const pt_scene* sc, const pt_nif* nf, const pt_render_cfg* cfg,
                                 const pt_cache* cache, int cache_vertex, int rec_vertex, float* d_rec, int64_t n_pix,
                                 const int64_t* d_pixels, float* d_pixel_rgb, float* d_slot_rgb, int32_t* d_hit_ids,
                                 int64_t n_slots, int64_t chunk, cudaStream_t s)
{
    pt_status st = PT_OK;
    if (rec_vertex > 0) PT_CUDA(cudaMemsetAsync(d_rec, 0, (size_t)n_slots * 16 * sizeof(float), s));
    PT_CUDA(cudaMemsetAsync(ctx->stats, 0, kStats * sizeof(unsigned long long), s));
    if (d_hit_ids) PT_CUDA(launch_fill_i32(d_hit_ids, n_slots * cfg->max_depth, -2, s));

    BounceParams bp = {};
    bp.sc = sc->dev;
    bp.sc.aspect = (float)((double)cfg->width / (double)cfg->height);
    bp.max_depth = cfg->max_depth;
    bp.rr = cfg->rr;
    bp.rr_start = cfg->rr_start;
    bp.seed = cfg->seed;
    bp.first_sample = 0;
    bp.first_sample_dev = ctx->d_first_sample;   // written before the sequence runs
    bp.n_pix = (uint32_t)n_pix;
    bp.pixels = d_pixels;
    bp.W = cfg->width;
    bp.H = cfg->height;
    bp.tiled = !d_pixels && cfg->width % 8 == 0 && cfg->height % 4 == 0;
    bp.esc = ctx->esc;
    bp.esc_count = ctx->counters + kEscCounter;
    bp.slot_L = ctx->slot_L;
    bp.hit_ids = d_hit_ids;
    bp.err = ctx->d_err;
    bp.stats = ctx->stats;
    bp.work = ctx->stats + kWorkBase;
    bp.cap = (uint32_t)chunk;
    bp.cache_vertex = cache ? cache_vertex : 0;
    bp.cache_rows = ctx->cache_rows;
    bp.cache_count = ctx->counters + kCacheCounter;
    bp.rec_vertex = rec_vertex;
    bp.rec = d_rec;
    bp.hits = ctx->hits;
    bp.fetch = ctx->counters + kFetchCounter;
    const int64_t n_chunks = (n_slots + chunk - 1) / chunk;
    for (int64_t c = 0; c < n_chunks; ++c) {
        const int64_t first = c * chunk;
        const int64_t n = std::min(chunk, n_slots - first);
        PT_CUDA(cudaMemsetAsync(ctx->counters, 0, kCounters * sizeof(uint32_t), s));
        bp.chunk_first = (uint64_t)first;
        bp.n_chunk = (uint32_t)n;
        // with a cache no path outlives its cache vertex
        const int k_end = cache ? std::min(cfg->max_depth, cache_vertex) : cfg->max_depth;
        const bool per_path = use_paths(ctx, sc, cfg, n);
        if (per_path) {
            bp.k = 1;
            const int resident = ctx->paths_threads[sc->dev.qnodes ? 2 : (sc->dev.wnodes ? 1 : 0)];
            PT_CUDA(timed(ctx, PT_KIND_TRACE, s, [&] { return launch_paths(bp, resident, s); }));
        }
        for (int k = 1; k <= k_end && !per_path; ++k) {
            bp.k = k;
            bp.qin = ctx->q[(k + 1) & 1];
            bp.qout = ctx->q[k & 1];
            bp.count_in = ctx->counters + (k - 1);
            bp.count_out = ctx->counters + k;
            PT_CUDA(timed(ctx, PT_KIND_TRACE, s, [&] { return launch_trace(bp, ctx->sm_count, s); }));
            PT_CUDA(timed(ctx, PT_KIND_SHADE, s, [&] { return launch_shade(bp, ctx->sm_count, s); }));
        }
        if (sc->dev.env_is_nif) {
            st = eval_nif_escapes(ctx, nf, cfg->precision, sc->dev.has_emission, s);
            if (st != PT_OK) return st;
        }
        if (cache) {
            // the cache runs in BF16 on the tensor cores whenever the NIF does (and the shape allows it)
            const bool tc = cfg->precision != PT_FP32 && cache->d_tc;
            PT_CUDA(timed(ctx, PT_KIND_CACHE, s, [&] {
                if (tc)
                    return cache_query_tc(cache->d_tc, cache->box, chunk, ctx->counters + kCacheCounter,
                                          ctx->cache_rows, ctx->slot_L, sc->dev.has_emission, ctx->d_err,
                                          ctx->stats + kCacheStat, ctx->sm_count, s);
                return cache_query(cache->d_params, cache->J, cache->L, cache->box, chunk,
                                   ctx->counters + kCacheCounter, ctx->cache_rows, ctx->slot_L, sc->dev.has_emission,
                                   ctx->d_err, ctx->stats + kCacheStat, ctx->sm_count, s);
            }));
        }
        const float scale = (c == n_chunks - 1) ? (float)(1.0 / cfg->spp) : 1.f;
        PT_CUDA(timed(ctx, PT_KIND_REDUCE, s, [&] {
            return launch_reduce(ctx->slot_L, d_pixel_rgb, (uint32_t)n_pix, (uint32_t)(n / n_pix), c == 0, scale, s);
        }));
        if (d_slot_rgb)
            PT_CUDA(cudaMemcpyAsync(d_slot_rgb + 3 * first, ctx->slot_L, (size_t)n * 3 * sizeof(float),
                                    cudaMemcpyDeviceToDevice, s));
    }
    return PT_OK;
}


// Key of a captured render: every value the launch sequence bakes into kernel
// parameters (object identities, configuration, buffers, scratch generation).
// The sample offset is not in it: it is a device word written per call.
struct GraphKey {
    uint64_t sc_uid, nf_uid, nf_version, cache_uid, scratch_gen;
    int32_t width, height, spp, max_depth, rr, rr_start, precision, cache_vertex, rec_vertex, schedule;
    uint32_t seed, cache_cap;
    int64_t chunk, n_pix;
    const void* ptrs[5];   // d_rec, d_pixels, d_pixel_rgb, d_slot_rgb, d_hit_ids
};
constexpr size_t kMaxGraphs = 8;

static pt_status render_impl(pt_ctx* ctx, const pt_scene* sc, const pt_nif* nf, const pt_render_cfg* cfg,
                             uint32_t first_sample, const pt_cache* cache, int cache_vertex, int rec_vertex, float* d_rec,
                             int64_t n_pix, const int64_t* d_pixels, float* d_pixel_rgb, float* d_slot_rgb,
                             int32_t* d_hit_ids, cudaStream_t s)
{
    pt_status st = PT_OK;
    const int64_t WH = (int64_t)cfg->width * cfg->height;
    if (!d_pixels) n_pix = WH;
    if (n_pix < 0 || (n_pix > 0 && !d_pixel_rgb)) return fail(ctx, PT_EINVAL, "bad pixel list or output");
    if (n_pix == 0) return PT_OK;
    const int64_t n_slots = n_pix * (int64_t)cfg->spp;
    if (n_slots > 0xFFFFFFFFll) return fail(ctx, PT_EINVAL, "more than 2^32 - 1 paths in one call");
    if (sc->dev.env_is_nif && cfg->precision != PT_FP32 && !(cfg->precision == PT_BF16 && nf->d_tc) &&
        !(cfg->precision == PT_FP8E4M3 && nf->fp8_ok))
        return fail(ctx, PT_EUNSUPPORTED, "no BF16 kernel for this NIF shape (F = 64 with H = 128 and L <= 5, H = 64 or 32 and L <= 8, H = 256 and L = 1; the paper's F = 20 skip network); FP8: F = 64, H = 128, L = 3");
    // chunk = whole samples
    int64_t chunk = cfg->chunk_slots > 0 ? cfg->chunk_slots : (int64_t)1 << 24;
    chunk = std::max<int64_t>(n_pix, (chunk / n_pix) * n_pix);
    chunk = std::min(chunk, n_slots);
    if (chunk > 0x7FFFFFFFll) chunk = (0x7FFFFFFFll / n_pix) * n_pix;
    st = ensure_scratch(ctx, (uint32_t)chunk);
    if (st != PT_OK) return st;
    if (cache && ctx->cache_cap < (uint32_t)chunk) {
        cudaFree(ctx->cache_rows);
        ctx->cache_rows = nullptr;
        ctx->cache_cap = 0;
        if (dalloc(&ctx->cache_rows, (size_t)chunk * 16)) return fail(ctx, PT_ENOMEM, "cache query rows allocation failed");
        ctx->cache_cap = (uint32_t)chunk;
        ++ctx->scratch_gen;
    }
    // host-side work a launch might otherwise do (the lazy FP8 image) happens before any capture
    if (sc->dev.env_is_nif && cfg->precision == PT_FP8E4M3 && nf->fp8_ok) {
        st = ensure_fp8(ctx, nf, s);
        if (st != PT_OK) return st;
    }
    ctx->last_depth = cfg->max_depth;
    ctx->last_schedule = use_paths(ctx, sc, cfg, n_slots - ((n_slots + chunk - 1) / chunk - 1) * chunk)
                             ? PT_SCHED_PATHS : PT_SCHED_WAVEFRONT;
    PT_CUDA(launch_set_u32(ctx->d_first_sample, first_sample, s));
    auto direct = [&](cudaStream_t st_) {
        return render_launches(ctx, sc, nf, cfg, cache, cache_vertex, rec_vertex, d_rec, n_pix, d_pixels, d_pixel_rgb,
                               d_slot_rgb, d_hit_ids, n_slots, chunk, st_);
    };
    if (ctx->prof_on) return direct(s);   // per-kernel events need the launches themselves
    GraphKey key;
    std::memset(&key, 0, sizeof key);
    key.sc_uid = sc->uid;
    key.nf_uid = nf ? nf->uid : 0;
    key.nf_version = nf ? nf->version : 0;
    key.cache_uid = cache ? cache->uid : 0;
    key.scratch_gen = ctx->scratch_gen;
    key.width = cfg->width; key.height = cfg->height; key.spp = cfg->spp; key.max_depth = cfg->max_depth;
    key.rr = cfg->rr; key.rr_start = cfg->rr_start; key.precision = cfg->precision;
    key.cache_vertex = cache_vertex; key.rec_vertex = rec_vertex; key.schedule = cfg->schedule;
    key.seed = cfg->seed; key.cache_cap = ctx->cache_cap;
    key.chunk = chunk; key.n_pix = n_pix;
    key.ptrs[0] = d_rec; key.ptrs[1] = d_pixels; key.ptrs[2] = d_pixel_rgb; key.ptrs[3] = d_slot_rgb;
    key.ptrs[4] = d_hit_ids;
    std::vector<unsigned char> kb(sizeof key);
    std::memcpy(kb.data(), &key, sizeof key);
    for (auto& g : ctx->graphs)
        if (g.key == kb) {
            PT_CUDA(cudaGraphLaunch(g.exec, s));
            count_launch(g.kernels);
            return PT_OK;
        }
    // a render seen for the first time launches directly (one-off renders never pay for a capture)
    bool seen = false;
    for (auto& k : ctx->graph_seen) seen = seen || k == kb;
    if (!seen) {
        if (ctx->graph_seen.size() < kMaxGraphs) {
            ctx->graph_seen.push_back(kb);
        } else {
            ctx->graph_seen[ctx->seen_next] = kb;
            ctx->seen_next = (ctx->seen_next + 1) % kMaxGraphs;
        }
        return direct(s);
    }
    // record the sequence on the capture stream (nothing runs there), instantiate, replay on `s`
    if (!ctx->cap_stream) PT_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const unsigned long long before = t_kernels_launched;
        const pt_status lst = direct(ctx->cap_stream);
        // the launches of a capture only record kernels: they count when the graph is launched
        const unsigned long long kernels = t_kernels_launched - before;
        g_kernels_launched.fetch_sub(kernels, std::memory_order_relaxed);
        t_kernels_launched = before;
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
        cudaGraphExec_t exec = nullptr;
        if (lst == PT_OK && ce == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
            cudaGraphDestroy(graph);
            if (ctx->graphs.size() < kMaxGraphs) {
                ctx->graphs.push_back({kb, exec, kernels});
            } else {
                cudaGraphExecDestroy(ctx->graphs[ctx->graph_next].exec);
                ctx->graphs[ctx->graph_next] = {kb, exec, kernels};
                ctx->graph_next = (ctx->graph_next + 1) % kMaxGraphs;
            }
            PT_CUDA(cudaGraphLaunch(exec, s));
            count_launch(kernels);
            return PT_OK;
        }
        if (graph) cudaGraphDestroy(graph);
    }
    (void)cudaGetLastError();   // a failed capture leaves nothing behind: launch directly
    return direct(s);
}


PT_API pt_status pt_render_pixels(pt_ctx* ctx, const pt_scene* sc, const pt_nif* nf, const pt_render_cfg* cfg,
                                  int64_t n_pix, const int64_t* d_pixels, float* d_pixel_rgb, float* d_slot_rgb,
                                  int32_t* d_hit_ids, void* stream)
{
    pt_status st = check_cfg(ctx, sc, nf, cfg);
    if (st != PT_OK) return st;
    if (cfg->cache_vertex != 0) return fail(ctx, PT_EINVAL, "cache_vertex needs a cache (pt_render, pt_render_cached)");
    return render_impl(ctx, sc, nf, cfg, (uint32_t)cfg->first_sample, nullptr, 0, 0, nullptr, n_pix, d_pixels,
                       d_pixel_rgb, d_slot_rgb, d_hit_ids, (cudaStream_t)stream);
}

PT_API pt_status pt_render_cached(pt_ctx* ctx, const pt_scene* sc, const pt_nif* nf, const pt_cache* cache,
                                  int32_t cache_vertex, int32_t rec_vertex, const pt_render_cfg* cfg, int64_t n_pix,
                                  const int64_t* d_pixels, float* d_pixel_rgb, float* d_slot_rgb, float* d_rec,
                                  int32_t* d_hit_ids, void* stream)
{
    pt_status st = check_cfg(ctx, sc, nf, cfg);
    if (st != PT_OK) return st;
    if ((cache != nullptr) != (cache_vertex != 0) || cache_vertex < 0 || cache_vertex == 1)
        return fail(ctx, PT_EINVAL, "cache and cache_vertex >= 2 go together");
    if (cfg->cache_vertex != 0 && cfg->cache_vertex != cache_vertex)
        return fail(ctx, PT_EINVAL, "cfg->cache_vertex differs from the cache_vertex argument");
    if (cache && cache->ctx->device != ctx->device) return fail(ctx, PT_EINVAL, "cache lives on another device");
    if (rec_vertex < 0 || rec_vertex > cfg->max_depth || (rec_vertex > 0 && !d_rec))
        return fail(ctx, PT_EINVAL, "rec_vertex must be in [0, max_depth] with d_rec");
    return render_impl(ctx, sc, nf, cfg, (uint32_t)cfg->first_sample, cache, cache_vertex, rec_vertex, d_rec, n_pix,
                       d_pixels, d_pixel_rgb, d_slot_rgb, d_hit_ids, (cudaStream_t)stream);
}

PT_API pt_status pt_render(pt_ctx* ctx, const pt_scene* sc, const pt_nif* nf, const pt_cache* cache,
                           const pt_render_cfg* cfg, float* d_image, void* stream)
{
    if (!d_image) return fail(ctx, PT_EINVAL, "null image");
    if (!cfg) return fail(ctx, PT_EINVAL, "null cfg");
    if (!cache) return pt_render_pixels(ctx, sc, nf, cfg, 0, nullptr, d_image, nullptr, nullptr, stream);
    if (cfg->cache_vertex < 2) return fail(ctx, PT_EINVAL, "a cache needs cfg->cache_vertex >= 2");
    return pt_render_cached(ctx, sc, nf, cache, cfg->cache_vertex, 0, cfg, 0, nullptr, d_image, nullptr, nullptr,
                            nullptr, stream);
}

PT_API pt_status pt_kernel_launches(uint64_t* count)
{
    if (!count) return PT_EINVAL;
    *count = g_kernels_launched.load(std::memory_order_relaxed);
    return PT_OK;
}

PT_API pt_status pt_last_render_schedule(pt_ctx* ctx, int32_t* schedule)
{
    if (!ctx || !schedule) return fail(ctx, PT_EINVAL, "bad argument");
    *schedule = ctx->last_schedule;
    return PT_OK;
}

PT_API pt_status pt_last_render_work(pt_ctx* ctx, int64_t* work, int32_t n)
{
    if (!ctx || !work || n < 0) return fail(ctx, PT_EINVAL, "bad argument");
    unsigned long long h[4] = {0, 0, 0, 0};
    PT_CUDA(cudaDeviceSynchronize());
    PT_CUDA(cudaMemcpy(h, ctx->stats + kWorkBase, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) work[i] = i < 4 ? (int64_t)h[i] : 0;
    return PT_OK;
}

PT_API pt_status pt_last_render_counts(pt_ctx* ctx, int64_t* counts, int32_t n)
{
    if (!ctx || !counts || n < 0) return fail(ctx, PT_EINVAL, "bad argument");
    std::vector<unsigned long long> h(kStats);
    PT_CUDA(cudaDeviceSynchronize());
    PT_CUDA(cudaMemcpy(h.data(), ctx->stats, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    const int D = ctx->last_depth;
    for (int i = 0; i < n; ++i)
        counts[i] = (i < D) ? (int64_t)h[i] : (i == D ? (int64_t)h[D] : (i == D + 1 ? (int64_t)h[kCacheStat] : 0));
    return PT_OK;
}

// ---------------------------------------------------------------------------
PT_API pt_status pt_philox(pt_ctx* ctx, uint32_t seed, uint32_t tag, int64_t n, const uint32_t* d_ctr, uint32_t* d_out,
                           void* stream)
{
    if (!ctx || n < 0 || (n > 0 && (!d_ctr || !d_out))) return fail(ctx, PT_EINVAL, "bad argument");
    PT_CUDA(launch_philox(seed, tag, n, d_ctr, d_out, (cudaStream_t)stream));
    return PT_OK;
}

PT_API pt_status pt_primary_rays(pt_ctx* ctx, const pt_scene* sc, const pt_render_cfg* cfg, int64_t first_slot,
                                 int64_t n, float* d_org, float* d_dir, void* stream)
{
    if (!ctx || !sc || !cfg || n < 0 || first_slot < 0 || (n > 0 && (!d_org || !d_dir)))
        return fail(ctx, PT_EINVAL, "bad argument");
    if (cfg->width < 1 || cfg->height < 1) return fail(ctx, PT_EINVAL, "image size must be >= 1");
    DevScene v = sc->dev;
    v.aspect = (float)((double)cfg->width / (double)cfg->height);
    PT_CUDA(launch_primary(v, cfg->width, cfg->height, cfg->seed, (uint32_t)cfg->first_sample, first_slot, n, d_org, d_dir,
                           (cudaStream_t)stream));
    return PT_OK;
}

PT_API pt_status pt_trace_rays(pt_ctx* ctx, const pt_scene* sc, int64_t n, const float* d_org, const float* d_dir,
                               float* d_t, int32_t* d_prim, void* stream)
{
    if (!ctx || !sc || n < 0 || (n > 0 && (!d_org || !d_dir || !d_t || !d_prim)))
        return fail(ctx, PT_EINVAL, "bad argument");
    PT_CUDA(launch_trace_rays(sc->dev, n, d_org, d_dir, d_t, d_prim, ctx->d_err, (cudaStream_t)stream));
    return PT_OK;
}

PT_API pt_status pt_profile_enable(pt_ctx* ctx, int32_t enable)
{
    if (!ctx) return PT_EINVAL;
    ctx->prof_on = enable != 0;
    ctx->prof_used = 0;
    return PT_OK;
}

PT_API pt_status pt_profile_read(pt_ctx* ctx, double* ms, int64_t* launches, int32_t n)
{
    if (!ctx || n < 0) return fail(ctx, PT_EINVAL, "bad argument");
    PT_CUDA(cudaDeviceSynchronize());
    double acc[PT_N_KINDS] = {};
    int64_t cnt[PT_N_KINDS] = {};
    for (size_t i = 0; i < ctx->prof_used; ++i) {
        float t = 0.f;
        PT_CUDA(cudaEventElapsedTime(&t, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]));
        acc[ctx->prof_kind[i]] += t;
        cnt[ctx->prof_kind[i]] += 1;
    }
    ctx->prof_used = 0;
    for (int k = 0; k < n && k < PT_N_KINDS; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = cnt[k];
    }
    return PT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoints (format in pt.h)
namespace {

struct CkptHeader {
    char magic[8];
    uint32_t kind, version;
    int32_t dims[4];
    float box[6];
    int64_t n_params, n_adam, adam_t;
};
static_assert(sizeof(CkptHeader) == 80, "checkpoint header layout");
constexpr char kCkptMagic[8] = {'P', 'T', 'C', 'K', 'P', 'T', '0', '1'};
constexpr uint32_t kCkptVersion = 1;

uint64_t fnv1a(uint64_t h, const void* data, size_t n)
{
    const unsigned char* p = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}
constexpr uint64_t kFnvBasis = 14695981039346656037ull;

// header + host arrays -> file; false when any write fails
bool write_ckpt(const char* path, const CkptHeader& hd, const std::vector<float>& params, const std::vector<float>& m,
                const std::vector<float>& v)
{
    FILE* f = std::fopen(path, "wb");
    if (!f) return false;
    uint64_t h = kFnvBasis;
    bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1;
    h = fnv1a(h, &hd, sizeof hd);
    for (const std::vector<float>* a : {&params, &m, &v}) {
        if (!ok || a->empty()) continue;
        ok = std::fwrite(a->data(), sizeof(float), a->size(), f) == a->size();
        h = fnv1a(h, a->data(), a->size() * sizeof(float));
    }
    ok = ok && std::fwrite(&h, sizeof h, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    return ok;
}

// file -> header + arrays, checked: magic, version, sizes against the file length, hash
pt_status read_ckpt(pt_ctx* ctx, const char* path, CkptHeader& hd, std::vector<float>* params, std::vector<float>* m,
                    std::vector<float>* v)
{
    if (!path) return fail(ctx, PT_EINVAL, "null path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(ctx, PT_EIO, std::string("cannot open checkpoint ") + path);
    std::fseek(f, 0, SEEK_END);
    const long len = std::ftell(f);
    std::fseek(f, 0, SEEK_SET);
    if (len < (long)(sizeof hd + 8) || std::fread(&hd, sizeof hd, 1, f) != 1) {
        std::fclose(f);
        return fail(ctx, PT_EIO, "checkpoint truncated");
    }
    if (std::memcmp(hd.magic, kCkptMagic, 8) != 0) {
        std::fclose(f);
        return fail(ctx, PT_EIO, "not a checkpoint (magic)");
    }
    if (hd.version != kCkptVersion) {
        std::fclose(f);
        return fail(ctx, PT_EINVAL, "unknown checkpoint version");
    }
    if (hd.n_params < 1 || hd.n_adam < 0 || hd.n_params > ((int64_t)1 << 28) || hd.n_adam > hd.n_params ||
        (long)(sizeof hd + 4 * (hd.n_params + 2 * hd.n_adam) + 8) != len) {
        std::fclose(f);
        return fail(ctx, PT_EIO, "checkpoint sizes do not match the file");
    }
    std::vector<float> P((size_t)hd.n_params), M((size_t)hd.n_adam), V((size_t)hd.n_adam);
    uint64_t stored = 0;
    bool ok = std::fread(P.data(), sizeof(float), P.size(), f) == P.size();
    if (ok && hd.n_adam > 0) {
        ok = std::fread(M.data(), sizeof(float), M.size(), f) == M.size() &&
             std::fread(V.data(), sizeof(float), V.size(), f) == V.size();
    }
    ok = ok && std::fread(&stored, sizeof stored, 1, f) == 1;
    std::fclose(f);
    if (!ok) return fail(ctx, PT_EIO, "checkpoint truncated");
    uint64_t h = fnv1a(kFnvBasis, &hd, sizeof hd);
    h = fnv1a(h, P.data(), P.size() * sizeof(float));
    h = fnv1a(h, M.data(), M.size() * sizeof(float));
    h = fnv1a(h, V.data(), V.size() * sizeof(float));
    if (h != stored) return fail(ctx, PT_EIO, "checkpoint hash mismatch (corrupted)");
    if (params) *params = std::move(P);
    if (m) *m = std::move(M);
    if (v) *v = std::move(V);
    return PT_OK;
}

pt_status download(pt_ctx* ctx, const float* d, int64_t n, std::vector<float>& out)
{
    out.resize((size_t)n);
    if (n > 0) PT_CUDA(cudaMemcpy(out.data(), d, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));
    return PT_OK;
}

}  // namespace

PT_API pt_status pt_checkpoint_read_info(const char* path, pt_checkpoint_info* out)
{
    if (!out) return PT_EINVAL;
    CkptHeader hd = {};
    const pt_status st = read_ckpt(nullptr, path, hd, nullptr, nullptr, nullptr);
    if (st != PT_OK) return st;
    *out = pt_checkpoint_info{};
    out->kind = (int32_t)hd.kind;
    out->version = (int32_t)hd.version;
    for (int i = 0; i < 4; ++i) out->dims[i] = hd.dims[i];
    for (int a = 0; a < 3; ++a) {
        out->lo[a] = hd.box[a];
        out->hi[a] = hd.box[3 + a];
    }
    out->n_params = hd.n_params;
    out->n_adam = hd.n_adam;
    out->adam_t = hd.adam_t;
    return PT_OK;
}

PT_API pt_status pt_save_nif(pt_ctx* ctx, const pt_nif* nf, const char* path, void* stream)
{
    if (!ctx || !nf || !path) return fail(ctx, PT_EINVAL, "null argument");
    PT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    CkptHeader hd = {};
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.kind = 1;
    hd.version = kCkptVersion;
    hd.dims[0] = nf->F;
    hd.dims[1] = nf->H;
    hd.dims[2] = nf->L;
    hd.dims[3] = nf->skip;
    hd.n_params = nf->n_params;
    hd.n_adam = nf->d_m ? nf->n_trainable : 0;
    hd.adam_t = nf->adam_t;
    std::vector<float> P, M, V;
    pt_status st = download(ctx, nf->d_params, nf->n_params, P);
    if (st == PT_OK && hd.n_adam) st = download(ctx, nf->d_m, hd.n_adam, M);
    if (st == PT_OK && hd.n_adam) st = download(ctx, nf->d_v, hd.n_adam, V);
    if (st != PT_OK) return st;
    if (!write_ckpt(path, hd, P, M, V)) return fail(ctx, PT_EIO, std::string("cannot write checkpoint ") + path);
    return PT_OK;
}

PT_API pt_status pt_load_nif_file(pt_ctx* ctx, const char* path, pt_nif** out)
{
    if (!ctx || !out) return fail(ctx, PT_EINVAL, "null argument");
    *out = nullptr;
    CkptHeader hd = {};
    std::vector<float> P, M, V;
    pt_status st = read_ckpt(ctx, path, hd, &P, &M, &V);
    if (st != PT_OK) return st;
    if (hd.kind != 1) return fail(ctx, PT_EINVAL, "checkpoint is not a NIF");
    pt_nif_desc d = {};
    d.n_freq = hd.dims[0];
    d.hidden = hd.dims[1];
    d.n_hidden_layers = hd.dims[2];
    d.skip_after = hd.dims[3];
    d.params = P.data();
    // the parameter count implied by the dimensions must be the file's before anything reads P
    {
        const int F = d.n_freq, H = d.hidden, L = d.n_hidden_layers, S = d.skip_after;
        if (F < 1 || F > 64 || H < 1 || H > 256 || L < 1 || L > 8 || S < 0 || S >= L || (S > 0 && H <= 2 * F))
            return fail(ctx, PT_EIO, "checkpoint dimensions out of range");
        int64_t n = 2 * (int64_t)F + 9;
        for (int l = 0; l <= L; ++l) {
            int in, o;
            nif_layer_dims(F, H, L, S, l, &in, &o);
            n += (int64_t)in * o + o;
        }
        if (n != hd.n_params || (hd.n_adam && hd.n_adam != n - 2 * F - 9))
            return fail(ctx, PT_EIO, "checkpoint sizes do not match its dimensions");
    }
    pt_nif* nf = nullptr;
    st = pt_load_nif(ctx, &d, &nf);
    if (st != PT_OK) return st;
    if (hd.n_adam) {
        st = ensure_train(ctx, nf, 0);
        if (st == PT_OK && (cudaMemcpy(nf->d_m, M.data(), M.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
                            cudaMemcpy(nf->d_v, V.data(), V.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess))
            st = fail(ctx, PT_ECUDA, "training state upload failed");
        if (st != PT_OK) {
            pt_destroy_nif(nf);
            return st;
        }
    }
    nf->adam_t = hd.adam_t;
    *out = nf;
    return PT_OK;
}

PT_API pt_status pt_save_cache(pt_ctx* ctx, const pt_cache* c, const char* path, void* stream)
{
    if (!ctx || !c || !path) return fail(ctx, PT_EINVAL, "null argument");
    PT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    CkptHeader hd = {};
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.kind = 2;
    hd.version = kCkptVersion;
    hd.dims[0] = c->J;
    hd.dims[1] = c->H;
    hd.dims[2] = c->L;
    for (int a = 0; a < 3; ++a) {
        hd.box[a] = c->box_lo[a];
        hd.box[3 + a] = c->box_hi[a];
    }
    hd.n_params = c->n_params;
    hd.n_adam = c->d_m ? c->n_params : 0;
    hd.adam_t = c->adam_t;
    std::vector<float> P, M, V;
    pt_status st = download(ctx, c->d_params, c->n_params, P);
    if (st == PT_OK && hd.n_adam) st = download(ctx, c->d_m, hd.n_adam, M);
    if (st == PT_OK && hd.n_adam) st = download(ctx, c->d_v, hd.n_adam, V);
    if (st != PT_OK) return st;
    if (!write_ckpt(path, hd, P, M, V)) return fail(ctx, PT_EIO, std::string("cannot write checkpoint ") + path);
    return PT_OK;
}

PT_API pt_status pt_load_cache_file(pt_ctx* ctx, const char* path, pt_cache** out)
{
    if (!ctx || !out) return fail(ctx, PT_EINVAL, "null argument");
    *out = nullptr;
    CkptHeader hd = {};
    std::vector<float> P, M, V;
    pt_status st = read_ckpt(ctx, path, hd, &P, &M, &V);
    if (st != PT_OK) return st;
    if (hd.kind != 2) return fail(ctx, PT_EINVAL, "checkpoint is not a radiance cache");
    pt_cache_desc d = {};
    d.n_freq = hd.dims[0];
    d.hidden = hd.dims[1];
    d.n_hidden_layers = hd.dims[2];
    d.params = P.data();
    for (int a = 0; a < 3; ++a) {
        d.lo[a] = hd.box[a];
        d.hi[a] = hd.box[3 + a];
    }
    // the parameter count implied by the dimensions must be the file's before anything reads P
    const int64_t J = d.n_freq, H = d.hidden, L = d.n_hidden_layers, in0 = 6 * J + 6;
    if (J < 1 || J > 15 || H < 1 || H > 128 || L < 1 || L > 7 ||
        in0 * H + H + (L - 1) * (H * H + H) + 3 * H + 3 != hd.n_params ||
        (hd.n_adam && hd.n_adam != hd.n_params))
        return fail(ctx, PT_EIO, "checkpoint sizes do not match its dimensions");
    pt_cache* c = nullptr;
    st = pt_create_cache(ctx, &d, &c);
    if (st != PT_OK) return st;
    if (hd.n_adam) {
        st = ensure_cache_train(ctx, c, 0);
        if (st == PT_OK && (cudaMemcpy(c->d_m, M.data(), M.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
                            cudaMemcpy(c->d_v, V.data(), V.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess))
            st = fail(ctx, PT_ECUDA, "training state upload failed");
        if (st != PT_OK) {
            pt_destroy_cache(c);
            return st;
        }
    }
    c->adam_t = hd.adam_t;
    *out = c;
    return PT_OK;
}

// ---------------------------------------------------------------------------
PT_API pt_status pt_selftest_wait_timeout(pt_ctx* ctx, double seconds, double* waited_s, void* stream)
{
    if (!ctx) return PT_EINVAL;
    if (!(seconds > 0.0 && seconds <= 2.0)) return fail(ctx, PT_EINVAL, "seconds must be in (0, 2]");
    PT_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* d_waited = nullptr;
    PT_CUDA(cudaMalloc((void**)&d_waited, sizeof(uint64_t)));
    cudaError_t e = wait_selftest(ctx->d_err, (uint64_t)(seconds * 1e9), d_waited, s);
    uint64_t waited = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&waited, d_waited, sizeof waited, cudaMemcpyDeviceToHost);
    cudaFree(d_waited);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "wait self-test");
    if (waited_s) *waited_s = (double)waited * 1e-9;
    return PT_OK;
}
