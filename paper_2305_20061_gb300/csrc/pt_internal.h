// Internal data layouts shared by the library's host and device sources.
// Nothing here is part of the C ABI (include/pt.h).
#pragma once

#include <atomic>
#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "pt.h"

namespace ptk {

// Kernels this library has put on a stream, process-wide: every launch site
// counts itself, and a CUDA-graph replay adds the kernels its graph holds
// (launches recorded during a capture are taken back out).
extern std::atomic<unsigned long long> g_kernels_launched;
extern thread_local unsigned long long t_kernels_launched;   // this thread's share (graph capture)
inline void count_launch(unsigned long long n = 1)
{
    g_kernels_launched.fetch_add(n, std::memory_order_relaxed);
    t_kernels_launched += n;
}

constexpr uint32_t kLeafBit = 0x80000000u;   // child reference is a primitive
constexpr uint32_t kEmptyRef = 0xFFFFFFFFu;  // empty scene
constexpr int kStackSize = 64;               // traversal stack entries per ray
constexpr uint32_t kIterCap = 1u << 22;      // node visits per ray before giving up

// Packed BVH node: the two children's boxes live in the parent (one fetch
// tests both), each as fp32 origin + fp16 extent rounded up so the decoded
// box contains the exact one (Section 3.1.4's "round-to-nearest-not-lower").
// 48 bytes = three 128-bit loads:
//   q0 = lo_l.x lo_l.y lo_l.z lo_r.x
//   q1 = lo_r.y lo_r.z (ext_l.x|ext_l.y<<16) (ext_l.z|ext_r.x<<16)
//   q2 = (ext_r.y|ext_r.z<<16) child_l child_r 0
// A child reference with kLeafBit set holds a global primitive ID.
struct PackedNode { uint32_t w[12]; };
static_assert(sizeof(PackedNode) == 48, "node packing");

// Quantised BVH node (the paper's "quarter precision" outlook, Section 5):
// the same tree as PackedNode, both children's boxes on an 8-bit grid of the
// node, 32 bytes = two 128-bit loads = one DRAM sector:
//   q0 = origin.x origin.y origin.z meta
//   q1 = refs qbytes[0..3] qbytes[4..7] qbytes[8..11]
// origin: per-axis minimum of the two children's decoded boxes (fp32).
// meta: bits 0-7 e (biased fp32 exponent), 8-9 / 10-11 / 12-13 the axis
// offsets dx, dy, dz (0..3), bit 14 left child is a primitive, bit 15 right
// child is a primitive, bits 16-31 the low 16 bits of the left reference.
// refs: bits 0-7 the high 8 bits of the left reference, bits 8-31 the right
// reference (24-bit node index or primitive ID).
// qbytes: lo_l.xyz hi_l.xyz lo_r.xyz hi_r.xyz; axis a's grid step is
// s_a = 2^(e - 127 - d_a) and a bound decodes as origin_a + q * s_a in fp32
// (the product is exact, the sum rounds to nearest), which the builder
// checks to contain the fp16-extent box (lo rounded down, hi up).
struct QuantNode { uint32_t w[8]; };
static_assert(sizeof(QuantNode) == 32, "quantised node packing");
constexpr uint32_t kQuantRefLimit = 1u << 24;   // node indices and primitive IDs a quantised node can hold

// Device view of a scene (passed by value in kernel parameters).
struct DevScene {
    const uint4* nodes;     // 3 x uint4 per node
    // nullable: the same tree with both child boxes decoded to fp32 (lo, hi), 4 x uint4 per node:
    //   lo_l.xyz hi_l.x | hi_l.yz lo_r.xy | lo_r.z hi_r.xyz | child_l child_r 0 0
    // kept for BVHs small enough to stay cache-resident, where decoding costs more than the bytes
    const uint4* wnodes;
    // nullable: the same tree as QuantNode, 2 x uint4 per node; when set, traversal reads this form
    const uint4* qnodes;
    uint32_t root;          // node index, leaf reference, or kEmptyRef
    uint32_t n_nodes;
    uint32_t nS, nQ, nT;    // primitive counts; IDs: [0,nS) spheres, [nS,nS+nQ) quads, rest triangles
    const float4* sph;      // (cx, cy, cz, r)
    const float4* quad;     // 2 per quad: (p, lo_u, hi_u, lo_v), (hi_v, axis, 0, 0)
    const float4* tri;      // 3 per triangle: v0, v1, v2 (w = 0)
    const int32_t* prim_mat;  // material per global primitive
    const float4* mat;      // 2 per material: (albedo rgb, roughness), (ior, emission rgb)
    const int32_t* mat_type;
    // camera (basis computed on the host in double, stored in float)
    float eye[3], right[3], up[3], fwd[3];
    float tan_half, aspect;
    int32_t env_is_nif;
    float env[3];
    int32_t has_emission;
};

// Escape queue handed from the shading kernel to the NIF kernel, as two
// arrays (24 B per escape): the NIF loads each part of an escape with one
// coalesced vector load per lane, not three 8-byte loads at a 24-byte stride.
struct EscapeQueue {
    float2* uv;             // [i] equirect (u, v) of the escape direction
    float4* tp;             // [i] path throughput (x, y, z) and the chunk-relative slot (w, as the uint32 bits)
};
constexpr size_t kEscapeBytes = sizeof(float2) + sizeof(float4);

// Ray queue in structure-of-arrays form (one float4 stream per field).
struct RayQueue {
    float4* o;   // origin xyz, w = chunk-relative slot (bits)
    float4* d;   // direction xyz
    float4* tp;  // throughput rgb
    float4* L;   // radiance gathered so far (only when the scene emits)
};

struct BounceParams {
    DevScene sc;
    int32_t k;              // vertex index of the rays traced now (1 = camera rays)
    int32_t max_depth;
    int32_t rr, rr_start;
    uint32_t seed;
    uint32_t first_sample;  // sample index offset (Philox counter word 1), unless first_sample_dev is set
    const uint32_t* first_sample_dev;   // nullable: the offset read on the device (one captured launch
                                        // sequence then serves every frame)
    uint64_t chunk_first;   // global slot of the chunk's first path
    uint32_t n_chunk;       // paths in the chunk
    uint32_t n_pix;
    const int64_t* pixels;  // nullable pixel list
    int32_t W, H;
    int32_t tiled;          // camera rays taken in 8x4-pixel tiles (whole images with W % 8 == 0, H % 4 == 0)
    RayQueue qin;           // unused when k == 1
    const uint32_t* count_in;
    RayQueue qout;
    uint32_t* count_out;
    uint32_t cap;
    EscapeQueue esc;
    uint32_t* esc_count;
    float* slot_L;          // [n_chunk][3]
    int32_t* hit_ids;       // nullable [global slot][max_depth]
    uint32_t* err;
    unsigned long long* stats;  // [max_depth + 1]
    unsigned long long* work;   // nullable [4]: node fetches, sphere, quad, triangle tests
    // radiance cache: a path that hits at vertex cache_vertex (0 = off) ends
    // there with a query row (16 floats) appended to cache_rows
    int32_t cache_vertex;
    float* cache_rows;
    uint32_t* cache_count;
    // vertex records: the state at vertex rec_vertex (0 = off) of each path,
    // rec [global slot][16] (the caller clears the valid words beforehand)
    int32_t rec_vertex;
    float* rec;
    // traversal results handed from k_trace to the shading kernel: (t bits, primitive) per queue entry
    int2* hits;
    uint32_t* fetch;        // ray-index claim counter of k_trace (zero before the launch)
};

// NIF parameters on the device.
// Widths of linear layer l (0 .. L, L = the head) of a NIF with F frequencies, width H, L hidden layers and
// skip layer `skip` (0: none; s >= 1: hidden layer s has H - 2F outputs and layer s + 1 takes them with the
// 2F Fourier features appended, Section 3.2).
#ifdef __CUDACC__
#define PT_HOST_DEVICE __host__ __device__
#else
#define PT_HOST_DEVICE
#endif
PT_HOST_DEVICE inline void nif_layer_dims(int F, int H, int L, int skip, int l, int* in, int* out)
{
    *in = l == 0 ? 2 * F : H;
    *out = l == L ? 3 : (skip > 0 && l == skip - 1 ? H - 2 * F : H);
}

// padded width D of the FP32 evaluation layout: 128, or 256 for networks wider than 128
PT_HOST_DEVICE inline int nif_fp32_width(int H) { return H > 128 ? 256 : 128; }

struct DevNif {
    int32_t F, H, L;         // frequencies, hidden width, hidden layers
    int32_t skip;            // 0, or the hidden layer whose output is joined with the features (1-based)
    int32_t D;               // padded width of the FP32 layout (nif_fp32_width(H))
    const float* B;          // [F][2]
    // FP32 path: each linear layer padded to D x D and stored transposed
    // ([in][out]); the output layer is stored [3][H] untransposed
    const float* Wt;         // [L][D][D]
    const float* bias;       // [L][D]
    const float* Wout;       // [3][D]
    const float* bout;       // [3]
    float M[9];
};

struct NifEvalParams {
    DevNif nif;
    // mode 0: plain evaluation of uv[] -> rgb[]
    const float* uv;
    float* rgb;
    int64_t n;
    // mode 1: escape records -> slot radiance += tp * rgb
    EscapeQueue esc;
    const uint32_t* esc_count;
    uint32_t esc_cap;
    float* slot_L;
    int accumulate;         // 1: slot radiance += tp * rgb; 0: slot radiance = tp * rgb (no emitters)
    uint32_t* err;
    unsigned long long* stats;
};

// kernel launchers (trace.cu)
cudaError_t launch_bounce(const BounceParams& p, int sm_count, cudaStream_t s);   // launch_trace + launch_shade
cudaError_t launch_trace(const BounceParams& p, int sm_count, cudaStream_t s);    // closest hits of vertex k
cudaError_t launch_shade(const BounceParams& p, int sm_count, cudaStream_t s);    // shading + compaction
// path-per-thread schedule: every vertex of the chunk's paths in one launch;
// resident_threads (from paths_resident_threads) caps the grid at one wave
cudaError_t launch_paths(const BounceParams& p, int resident_threads, cudaStream_t s);
// threads of k_paths resident at once on the device (0 if the query failed)
int paths_resident_threads(int form, int sm_count);   // form: node form of the traversal (device_common.cuh)
// Looks up (once per device; `device` current) the fixed scratch array of
// pt_render_noalloc, which makes the driver load and reserve it.
cudaError_t noalloc_setup(int device, unsigned char** out);
cudaError_t launch_reduce(const float* slot_L, float* pix, uint32_t n_pix, uint32_t s_count, int first, float scale,
                          cudaStream_t s);
cudaError_t launch_fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s);
cudaError_t launch_philox(uint32_t seed, uint32_t tag, int64_t n, const uint32_t* ctr, uint32_t* out, cudaStream_t s);
cudaError_t launch_primary(const DevScene& sc, int W, int H, uint32_t seed, uint32_t first_sample, int64_t first,
                           int64_t n, float* org, float* dir, cudaStream_t s);
cudaError_t launch_trace_rays(const DevScene& sc, int64_t n, const float* org, const float* dir, float* t,
                              int32_t* prim, uint32_t* err, cudaStream_t s);
// NIF kernels (nif_fp32.cu)
cudaError_t launch_nif_fp32(const NifEvalParams& p, int mode, int sm_count, cudaStream_t s);

// tensor-core NIF (nif_tc.cu): F = 64; H = 128 with L = 1 .. 5, H = 64 or 32 with L = 1 .. 8 hidden layers
// (weights resident in shared memory)
// the BF16 tensor-core NIF: shapes (F, H, L, skip layer) with a kernel, image packing, launch
bool nif_tc_supported(int F, int H, int L, int S);
bool pack_nif_tc_image(const float* params, int F, int H, int L, int S, std::vector<unsigned char>& out);
cudaError_t launch_nif_tc(const unsigned char* image, int F, int H, int L, int S, const NifEvalParams& p, int mode,
                          int sm_count, cudaStream_t s);
// FP8 E4M3 tensor-core NIF (nif_fp8.cu): same shape; scales_out [4] = activation scales
bool pack_nif_fp8_image(const float* params, int F, int H, int L, std::vector<unsigned char>& out, float* scales_out);
cudaError_t launch_nif_fp8(const unsigned char* image, const NifEvalParams& p, int mode, int sm_count, cudaStream_t s);

// NIF training (train.cu).  Pointers into the flat FP32 master weights and
// into the flat gradient (same order as the trainable part of the weights).
struct TrainNet {
    int32_t F, H, L;
    int32_t in0;                    // width of layer 0's input (2F for the NIF, 6J + 6 for the cache)
    int32_t skip;                   // NIF skip layer (1-based) or 0; its output is joined with the features
    int32_t in[9], out[9];          // widths of each linear layer
    const float* B;                 // [F][2]
    const float* W[9];              // per linear layer, [out][in]
    const float* b[9];
    const float* M;                 // [3][3]
    float* gW[9];
    float* gb[9];
};
struct TrainWork {
    int32_t n_blocks;               // partial slots allocated (at most this many CTAs per launch)
    int32_t sm_count;
    float* X[9];                    // X[0] features, X[l] hidden outputs, each [batch][128]
    float* dX[2];                   // ping-pong [batch][128]
    unsigned char* Xb[8];           // tensor-core path: BF16 operand tiles of X[l] and of the gradient G[l] at
    unsigned char* Gb[8];           // layer l's pre-activation, l < L; [128-row tile][core-matrix layout]
    float* partial;                 // [n_blocks][128 * 128 + 128]
    double* loss_partial;           // [n_blocks]
    unsigned int* err;              // PT_ERR_* word of the context
};
cudaError_t train_inputs(uint32_t seed, uint32_t step, int64_t B, const float* sky, int w, int h, float* uv,
                         float* target, cudaStream_t s);
cudaError_t nif_loss_grad(const TrainNet& net, int64_t B, const float* uv, const float* target, float delta,
                          int precision, TrainWork& wk, double* loss_d, float* loss_f, cudaStream_t s);
cudaError_t adam_step(int64_t n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                      float c1, float c2, cudaStream_t s);
// precision PT_FP32: FP32 SIMT GEMMs; PT_BF16: tcgen05 GEMMs (train_tc.cu) with BF16 operands
cudaError_t mlp_loss_grad(const TrainNet& net, int64_t B, const float* target, float delta, int mode,
                          const int32_t* mask, int precision, TrainWork& wk, double* loss_d, float* loss_f,
                          cudaStream_t s);
// self-test of the bounded device wait (selftest.cu): waits on a barrier nothing arrives on for budget_ns,
// then sets PT_ERR_TIMEOUT in *err; *d_waited_ns receives the time waited
cudaError_t wait_selftest(uint32_t* err, uint64_t budget_ns, uint64_t* d_waited_ns, cudaStream_t s);
// one 32-bit word written on the stream by a tiny kernel (values that change between graph replays)
cudaError_t launch_set_u32(uint32_t* dst, uint32_t value, cudaStream_t s);
// tensor-core GEMMs of training (train_tc.cu): forward X[0] -> X[1..L] (and BF16 tiles Xb); backward from
// G[L-1] = dX[0] -> BF16 tiles Gb and per-CTA partials of every layer's dW / db (Gl CTAs per layer, stride
// floats each, layer l's at partial + l * Gl * stride: [H][pitch[l]] dW then [H] db)
bool train_tc_supported(const TrainNet& net);
cudaError_t train_tc_forward(const TrainNet& net, int64_t B, TrainWork& wk, unsigned int* err, cudaStream_t s);
cudaError_t train_tc_backward(const TrainNet& net, int64_t B, TrainWork& wk, unsigned int* err, int* Gl, int* stride,
                              int* pitch, cudaStream_t s);

// Radiance cache (train.cu).  Rows of 16 floats: x[3], wo[3], n[3], tp[3],
// L[3] (radiance gathered before the vertex), slot (query) or valid (record).
struct CacheBox {
    float lo[3];
    float eh[3], el[3];             // hi - lo as an exact float pair eh + el
    int32_t J;                      // frequencies per axis
};
// layer-0 inputs from record rows; with slot_L (path radiance) also targets and mask
cudaError_t cache_train_inputs(int64_t n, const float* rec, const float* slot_L, CacheBox box, float* X0, float* target,
                               int32_t* mask, cudaStream_t s);
cudaError_t cache_train_pixels(uint32_t seed, uint32_t frame, int64_t n, uint32_t n_pix, int64_t* pixels, cudaStream_t s);
// fused cache MLP (cache.cu): H = 64 only.  q [n][9] -> raw outputs [n][3];
// render queries (rows [cap][16], live count on the device) -> slot radiance
size_t cache_eval_smem_bytes(int in0, int L);
cudaError_t cache_eval(const float* params, int J, int L, CacheBox box, int64_t n, const float* q, float* out,
                       int sm_count, cudaStream_t s);
cudaError_t cache_query(const float* params, int J, int L, CacheBox box, int64_t cap, const uint32_t* n_dev,
                        const float* rows, float* slot_L, int accumulate, uint32_t* err, unsigned long long* stats,
                        int sm_count, cudaStream_t s);
// BF16 tensor-core cache (cache_tc.cu): J = 12, H = 64, L = 5 only
bool cache_tc_supported(int J, int H, int L);
size_t cache_tc_image_bytes();
cudaError_t repack_cache_tc(const float* params, unsigned char* image, cudaStream_t s);
cudaError_t cache_eval_tc(const unsigned char* image, CacheBox box, int64_t n, const float* q, float* out,
                          uint32_t* err, int sm_count, cudaStream_t s);
cudaError_t cache_query_tc(const unsigned char* image, CacheBox box, int64_t cap, const uint32_t* n_dev,
                           const float* rows, float* slot_L, int accumulate, uint32_t* err, unsigned long long* stats,
                           int sm_count, cudaStream_t s);
// rebuild the packed FP32 layout and (when present) the tensor-core image from the master weights
cudaError_t repack_nif_fp32(const float* params, int F, int H, int L, int skip, float* packed, cudaStream_t s);
cudaError_t repack_nif_tc_image(const float* params, int F, int H, int L, int S, unsigned char* image, cudaStream_t s);

// read-only views of the C-ABI handles (api.cu)
const DevScene* scene_view(const pt_scene* s, int* device);
const DevNif* nif_view(const pt_nif* n);

// host BVH builder (bvh_build.cpp)

// An allocator whose value-initialisation leaves trivially constructible
// elements as they are, so the builder's arrays of tens of millions of
// records are not zeroed serially before its threads fill them.
template <class T>
struct NoInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind { using other = NoInitAlloc<U>; };
    NoInitAlloc() = default;
    template <class U>
    NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
    template <class U>
    void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) { ::new ((void*)p) U; }
    template <class U, class... A>
    void construct(U* p, A&&... a) { ::new ((void*)p) U(std::forward<A>(a)...); }
};
using NodeVec = std::vector<PackedNode, NoInitAlloc<PackedNode>>;

// f(t, lo, hi) over T contiguous chunks [b + n t / T, b + n (t + 1) / T) of [b, e), one host thread each
// (the caller runs chunk 0, and every chunk whose thread could not be started); f must not throw
template <class F>
void for_chunks(int64_t b, int64_t e, int T, F&& f)
{
    const int64_t n = e - b;
    if (T <= 1) {
        f(0, b, e);
        return;
    }
    std::vector<std::thread> th;
    int started = 1;   // chunks 1 .. started - 1 have a thread
    try {
        th.reserve((size_t)T - 1);
        for (int t = 1; t < T; ++t) {
            th.emplace_back([&f, t, b, n, T] { f(t, b + n * t / T, b + n * (t + 1) / T); });
            started = t + 1;
        }
    } catch (...) {
        // out of threads or memory: the remaining chunks run here
    }
    for (int t = started; t < T; ++t) f(t, b + n * t / T, b + n * (t + 1) / T);
    f(0, b, b + n / T);
    for (auto& x : th) x.join();
}
// host threads for a pass over n records: all hardware threads from 2^16 records up, else one
inline int host_pass_threads(int64_t n)
{
    return n >= ((int64_t)1 << 16) ? (int)std::max(1u, std::thread::hardware_concurrency()) : 1;
}
using QuantVec = std::vector<QuantNode, NoInitAlloc<QuantNode>>;

struct BuildInput {
    int64_t n_prims;
    std::vector<float> lo, hi;  // [n][3] primitive bounds (the builder splits on the box midpoints)
};
struct BuildOutput {
    NodeVec nodes;
    uint32_t root = kEmptyRef;
    int32_t depth = 0;
    std::string error;
};
// threads = 0: all hardware threads; the tree does not depend on the count
bool build_bvh(const BuildInput& in, BuildOutput& out, unsigned threads = 0);
bool round_up_half_extent(float lo, float hi, uint16_t* out_bits);
// value of a non-negative IEEE binary16 bit pattern (fp16 extents of the packed nodes)
float half_bits_to_float(uint16_t h);
// The packed tree's children boxes as decoded on the device (fp32 origin + fp16 extent, fp32 sum):
// box[0..2] lo_l, [3..5] hi_l, [6..8] lo_r, [9..11] hi_r.
void decode_packed_boxes(const PackedNode& n, float box[12]);
// Quantised form of a packed tree of n nodes (same node order and references; nodes on all hardware
// threads); false with *error set (the first failing node's reason) when a reference or primitive ID does
// not fit 24 bits or a box does not fit the grid.
bool quantize_bvh(const PackedNode* in, size_t n, QuantVec& out, std::string* error);

}  // namespace ptk
