// Fused tensor-core evaluation of the HDR neural image field (Section 3.2)
// on sm_103a tcgen05 tensor cores, templated over the network shape: F
// frequencies (64 in the workloads, the paper's 20), hidden width H in {32,
// 64, 128, 256}, L hidden FC-H ReLU layers (three of width 128 in the
// workloads) and the FC-3 head, optionally with the paper's skip join (hidden
// layer S narrowed to H - 2F outputs and joined with the Fourier features
// before layer S + 1).  Included by the translation units that instantiate
// it (nif_tc.cu: F = 64, H = 128; nif_tc_small.cu: H = 64 and 32;
// nif_tc_shapes.cu: H = 256 and the paper's skip network).
//
// The paper keeps the network's weights in IPU tile SRAM and lets the
// Poplibs planner replicate layers across tiles (Section 3.3.1); here one
// persistent CTA per SM holds all BF16 weights in shared memory for the
// whole kernel and streams 128-row tiles of queries through them.  The
// operand tile slots (128 rows x 128 BF16, 32 KB; 64 KB for H = 256) that fit
// beside the weights and in TMEM set the overlap: for H = 128 and F = 64
// three for L <= 3, two for L = 4, one for L = 5, none from L = 6 (where SRAM
// residency breaks on this GPU); narrower networks keep up to four; H = 256
// keeps two slots at L = 1 only.  Tile slots of four warps (one warpgroup)
// each: thread t of a slot owns row t of the tile, which is TMEM lane t, with
// all accumulator columns and all Fourier frequencies of that row.  A slot's
// warps compute the features, and after each MMA read their accumulator row
// from TMEM (bias included, 32 columns per load with the next load in
// flight), apply ReLU while packing to BF16 and write it back into the
// slot's operand buffer in the UMMA SWIZZLE_128B K-major layout.  Each step
// ends with a slot-wide named barrier (bar.red.or, which also carries the
// abort vote); the slot's first thread then issues the next tcgen05.mma group
// itself (128xNx16 BF16 -> FP32 for the hidden layers plus one K = 16 step
// that adds the bias, 128x16x16 for the head) and commits it to the slot's
// mbarrier.  With several slots in flight the epilogue of one tile overlaps
// the MMAs of the others.  Every wait is bounded in time: a wait that gives
// up sets PT_ERR_TIMEOUT, raises a CTA-wide abort flag, drains in-flight MMAs
// and frees TMEM.
#pragma once

#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "tc_ptx.cuh"

namespace ptk {
namespace tcnif {

using namespace tc;

constexpr int kRows = 128;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kHeadRows = 16;
// Hidden-layer biases ride on the tensor core as one more K = 16 step: A is a
// block of ones (columns 0 and 1), B holds bias = hi + lo in BF16 (columns 0
// and 1), both K-major without swizzle (core matrices 8 rows x 16 B, K step
// 128 B, 8-row step 256 B).
constexpr uint32_t kBiasLbo = 128, kBiasSbo = 256;
constexpr int kSmemLimit = 227 * 1024;

constexpr int imin(int a, int b) { return a < b ? a : b; }

// Shared-memory image of a NIF of shape (F, H, L, S) (offsets from a
// 1024-byte aligned base): W1 .. WL | head | bias blocks b1 .. bL | ones |
// FP32 tail (b_head [4], B [2F] as frequency pairs (B[f][0], B[f+1][0],
// B[f][1], B[f+1][1]) so that one 16-byte load gives both packed FP32x2
// operands, M [12]), then the tile slots.  Weights are K-major SWIZZLE_128B
// blocks of 64 K-elements, one row per output (padded to the MMA width).  The
// features sit in the operand tile as [sin (F) | cos (F)] when F % 8 == 0 and
// nothing is joined, else interleaved, sin f and cos f in columns 2f and
// 2f + 1 (an 8-column chunk holds four frequencies, so a join may start at
// any multiple of eight columns); the weights that read them are permuted to
// match.  Each slot owns H + 32 TMEM columns
// (accumulator, head) or, for H = 256, H (the head reuses the accumulator).
template <int F, int H, int L, int S>
struct Layout {
    static_assert(F % 4 == 0 && 2 * F <= 128, "features: four frequencies per 16-byte chunk, at most 128 columns");
    static_assert(H == 32 || H == 64 || H == 128 || H == 256, "hidden width");
    static_assert(S == 0 || (S < L && H - 2 * F >= 16 && (H - 2 * F) % 8 == 0), "skip join");
    static constexpr int k0 = (2 * F + 15) / 16 * 16;                  // K of the first layer (features, padded)
    static constexpr int n_skip = S ? (H - 2 * F + 31) / 32 * 32 : H;   // MMA width of the narrowed layer
    static constexpr int aw = H > 128 ? 256 : 128;                      // operand tile width (elements)
    static constexpr uint32_t a_bytes = (uint32_t)kRows * aw * 2;
    // output rows (MMA N) and input columns (MMA K) of linear layer l (l = L: the head)
    __host__ __device__ static constexpr int n_out(int l) { return l == L ? (int)kHeadRows : (S && l == S - 1 ? n_skip : H); }
    __host__ __device__ static constexpr int k_in(int l) { return l == 0 ? k0 : H; }
    __host__ __device__ static constexpr uint32_t w_bytes(int l) { return (uint32_t)((k_in(l) + 63) / 64) * n_out(l) * 128u; }
    __host__ __device__ static constexpr uint32_t w_off(int l)
    {
        uint32_t o = 0;
        for (int q = 0; q < l; ++q) o += w_bytes(q);
        return o;
    }
    static constexpr uint32_t off_head = w_off(L);
    static constexpr uint32_t bias_bytes = H * 32;              // H rows x K = 16 BF16
    static constexpr uint32_t off_bias = off_head + w_bytes(L);
    static constexpr uint32_t off_ones = off_bias + L * bias_bytes;
    static constexpr uint32_t off_tail = off_ones + kRows * 32;
    static constexpr uint32_t tail_floats = 4 + 2 * F + 12;
    static constexpr uint32_t image_bytes = off_tail + tail_floats * 4;
    static constexpr uint32_t off_a = (image_bytes + 1023) & ~1023u;
    static constexpr bool head_in_acc = H > 128;
    static constexpr uint32_t tmem_per_slot = head_in_acc ? H : H + 32;
    static constexpr int room = (kSmemLimit - 1024 - 128 - (int)off_a) / (int)a_bytes;
    // three slots for H = 128 (480 TMEM columns, 168 registers a thread); four for narrower networks
    static constexpr int slots = imin(imin(room, (int)(kTmemCols / tmem_per_slot)), H >= 128 ? 3 : 4);
    static constexpr uint32_t off_bar = off_a + (slots > 0 ? slots : 0) * a_bytes;
    static constexpr uint32_t smem_bytes = off_bar + 128 + 1024;   // barriers + alignment slack
    static constexpr int threads = (slots > 0 ? slots : 1) * 128;
};

// Flat parameter layout (pt_nif_desc): widths of linear layer l of the shape
__host__ __device__ constexpr int flat_in(int F, int H, int l) { return l == 0 ? 2 * F : H; }
__host__ __device__ constexpr int flat_out(int F, int H, int L, int S, int l)
{
    return l == L ? 3 : (S && l == S - 1 ? H - 2 * F : H);
}
#ifndef PT_NIF_FEAT_BLOCKED
#define PT_NIF_FEAT_BLOCKED 1
#endif
// Features in the operand tile: [sin (F) | cos (F)] in blocks of eight frequencies when F % 8 == 0 and
// nothing is joined, else interleaved (sin f, cos f in columns 2f, 2f + 1; four frequencies per chunk).
__host__ __device__ constexpr bool features_blocked(int F, int S) { return PT_NIF_FEAT_BLOCKED && S == 0 && F % 8 == 0; }
// operand-tile column of feature j (j < F: sin of frequency j, else cos of frequency j - F)
__host__ __device__ constexpr int feature_col(int F, int S, int j)
{
    return features_blocked(F, S) ? j : (j < F ? 2 * j : 2 * (j - F) + 1);
}
// operand-tile column of input k of linear layer l (the features are laid out alike wherever they enter)
__host__ __device__ constexpr int input_col(int F, int H, int S, int l, int k)
{
    return l == 0 ? feature_col(F, S, k)
                  : (S && l == S && k >= H - 2 * F ? H - 2 * F + feature_col(F, S, k - (H - 2 * F)) : k);
}

// byte offset of element (row r, k < 16) of a bias / ones block
__host__ __device__ constexpr uint32_t bias_elem(uint32_t r, uint32_t k)
{
    return (r >> 3) * kBiasSbo + (k >> 3) * kBiasLbo + (r & 7) * 16 + (k & 7) * 2;
}

// byte offset of element (row r, k) of a SWIZZLE_128B K-major operand with `rows` rows
__host__ __device__ constexpr uint32_t sw128_elem(uint32_t rows, uint32_t r, uint32_t k)
{
    return (k >> 6) * (rows * 128) + r * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) + (k & 7) * 2;
}

// byte offset of the 16-byte chunk holding elements [8c, 8c+8) of row r of a
// 128-row BF16 operand tile in SWIZZLE_128B K-major form
__device__ __forceinline__ uint32_t sw128_chunk(uint32_t r, uint32_t c)
{
    return (c >> 3) * (kRows * 128) + r * 128 + (((c & 7) ^ (r & 7)) << 4);
}

struct TileIn {
    float u, v, tr, tg, tb;
    uint32_t slot;
};

struct TcParams {
    const unsigned char* image;  // packed weights (Layout::image_bytes)
    // mode 0
    const float* uv;
    float* rgb;
    int64_t n;
    // mode 1
    EscapeQueue esc;
    const uint32_t* esc_count;
    uint32_t esc_cap;
    float* slot_L;
    int accumulate;   // 1: add to the radiance the path gathered before escaping
    uint32_t* err;
    unsigned long long* stats;
};

// bar.red.or over the 128 threads of a slot: true on every thread if any passed true
__device__ __forceinline__ bool slot_vote_any(int id, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\n"
        "setp.ne.u32 p, %1, 0;\n"
        "bar.red.or.pred q, %2, 128, p;\n"
        "selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id)
        : "memory");
    return r != 0;
}

// ReLU'd BF16 of 32 accumulator columns [32 gq, 32 gq + 32) of this thread's row into the operand tile
__device__ __forceinline__ void put32(uint32_t a_base, uint32_t row, const uint32_t (&x)[32], int gq)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            pk[j] = pack_relu_bf16(__uint_as_float(x[16 * h + 2 * j]), __uint_as_float(x[16 * h + 2 * j + 1]));
        const int c8 = 4 * gq + 2 * h;
        st_shared_v4(a_base + sw128_chunk(row, c8), pk[0], pk[1], pk[2], pk[3]);
        st_shared_v4(a_base + sw128_chunk(row, c8 + 1), pk[4], pk[5], pk[6], pk[7]);
    }
}

// Epilogue of a hidden layer of N columns: TMEM -> ReLU -> BF16 -> operand
// tile, 32 columns per load with the next load in flight.
template <int N>
__device__ __forceinline__ void epilogue(uint32_t tcol, uint32_t a_base, uint32_t row)
{
    constexpr int G = N / 32;
    static_assert(N % 32 == 0, "epilogue width");
    uint32_t ra[32], rb[32];
    TMEM_LD32(tcol, ra);
    tmem_wait_ld();
#pragma unroll
    for (int g = 0; g < G; g += 2) {
        if (g + 1 < G) TMEM_LD32(tcol + 32 * (g + 1), rb);
        put32(a_base, row, ra, g);
        if (g + 1 < G) {
            tmem_wait_ld();
            if (g + 2 < G) TMEM_LD32(tcol + 32 * (g + 2), ra);
            put32(a_base, row, rb, g + 1);
            if (g + 2 < G) tmem_wait_ld();
        }
    }
}

// Features of four frequencies 4c .. 4c + 3 of (u, v) as one 16-byte chunk
// (sin, cos interleaved, BF16): phases t = B (u, v) in packed FP32x2, reduced
// to t - rint(t) by the 1.5 * 2^23 shift (exact for |t| < 2^22; beyond, n is
// still an integer and only the phase's precision, not its value modulo 1,
// degrades), then sincos of 2 pi (t - rint(t)).
__device__ __forceinline__ void feature_chunk(const float* Bm, float u, float v, int c, uint32_t (&pk)[4])
{
    const uint64_t uu = pack_f32x2(u, u), vv = pack_f32x2(v, v);
    const uint64_t two_pi = pack_f32x2(6.28318530717958648f, 6.28318530717958648f);
    const uint64_t magic = pack_f32x2(12582912.f, 12582912.f);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int f = 4 * c + 2 * j;
        const float4 bq = *reinterpret_cast<const float4*>(Bm + 2 * f);   // frequencies f, f + 1
        const uint64_t t = fma_f32x2(pack_f32x2(bq.x, bq.y), uu, mul_f32x2(pack_f32x2(bq.z, bq.w), vv));
        const uint64_t n = sub_f32x2(add_f32x2(t, magic), magic);
        const uint64_t a = mul_f32x2(sub_f32x2(t, n), two_pi);
        float s0, c0, s1, c1;
        __sincosf(lo_f32(a), &s0, &c0);
        __sincosf(hi_f32(a), &s1, &c1);
        pk[2 * j] = pack_bf16(s0, c0);
        pk[2 * j + 1] = pack_bf16(s1, c1);
    }
}

// Features of eight frequencies 8c .. 8c + 7 as two 16-byte chunks, the
// sines (sp) and the cosines (cp), BF16 (the blocked layout).
__device__ __forceinline__ void feature_chunk8(const float* Bm, float u, float v, int c, uint32_t (&sp)[4],
                                               uint32_t (&cp)[4])
{
    const uint64_t uu = pack_f32x2(u, u), vv = pack_f32x2(v, v);
    const uint64_t two_pi = pack_f32x2(6.28318530717958648f, 6.28318530717958648f);
    const uint64_t magic = pack_f32x2(12582912.f, 12582912.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int f = 8 * c + 2 * j;
        const float4 bq = *reinterpret_cast<const float4*>(Bm + 2 * f);   // frequencies f, f + 1
        const uint64_t t = fma_f32x2(pack_f32x2(bq.x, bq.y), uu, mul_f32x2(pack_f32x2(bq.z, bq.w), vv));
        const uint64_t n = sub_f32x2(add_f32x2(t, magic), magic);
        const uint64_t a = mul_f32x2(sub_f32x2(t, n), two_pi);
        float s0, c0, s1, c1;
        __sincosf(lo_f32(a), &s0, &c0);
        __sincosf(hi_f32(a), &s1, &c1);
        sp[j] = pack_bf16(s0, s1);
        cp[j] = pack_bf16(c0, c1);
    }
}

// One layer's MMA group: K / 16 steps of 128 x N x 16 over the operand tile
// and a weight block with N rows.
template <int K, int N>
__device__ __forceinline__ void mma_layer(uint32_t acc, uint32_t a_base, uint32_t w_base, uint32_t idesc)
{
#pragma unroll
    for (int kk = 0; kk < K / 16; ++kk) {
        const uint32_t aoff = (kk >> 2) * (kRows * 128) + (kk & 3) * 32;
        const uint32_t boff = (kk >> 2) * (N * 128) + (kk & 3) * 32;
        mma_bf16(acc, sw128_desc(a_base + aoff), sw128_desc(w_base + boff), idesc, kk > 0);
    }
}

template <int F, int H, int L, int S>
__global__ void __launch_bounds__(Layout<F, H, L, S>::threads, 1) k_nif_tc(const TcParams p, int mode)
{
    using LY = Layout<F, H, L, S>;
    constexpr int kSlots = LY::slots;
    constexpr uint32_t kOffHead = LY::off_head, kOffBias = LY::off_bias, kOffOnes = LY::off_ones,
                       kOffTail = LY::off_tail, kImageBytes = LY::image_bytes, kOffA = LY::off_a,
                       kOffBar = LY::off_bar;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar_acc = sbase + kOffBar;            // [kSlots] accumulator ready (commit)
    const uint32_t bar_w = bar_acc + 8 * kSlots;         // weights loaded
    const uint32_t bar_drain = bar_w + 8;                // [kSlots] final drain after an abort
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 96);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + kOffBar + 100);
    const float* tail = reinterpret_cast<const float*>(smem + kOffTail);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = warp >> 2;                       // tile slot (4 warps each)
    const uint32_t row = (warp & 3) * 32 + lane;   // row in tile == TMEM lane
    const uint32_t lane_base = ((uint32_t)(warp & 3) * 32u) << 16;
    const int64_t count = mode == 0 ? p.n : (int64_t)min(*p.esc_count, p.esc_cap);
    const int64_t n_tiles = (count + kRows - 1) / kRows;

    if (threadIdx.x == 0) {
        for (int t = 0; t < kSlots; ++t) {
            mbar_init(bar_acc + 8 * t, 1);
            mbar_init(bar_drain + 8 * t, 1);
        }
        mbar_init(bar_w, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar_w, kImageBytes);
        for (uint32_t off = 0; off < kImageBytes; off += 32768u)
            bulk_g2s(sbase + off, p.image + off, min(32768u, kImageBytes - off), bar_w);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    mbar_wait(bar_w, 0, abort, p.err);
    __syncthreads();
    bool dead = *abort != 0;   // CTA-uniform

    const bool issuer = (warp & 3) == 0 && lane == 0;
    const int bar_id = 1 + s;
    const uint32_t a_base = sbase + kOffA + s * LY::a_bytes;
    const uint32_t acc = tmem + s * LY::tmem_per_slot;
    const uint32_t head = LY::head_in_acc ? acc : acc + H;
    const uint32_t bar = bar_acc + 8 * s;
    const float* Bm = tail + 4;
    const float* Mm = Bm + 2 * F;
    constexpr uint32_t id_0 = idesc_bf16(128, LY::n_out(0)), id_h = idesc_bf16(128, H),
                       id_skip = idesc_bf16(128, LY::n_skip), id_o = idesc_bf16(128, kHeadRows);
    uint32_t ph = 0;
    auto load_inputs = [&](int64_t tile) {
        TileIn t = {};
        const int64_t gg = tile * kRows + row;
        if (tile < n_tiles && gg < count) {
            if (mode == 0) {
                const float2 q = reinterpret_cast<const float2*>(p.uv)[gg];
                t.u = q.x; t.v = q.y;
            } else {
                const float2 uv = p.esc.uv[gg];
                const float4 tp = p.esc.tp[gg];
                t.slot = __float_as_uint(tp.w); t.u = uv.x; t.v = uv.y; t.tr = tp.x; t.tg = tp.y; t.tb = tp.z;
            }
        }
        return t;
    };
    TileIn in = load_inputs((int64_t)blockIdx.x * kSlots + s);
    for (int64_t i = 0; !dead; ++i) {
        const int64_t tile = ((int64_t)i * gridDim.x + blockIdx.x) * kSlots + s;
        if (tile >= n_tiles) break;   // slot-uniform
        const int64_t g = tile * kRows + row;
        const bool valid = g < count;
        if constexpr (features_blocked(F, S)) {
#pragma unroll
            for (int c = 0; c < F / 8; ++c) {
                uint32_t sp[4], cp[4];
                feature_chunk8(Bm, in.u, in.v, c, sp, cp);
                st_shared_v4(a_base + sw128_chunk(row, c), sp[0], sp[1], sp[2], sp[3]);
                st_shared_v4(a_base + sw128_chunk(row, F / 8 + c), cp[0], cp[1], cp[2], cp[3]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < F / 4; ++c) {
                uint32_t pk[4];
                feature_chunk(Bm, in.u, in.v, c, pk);
                st_shared_v4(a_base + sw128_chunk(row, c), pk[0], pk[1], pk[2], pk[3]);
            }
        }
        // columns between the features and the first layer's padded K: zeros (the tile holds the last tile's
        // activations there, and the padded weights are zero, but an infinite activation times zero is NaN)
#pragma unroll
        for (int c = F / 4; c < LY::k0 / 8; ++c) st_shared_v4(a_base + sw128_chunk(row, c), 0u, 0u, 0u, 0u);
        const float tr = in.tr, tg = in.tg, tb = in.tb, u = in.u, v = in.v;
        const uint32_t slot = in.slot;
        in = load_inputs(((int64_t)(i + 1) * gridDim.x + blockIdx.x) * kSlots + s);
        fence_proxy_async();
        bool fail = false;
        for (int stage = 0; stage <= L; ++stage) {   // the hidden layers, then the head
            tc_fence_before();
            if (slot_vote_any(bar_id, fail)) { dead = true; break; }
            if (issuer) {
                tc_fence_after();
                if (stage < L) {
                    uint32_t w_base = sbase;   // weights of layer `stage`
                    if constexpr (S == 0) {
                        if (stage > 0) w_base += LY::w_bytes(0) + (stage - 1) * LY::w_bytes(1);
                    } else {
#pragma unroll
                        for (int q = 0; q < L; ++q)
                            if (q < stage) w_base += LY::w_bytes(q);
                    }
                    uint32_t id;
                    if (LY::k0 == H && S == 0) {   // every hidden layer is K = N = H
                        mma_layer<H, H>(acc, a_base, w_base, id_h);
                        id = id_h;
                    } else if (stage == 0) {
                        mma_layer<LY::k0, LY::n_out(0)>(acc, a_base, w_base, id_0);
                        id = id_0;
                    } else if (S > 1 && stage == S - 1) {
                        mma_layer<H, LY::n_skip>(acc, a_base, w_base, id_skip);
                        id = id_skip;
                    } else {
                        mma_layer<H, H>(acc, a_base, w_base, id_h);
                        id = id_h;
                    }
                    mma_bf16(acc, plain_desc(sbase + kOffOnes, kBiasLbo, kBiasSbo),
                             plain_desc(sbase + kOffBias + stage * LY::bias_bytes, kBiasLbo, kBiasSbo), id, 1);
                } else {
                    mma_layer<H, kHeadRows>(head, a_base, sbase + kOffHead, id_o);
                }
                mma_commit(bar);
            }
            const bool got = mbar_wait(bar, ph, abort, p.err);
            ph ^= 1;
            tc_fence_after();
            if (!__all_sync(0xFFFFFFFFu, got)) { fail = true; continue; }   // voted at the next barrier
            if (stage < L) {
                const uint32_t tcol = acc + lane_base;
                if (S && stage == S - 1) {
                    epilogue<LY::n_skip>(tcol, a_base, row);
                    // the narrowed layer's H - 2F outputs are followed by the features (Section 3.2)
#pragma unroll
                    for (int c = 0; c < F / 4; ++c) {
                        uint32_t pk[4];
                        feature_chunk(Bm, u, v, c, pk);
                        st_shared_v4(a_base + sw128_chunk(row, (H - 2 * F) / 8 + c), pk[0], pk[1], pk[2], pk[3]);
                    }
                } else {
                    epilogue<H>(tcol, a_base, row);
                }
                fence_proxy_async();
            }
        }
        if (dead) break;
        tc_fence_before();
        if (slot_vote_any(bar_id, fail)) { dead = true; break; }
        {
            tc_fence_after();
            uint32_t yr[4];
            tmem_ld4(head + lane_base, yr);
            tmem_wait_ld();
            const float* b4 = tail;
            const float y0 = __uint_as_float(yr[0]) + b4[0];
            const float y1 = __uint_as_float(yr[1]) + b4[1];
            const float y2 = __uint_as_float(yr[2]) + b4[2];
            const float r0 = expf(Mm[0] * y0 + Mm[1] * y1 + Mm[2] * y2);
            const float r1 = expf(Mm[3] * y0 + Mm[4] * y1 + Mm[5] * y2);
            const float r2 = expf(Mm[6] * y0 + Mm[7] * y1 + Mm[8] * y2);
            if (valid) {
                if (mode == 0) {
                    p.rgb[3 * g] = r0; p.rgb[3 * g + 1] = r1; p.rgb[3 * g + 2] = r2;
                } else {
                    float* Lp = p.slot_L + 3 * (size_t)slot;
                    float a = tr * r0, b = tg * r1, c = tb * r2;
                    if (p.accumulate) { a += Lp[0]; b += Lp[1]; c += Lp[2]; }
                    if (!(isfinite(a) && isfinite(b) && isfinite(c))) atomicOr(p.err, PT_ERR_NONFINITE);
                    Lp[0] = a; Lp[1] = b; Lp[2] = c;
                }
            }
        }
    }
    if (issuer && *abort) {
        // make sure no MMA of this slot is still writing TMEM before it is freed
        mma_commit(bar_drain + 8 * s);
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(bar_drain + 8 * s, 0) && global_ns() - t0 < kWaitBudgetNs) {
        }
    }
    if (mode == 1 && blockIdx.x == 0 && threadIdx.x == 0 && p.stats) atomicAdd(p.stats, (unsigned long long)count);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// the B pair layout of the tail: element i holds B[(i & ~3) | ((i & 1) << 1) | ((i >> 1) & 1)] of the flat [F][2]
__host__ __device__ constexpr int tail_b_index(int i) { return (i & ~3) | ((i & 1) << 1) | ((i >> 1) & 1); }

// Host-side packing of the weight image for k_nif_tc<F, H, L, S> (see
// Layout).  W[l] are PyTorch-layout [out][in] float matrices.
template <int F, int H, int L, int S>
void pack_image(const float* params, std::vector<unsigned char>& out)
{
    using LY = Layout<F, H, L, S>;
    out.assign(LY::image_bytes, 0);
    auto to_bf16 = [](float x) -> uint16_t {
        uint32_t u;
        std::memcpy(&u, &x, 4);
        const uint32_t rounding = 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
        return (uint16_t)((u + rounding) >> 16);
    };
    auto put = [&](uint32_t off, float x) {
        const uint16_t b = to_bf16(x);
        std::memcpy(&out[off], &b, 2);
    };
    auto from_bf16 = [](uint16_t b) -> float {
        const uint32_t u = (uint32_t)b << 16;
        float x;
        std::memcpy(&x, &u, 4);
        return x;
    };
    for (uint32_t r = 0; r < kRows; ++r) {
        put(LY::off_ones + bias_elem(r, 0), 1.f);
        put(LY::off_ones + bias_elem(r, 1), 1.f);
    }
    const float* p = params;
    const float* Bsrc = p;
    p += 2 * F;
    float* tail = reinterpret_cast<float*>(&out[LY::off_tail]);
    for (int l = 0; l <= L; ++l) {
        const int in = flat_in(F, H, l), o = flat_out(F, H, L, S, l);
        for (int j = 0; j < o; ++j)
            for (int k = 0; k < in; ++k)
                put(LY::w_off(l) + sw128_elem(LY::n_out(l), j, input_col(F, H, S, l, k)), p[(size_t)j * in + k]);
        p += (size_t)in * o;
        if (l < L) {
            for (int j = 0; j < o; ++j) {
                const float hi = from_bf16(to_bf16(p[j]));
                put(LY::off_bias + l * LY::bias_bytes + bias_elem(j, 0), hi);
                put(LY::off_bias + l * LY::bias_bytes + bias_elem(j, 1), p[j] - hi);
            }
        } else {
            for (int j = 0; j < 3; ++j) tail[j] = p[j];
        }
        p += o;
    }
    for (int i = 0; i < 2 * F; ++i) tail[4 + i] = Bsrc[tail_b_index(i)];
    for (int i = 0; i < 9; ++i) tail[4 + 2 * F + i] = p[i];
}

// Flat master weights -> the same image on the device (BF16 round-to-nearest-even).
template <int F, int H, int L, int S>
__global__ void k_repack_tc(const float* __restrict__ params, unsigned char* __restrict__ image)
{
    using LY = Layout<F, H, L, S>;
    const float* W[L + 1];
    const float* b[L + 1];
    int woff[L + 2];   // start of layer l's weights in a count of all layers' weight elements
    const float* p = params + 2 * F;
    woff[0] = 0;
    for (int l = 0; l <= L; ++l) {
        const int in = flat_in(F, H, l), o = flat_out(F, H, L, S, l);
        W[l] = p;
        p += (size_t)in * o;
        b[l] = p;
        p += o;
        woff[l + 1] = woff[l] + in * o;
    }
    const float* Mp = p;
    // bias blocks (hi, lo in columns 0, 1) and the block of ones; the rest of those blocks stays zero
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L * H + kRows; idx += gridDim.x * blockDim.x) {
        const bool bias = idx < L * H;
        const int l = bias ? idx / H : 0, r = bias ? idx % H : idx - L * H;
        if (bias && r >= flat_out(F, H, L, S, l)) continue;
        const uint32_t base = bias ? LY::off_bias + l * LY::bias_bytes : LY::off_ones;
        unsigned short* hi = reinterpret_cast<unsigned short*>(image + base + bias_elem(r, 0));
        unsigned short* lo = reinterpret_cast<unsigned short*>(image + base + bias_elem(r, 1));
        if (bias) {
            const float x = b[l][r];
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            *hi = __bfloat16_as_ushort(h);
            *lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
        } else {
            *hi = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
            *lo = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
        }
    }
    // every weight element (padding rows and columns stay zero), then the FP32 tail
    const int n_w = woff[L + 1];
    const int n_total = n_w + (int)LY::tail_floats;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_total; idx += gridDim.x * blockDim.x) {
        if (idx < n_w) {
            int l = 0;
            while (idx >= woff[l + 1]) ++l;
            const int in = flat_in(F, H, l), q = idx - woff[l], j = q / in, k = q % in;
            const uint32_t off = LY::w_off(l) + sw128_elem(LY::n_out(l), j, input_col(F, H, S, l, k));
            *reinterpret_cast<unsigned short*>(image + off) = __bfloat16_as_ushort(__float2bfloat16_rn(W[l][q]));
        } else {
            const int t = idx - n_w;
            float val = 0.f;
            if (t < 4) val = t < 3 ? b[L][t] : 0.f;
            else if (t < 4 + 2 * F) val = params[tail_b_index(t - 4)];
            else if (t < 4 + 2 * F + 9) val = Mp[t - 4 - 2 * F];
            reinterpret_cast<float*>(image + LY::off_tail)[t] = val;
        }
    }
}

template <int F, int H, int L, int S>
cudaError_t launch_shape(const TcParams& p, int mode, int sm_count, cudaStream_t s)
{
    using LY = Layout<F, H, L, S>;
    cudaError_t e = cudaFuncSetAttribute(k_nif_tc<F, H, L, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)LY::smem_bytes);
    if (e != cudaSuccess) return e;
    k_nif_tc<F, H, L, S><<<sm_count, LY::threads, LY::smem_bytes, s>>>(p, mode); count_launch();
    return cudaGetLastError();
}

template <int F, int H, int L, int S>
cudaError_t repack_shape(const float* params, unsigned char* image, cudaStream_t s)
{
    k_repack_tc<F, H, L, S><<<128, 256, 0, s>>>(params, image); count_launch();
    return cudaGetLastError();
}

// Per-width entry points of the F = 64 networks without a skip join (one
// translation unit per width group): L in 1 .. max_layers(H)
template <int H>
struct NifTcWidth {
    static bool pack(const float* params, int L, std::vector<unsigned char>& out);
    static cudaError_t launch(int L, const TcParams& p, int mode, int sm_count, cudaStream_t s);
    static cudaError_t repack(const float* params, int L, unsigned char* image, cudaStream_t s);
};

// explicit specialisations, defined by the translation unit of each width
#define PT_NIF_TC_DECLARE(HH)                                                                                   \
    template <>                                                                                                \
    bool NifTcWidth<HH>::pack(const float* params, int L, std::vector<unsigned char>& out);                    \
    template <>                                                                                                \
    cudaError_t NifTcWidth<HH>::launch(int L, const TcParams& p, int mode, int sm_count, cudaStream_t s);      \
    template <>                                                                                                \
    cudaError_t NifTcWidth<HH>::repack(const float* params, int L, unsigned char* image, cudaStream_t s);
PT_NIF_TC_DECLARE(32)
PT_NIF_TC_DECLARE(64)
PT_NIF_TC_DECLARE(128)
PT_NIF_TC_DECLARE(256)
#undef PT_NIF_TC_DECLARE

// The paper's network (F = 20, H = 128, four layers, joined after the second), nif_tc_shapes.cu
constexpr int kPaperF = 20, kPaperH = 128, kPaperL = 4, kPaperS = 2;
bool pack_paper_skip(const float* params, std::vector<unsigned char>& out);
cudaError_t launch_paper_skip(const TcParams& p, int mode, int sm_count, cudaStream_t s);
cudaError_t repack_paper_skip(const float* params, unsigned char* image, cudaStream_t s);

// the deepest L with at least one slot resident, capped at the library's eight hidden layers
template <int H, int L = 1>
constexpr int max_layers()
{
    if constexpr (L > 8) return 8;
    else if constexpr (Layout<64, H, L, 0>::slots < 1) return L - 1;
    else return max_layers<H, L + 1>();
}

// dispatch over L = 1 .. max_layers<H>() for one width (F = 64, no skip join)
#define PT_NIF_TC_WIDTH(HH)                                                                                      \
    template <int L>                                                                                           \
    static bool pack_l##HH(const float* params, int l, std::vector<unsigned char>& out)                        \
    {                                                                                                          \
        if constexpr (L <= max_layers<HH>()) {                                                                 \
            if (l == L) { pack_image<64, HH, L, 0>(params, out); return true; }                               \
            return pack_l##HH<L + 1>(params, l, out);                                                          \
        } else {                                                                                               \
            return false;                                                                                      \
        }                                                                                                      \
    }                                                                                                          \
    template <int L>                                                                                           \
    static cudaError_t launch_l##HH(int l, const TcParams& p, int mode, int sm_count, cudaStream_t s)          \
    {                                                                                                          \
        if constexpr (L <= max_layers<HH>()) {                                                                 \
            if (l == L) return launch_shape<64, HH, L, 0>(p, mode, sm_count, s);                               \
            return launch_l##HH<L + 1>(l, p, mode, sm_count, s);                                               \
        } else {                                                                                               \
            return cudaErrorInvalidValue;                                                                      \
        }                                                                                                      \
    }                                                                                                          \
    template <int L>                                                                                           \
    static cudaError_t repack_l##HH(const float* params, int l, unsigned char* image, cudaStream_t s)          \
    {                                                                                                          \
        if constexpr (L <= max_layers<HH>()) {                                                                 \
            if (l == L) return repack_shape<64, HH, L, 0>(params, image, s);                                   \
            return repack_l##HH<L + 1>(params, l, image, s);                                                   \
        } else {                                                                                               \
            return cudaErrorInvalidValue;                                                                      \
        }                                                                                                      \
    }                                                                                                          \
    template <>                                                                                                \
    bool NifTcWidth<HH>::pack(const float* params, int L, std::vector<unsigned char>& out)                     \
    {                                                                                                          \
        return pack_l##HH<1>(params, L, out);                                                                  \
    }                                                                                                          \
    template <>                                                                                                \
    cudaError_t NifTcWidth<HH>::launch(int L, const TcParams& p, int mode, int sm_count, cudaStream_t s)       \
    {                                                                                                          \
        return launch_l##HH<1>(L, p, mode, sm_count, s);                                                       \
    }                                                                                                          \
    template <>                                                                                                \
    cudaError_t NifTcWidth<HH>::repack(const float* params, int L, unsigned char* image, cudaStream_t s)       \
    {                                                                                                          \
        return repack_l##HH<1>(params, L, image, s);                                                           \
    }

}  // namespace tcnif
}  // namespace ptk
