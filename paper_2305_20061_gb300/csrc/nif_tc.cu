// Fused tensor-core evaluation of the HDR neural image field (Section 3.2)
// for F = 64 frequencies, L = 1 .. 5 hidden FC-128 ReLU layers (three in the
// workloads), FC-3 head, on sm_103a tcgen05 tensor cores.
//
// The paper keeps the network's weights in IPU tile SRAM and lets the
// Poplibs planner replicate layers across tiles (Section 3.3.1); here one
// persistent CTA per SM holds all BF16 weights in shared memory for the
// whole kernel and streams 128-row tiles of queries through them.  The
// 32 KB tile slots that fit beside the weights set the overlap: three for
// L <= 3, two for L = 4, one for L = 5; from L = 6 the weights and one tile
// no longer fit in the 227 KB of shared memory (where SRAM residency breaks
// on this GPU).  Tile slots of four warps (one warpgroup) each: thread t of
// a slot owns row t of the tile, which is TMEM lane t, with all 128
// accumulator columns and all 64 Fourier frequencies of that row.  A slot's
// warps compute the features, and after each MMA read their accumulator row
// from TMEM (bias included, 32 columns per load with the next load in
// flight), apply ReLU while packing to BF16 and write it back into the
// slot's operand buffer in the UMMA SWIZZLE_128B K-major layout.  Each step
// ends with a slot-wide named barrier (bar.red.or, which also carries the
// abort vote); the slot's first thread then issues the next tcgen05.mma
// group itself (128x128x16 BF16 -> FP32 for the hidden layers plus one
// K = 16 step that adds the bias, 128x16x16 for the head) and
// commits it to the slot's mbarrier.  With three slots in flight the
// epilogue of one tile overlaps the MMAs of the others.  Every wait is
// bounded in time: a wait that gives up sets PT_ERR_TIMEOUT, raises a
// CTA-wide abort flag, drains in-flight MMAs and frees TMEM.
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "tc_ptx.cuh"

namespace ptk {

namespace {

constexpr int kF = 64, kH = 128, kRows = 128;
constexpr int kMinL = 1, kMaxL = 5;
constexpr uint32_t kTmemCols = 512;

constexpr uint32_t kWBytes = kH * kH * 2;            // 32 KB per hidden layer (2 K-blocks x 128 rows x 128 B)
constexpr uint32_t kHeadRows = 16;
constexpr uint32_t kHeadBytes = kHeadRows * kH * 2;  // 4 KB
// Hidden-layer biases ride on the tensor core as one more K = 16 step: A is a
// block of ones (columns 0 and 1), B holds bias = hi + lo in BF16 (columns 0
// and 1), both K-major without swizzle (core matrices 8 rows x 16 B, K step
// 128 B, 8-row step 256 B).
constexpr uint32_t kBiasBytes = kRows * 32;              // 4096 per block
constexpr uint32_t kBiasLbo = 128, kBiasSbo = 256;
constexpr uint32_t kABytes = kRows * kH * 2;             // one 128-row BF16 activation tile
constexpr int kSmemLimit = 227 * 1024;

// Shared-memory image of a NIF with L hidden layers (offsets from a
// 1024-byte aligned base): W1 .. WL | head | bias blocks b1 .. bL | ones |
// FP32 tail (b1 .. bL [L x 128], b_head [4], B [128], M [12]), then the tile
// slots that fit (at most three: TMEM holds 3 x (128 + 32) columns).  The
// tail holds B in pairs of frequencies (B[f][0], B[f+1][0], B[f][1],
// B[f+1][1]) so that one 16-byte load gives both packed FP32x2 operands.
template <int L>
struct Layout {
    static constexpr uint32_t off_w = 0;
    static constexpr uint32_t off_head = L * kWBytes;
    static constexpr uint32_t off_bias = off_head + kHeadBytes;
    static constexpr uint32_t off_ones = off_bias + L * kBiasBytes;
    static constexpr uint32_t off_tail = off_ones + kBiasBytes;
    static constexpr uint32_t tail_floats = L * kH + 4 + 2 * kF + 12;
    static constexpr uint32_t image_bytes = off_tail + tail_floats * 4;
    static constexpr uint32_t off_a = (image_bytes + 1023) & ~1023u;
    static constexpr int room = (kSmemLimit - 1024 - 128 - (int)off_a) / (int)kABytes;
    static constexpr int slots = room > 3 ? 3 : room;
    static constexpr uint32_t off_bar = off_a + (slots > 0 ? slots : 0) * kABytes;
    static constexpr uint32_t smem_bytes = off_bar + 128 + 1024;   // barriers + alignment slack
    static constexpr int threads = (slots > 0 ? slots : 1) * 128;
};
static_assert(Layout<3>::off_a == 121856 && Layout<3>::slots == 3, "the three-layer image");
static_assert(Layout<kMaxL>::slots >= 1 && Layout<kMaxL + 1>::slots < 1, "residency limit");

// --- PTX wrappers: tc_ptx.cuh ------------------------------------------------
using namespace tc;

// byte offset of element (row r, k < 16) of a bias / ones block
__host__ __device__ constexpr uint32_t bias_elem(uint32_t r, uint32_t k)
{
    return (r >> 3) * kBiasSbo + (k >> 3) * kBiasLbo + (r & 7) * 16 + (k & 7) * 2;
}

// byte offset of the 16-byte chunk holding elements [8c, 8c+8) of row r of a
// 128-row, 128-column BF16 operand in SWIZZLE_128B K-major form
__device__ __forceinline__ uint32_t sw128_chunk(uint32_t r, uint32_t c)
{
    return (c >> 3) * (kRows * 128) + r * 128 + (((c & 7) ^ (r & 7)) << 4);
}


struct TileIn {
    float u, v, tr, tg, tb;
    uint32_t slot;
};

struct TcParams {
    const unsigned char* image;  // packed weights (kImageBytes)
    // mode 0
    const float* uv;
    float* rgb;
    int64_t n;
    // mode 1
    const EscapeRec* esc;
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

// three slots = 12 warps: three per SM sub-partition, up to 168 registers per thread
template <int L>
__global__ void __launch_bounds__(Layout<L>::threads, 1) k_nif_tc(const TcParams p, int mode)
{
    using LY = Layout<L>;
    constexpr int kSlots = LY::slots;
    constexpr uint32_t kOffW = LY::off_w, kOffHead = LY::off_head, kOffBias = LY::off_bias, kOffOnes = LY::off_ones,
                       kOffTail = LY::off_tail, kImageBytes = LY::image_bytes, kOffA = LY::off_a,
                       kOffBar = LY::off_bar;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar_acc = sbase + kOffBar;            // [kSlots] accumulator ready (commit)
    const uint32_t bar_w = bar_acc + 8 * kSlots;         // weights loaded
    const uint32_t bar_drain = bar_w + 8;                // [kSlots] final drain after an abort
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 64);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + kOffBar + 68);
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
    const uint32_t a_base = sbase + kOffA + s * kABytes;
    const uint32_t acc = tmem + s * 128;
    const uint32_t head = tmem + 384 + 32 * s;
    const uint32_t bar = bar_acc + 8 * s;
    const float* Bm = tail + L * kH + 4;
    const float* Mm = Bm + 2 * kF;
    const uint32_t id_h = idesc_bf16(128, 128), id_o = idesc_bf16(128, kHeadRows);
    uint32_t ph = 0;
    auto load_inputs = [&](int64_t tile) {
        TileIn t = {};
        const int64_t gg = tile * kRows + row;
        if (tile < n_tiles && gg < count) {
            if (mode == 0) {
                const float2 q = reinterpret_cast<const float2*>(p.uv)[gg];
                t.u = q.x; t.v = q.y;
            } else {
                const float2* e = reinterpret_cast<const float2*>(p.esc + gg);
                const float2 a = e[0], b = e[1], c = e[2];
                t.slot = __float_as_uint(a.x); t.u = a.y; t.v = b.x; t.tr = b.y; t.tg = c.x; t.tb = c.y;
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
        {
            const uint64_t uu = pack_f32x2(in.u, in.u), vv = pack_f32x2(in.v, in.v);
            const uint64_t two_pi = pack_f32x2(6.28318530717958648f, 6.28318530717958648f);
            const uint64_t magic = pack_f32x2(12582912.f, 12582912.f);
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) {
                uint32_t sp[4], cp[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int f = c8 * 8 + 2 * j;
                    const float4 bq = *reinterpret_cast<const float4*>(Bm + 2 * f);   // frequencies f, f + 1
                    const uint64_t t = fma_f32x2(pack_f32x2(bq.x, bq.y), uu, mul_f32x2(pack_f32x2(bq.z, bq.w), vv));
                    // t - rint(t) by the 1.5 * 2^23 shift: exact for |t| < 2^22; beyond, n is still an integer
                    // and only the phase's precision (not its value modulo 1) degrades
                    const uint64_t n = sub_f32x2(add_f32x2(t, magic), magic);
                    const uint64_t r = sub_f32x2(t, n);
                    const uint64_t a = mul_f32x2(r, two_pi);
                    float sv[2], cv[2];
                    __sincosf(lo_f32(a), &sv[0], &cv[0]);
                    __sincosf(hi_f32(a), &sv[1], &cv[1]);
                    sp[j] = pack_bf16(sv[0], sv[1]);
                    cp[j] = pack_bf16(cv[0], cv[1]);
                }
                st_shared_v4(a_base + sw128_chunk(row, c8), sp[0], sp[1], sp[2], sp[3]);
                st_shared_v4(a_base + sw128_chunk(row, kF / 8 + c8), cp[0], cp[1], cp[2], cp[3]);
            }
        }
        const float tr = in.tr, tg = in.tg, tb = in.tb;
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
                    const uint32_t w_base = sbase + kOffW + stage * kWBytes;
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint32_t koff = (kk >> 2) * (kRows * 128) + (kk & 3) * 32;
                        mma_bf16(acc, sw128_desc(a_base + koff), sw128_desc(w_base + koff), id_h, kk > 0);
                    }
                    mma_bf16(acc, plain_desc(sbase + kOffOnes, kBiasLbo, kBiasSbo),
                             plain_desc(sbase + kOffBias + stage * kBiasBytes, kBiasLbo, kBiasSbo), id_h, 1);
                } else {
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint32_t aoff = (kk >> 2) * (kRows * 128) + (kk & 3) * 32;
                        const uint32_t boff = (kk >> 2) * (kHeadRows * 128) + (kk & 3) * 32;
                        mma_bf16(head, sw128_desc(a_base + aoff), sw128_desc(sbase + kOffHead + boff), id_o, kk > 0);
                    }
                }
                mma_commit(bar);
            }
            const bool got = mbar_wait(bar, ph, abort, p.err);
            ph ^= 1;
            tc_fence_after();
            if (!__all_sync(0xFFFFFFFFu, got)) { fail = true; continue; }   // voted at the next barrier
            if (stage < L) {
                const uint32_t tcol = acc + lane_base;
                uint32_t ra[32], rb[32];
                auto put32 = [&](const uint32_t (&x)[32], int gq) {
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
                };
                TMEM_LD32(tcol, ra);
                tmem_wait_ld();
                TMEM_LD32(tcol + 32, rb);
                put32(ra, 0);
                tmem_wait_ld();
                TMEM_LD32(tcol + 64, ra);
                put32(rb, 1);
                tmem_wait_ld();
                TMEM_LD32(tcol + 96, rb);
                put32(ra, 2);
                tmem_wait_ld();
                put32(rb, 3);
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
            const float* b4 = tail + L * kH;
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
                    float* L = p.slot_L + 3 * (size_t)slot;
                    float a = tr * r0, b = tg * r1, c = tb * r2;
                    if (p.accumulate) { a += L[0]; b += L[1]; c += L[2]; }
                    if (!(isfinite(a) && isfinite(b) && isfinite(c))) atomicOr(p.err, PT_ERR_NONFINITE);
                    L[0] = a; L[1] = b; L[2] = c;
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

// Host-side packing of the weight image for k_nif_tc<L> (see Layout).
// W[l] are PyTorch-layout [out][in] float matrices.
template <int L>
void pack_image(const float* params, int F, int H, std::vector<unsigned char>& out)
{
    using LY = Layout<L>;
    out.assign(LY::image_bytes, 0);
    auto to_bf16 = [](float x) -> uint16_t {
        uint32_t u;
        std::memcpy(&u, &x, 4);
        const uint32_t rounding = 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
        return (uint16_t)((u + rounding) >> 16);
    };
    auto put = [&](uint32_t base, uint32_t rows_total, uint32_t r, uint32_t k, float x) {
        const uint32_t off = base + (k >> 6) * (rows_total * 128) + r * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) +
                             (k & 7) * 2;
        const uint16_t b = to_bf16(x);
        std::memcpy(&out[off], &b, 2);
    };
    auto put_plain = [&](uint32_t off, float x) {
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
        put_plain(LY::off_ones + bias_elem(r, 0), 1.f);
        put_plain(LY::off_ones + bias_elem(r, 1), 1.f);
    }
    const float* p = params;
    const float* Bsrc = p;
    p += 2 * F;
    float* tail = reinterpret_cast<float*>(&out[LY::off_tail]);
    for (int l = 0; l <= L; ++l) {
        const int in = l == 0 ? 2 * F : H, o = l == L ? 3 : H;
        if (l < L) {
            for (int j = 0; j < o; ++j)
                for (int k = 0; k < in; ++k) put(LY::off_w + l * kWBytes, kRows, j, k, p[(size_t)j * in + k]);
            p += (size_t)in * o;
            for (int j = 0; j < o; ++j) {
                tail[l * kH + j] = p[j];
                const float hi = from_bf16(to_bf16(p[j]));
                put_plain(LY::off_bias + l * kBiasBytes + bias_elem(j, 0), hi);
                put_plain(LY::off_bias + l * kBiasBytes + bias_elem(j, 1), p[j] - hi);
            }
            p += o;
        } else {
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < in; ++k) put(LY::off_head, kHeadRows, j, k, p[(size_t)j * in + k]);
            p += (size_t)in * 3;
            for (int j = 0; j < 3; ++j) tail[L * kH + j] = p[j];
            p += 3;
        }
    }
    for (int i = 0; i < 2 * F; ++i) tail[L * kH + 4 + i] = Bsrc[(i & ~3) | ((i & 1) << 1) | ((i >> 1) & 1)];
    for (int i = 0; i < 9; ++i) tail[L * kH + 4 + 2 * F + i] = p[i];
}

template <int L>
cudaError_t launch_l(const unsigned char* image, const TcParams& p, int mode, int sm_count, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_nif_tc<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Layout<L>::smem_bytes);
    if (e != cudaSuccess) return e;
    k_nif_tc<L><<<sm_count, Layout<L>::threads, Layout<L>::smem_bytes, s>>>(p, mode); count_launch();
    return cudaGetLastError();
}

}  // namespace

bool nif_tc_supported(int F, int H, int L) { return F == kF && H == kH && L >= kMinL && L <= kMaxL; }

bool pack_nif_tc_image(const float* params, int F, int H, int L, std::vector<unsigned char>& out)
{
    if (!nif_tc_supported(F, H, L)) return false;
    switch (L) {
    case 1: pack_image<1>(params, F, H, out); break;
    case 2: pack_image<2>(params, F, H, out); break;
    case 3: pack_image<3>(params, F, H, out); break;
    case 4: pack_image<4>(params, F, H, out); break;
    default: pack_image<5>(params, F, H, out); break;
    }
    return true;
}

cudaError_t launch_nif_tc(const unsigned char* image, int L, const NifEvalParams& np, int mode, int sm_count,
                          cudaStream_t s)
{
    TcParams p = {};
    p.image = image;
    p.uv = np.uv;
    p.rgb = np.rgb;
    p.n = np.n;
    p.esc = np.esc;
    p.esc_count = np.esc_count;
    p.esc_cap = np.esc_cap;
    p.slot_L = np.slot_L;
    p.accumulate = np.accumulate;
    p.err = np.err;
    p.stats = np.stats;
    switch (L) {
    case 1: return launch_l<1>(image, p, mode, sm_count, s);
    case 2: return launch_l<2>(image, p, mode, sm_count, s);
    case 3: return launch_l<3>(image, p, mode, sm_count, s);
    case 4: return launch_l<4>(image, p, mode, sm_count, s);
    case 5: return launch_l<5>(image, p, mode, sm_count, s);
    default: return cudaErrorInvalidValue;
    }
}



}  // namespace ptk

namespace ptk {
namespace {
// Flat master weights -> the tensor-core kernel's shared-memory image (same
// layout as pack_nif_tc_image builds on the host; BF16 round-to-nearest-even).
template <int L>
__global__ void k_repack_tc(const float* __restrict__ params, unsigned char* __restrict__ image)
{
    using LY = Layout<L>;
    const float* W[L + 1];
    const float* b[L + 1];
    const float* p = params + 2 * kF;
    for (int l = 0; l <= L; ++l) {
        const int in = l == 0 ? 2 * kF : kH, o = l == L ? 3 : kH;
        W[l] = p;
        p += (size_t)in * o;
        b[l] = p;
        p += o;
    }
    const float* Mp = p;
    // bias blocks (hi, lo in columns 0, 1) and the block of ones; the rest of those blocks stays zero
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < (L + 1) * kRows; idx += gridDim.x * blockDim.x) {
        const int l = idx / kRows, r = idx % kRows;
        unsigned short* hi = reinterpret_cast<unsigned short*>(image + LY::off_bias + l * kBiasBytes + bias_elem(r, 0));
        unsigned short* lo = reinterpret_cast<unsigned short*>(image + LY::off_bias + l * kBiasBytes + bias_elem(r, 1));
        if (l < L) {
            const float x = b[l][r];
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            *hi = __bfloat16_as_ushort(h);
            *lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
        } else {   // l == L: the ones block directly follows the bias blocks
            *hi = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
            *lo = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
        }
    }
    const int n_hidden = L * kH * kH, n_head = kHeadRows * kH;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_hidden + n_head + (int)LY::tail_floats;
         idx += gridDim.x * blockDim.x) {
        if (idx < n_hidden + n_head) {
            uint32_t base, rows, r, k;
            float x;
            if (idx < n_hidden) {
                const int l = idx / (kH * kH);
                r = (idx / kH) % kH;
                k = idx % kH;
                base = LY::off_w + l * kWBytes;
                rows = kRows;
                x = W[l][(size_t)r * kH + k];
            } else {
                const int q = idx - n_hidden;
                r = q / kH;
                k = q % kH;
                base = LY::off_head;
                rows = kHeadRows;
                x = r < 3 ? W[L][(size_t)r * kH + k] : 0.f;
            }
            const uint32_t off = base + (k >> 6) * (rows * 128) + r * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) + (k & 7) * 2;
            const unsigned short bits = __bfloat16_as_ushort(__float2bfloat16_rn(x));
            *reinterpret_cast<unsigned short*>(image + off) = bits;
        } else {
            const int t = idx - n_hidden - n_head;
            float val = 0.f;
            if (t < L * kH) val = b[t / kH][t % kH];
            else if (t < L * kH + 4) val = (t - L * kH) < 3 ? b[L][t - L * kH] : 0.f;
            else if (t < L * kH + 4 + 2 * kF) {
                const int i = t - L * kH - 4;
                val = params[(i & ~3) | ((i & 1) << 1) | ((i >> 1) & 1)];
            }
            else if (t < L * kH + 4 + 2 * kF + 9) val = Mp[t - L * kH - 4 - 2 * kF];
            reinterpret_cast<float*>(image + LY::off_tail)[t] = val;
        }
    }
}
}  // namespace

cudaError_t repack_nif_tc_image(const float* params, int L, unsigned char* image, cudaStream_t s)
{
    switch (L) {
    case 1: k_repack_tc<1><<<128, 256, 0, s>>>(params, image); break;
    case 2: k_repack_tc<2><<<128, 256, 0, s>>>(params, image); break;
    case 3: k_repack_tc<3><<<128, 256, 0, s>>>(params, image); break;
    case 4: k_repack_tc<4><<<128, 256, 0, s>>>(params, image); break;
    case 5: k_repack_tc<5><<<128, 256, 0, s>>>(params, image); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}
}  // namespace ptk
