// Fused tensor-core evaluation of the HDR neural image field (Section 3.2)
// for the shape F = 64 frequencies, three hidden FC-128 ReLU layers, FC-3
// head, on sm_103a tcgen05 tensor cores.
//
// The paper keeps the network's weights in IPU tile SRAM and lets the
// Poplibs planner replicate layers across tiles (Section 3.3.1); here one
// persistent CTA per SM holds all BF16 weights in shared memory for the
// whole kernel and streams 128-row tiles of queries through them:
//
//   warps 0..23  three groups of eight; group s owns tile slot s.  Within a
//                group, warps 4h..4h+3 handle half h of every row: row t is
//                TMEM lane t, and half h covers accumulator columns
//                [64h, 64h + 64) and Fourier frequencies [32h, 32h + 32).
//                They compute the features, and after each MMA read their
//                accumulator half-row from TMEM (bias included), apply ReLU
//                while packing to BF16 and write it back into the slot's
//                operand buffer in the UMMA SWIZZLE_128B K-major layout.
//   warp 24      allocates TMEM; lane 0 issues every tcgen05.mma (128x128x16
//                BF16 -> FP32 for the hidden layers plus one K = 16 step that
//                adds the bias, 128x16x16 for the head) and commits each
//                layer to the slot's mbarrier.
//
// Three slots in flight let the epilogue of one tile overlap the MMAs of
// the others.  Every wait is bounded in time: a wait that gives up sets
// PT_ERR_TIMEOUT, raises a CTA-wide abort flag, drains in-flight MMAs and
// frees TMEM before the CTA returns.
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "tc_ptx.cuh"

namespace ptk {

namespace {

constexpr int kF = 64, kH = 128, kRows = 128;
constexpr int kSlots = 3;
constexpr int kThreads = 25 * 32;        // 3 slots x 8 epilogue warps + the MMA warp
constexpr int kMmaWarp = 24;
constexpr uint32_t kTmemCols = 512;

// shared-memory image (offsets from a 1024-byte aligned base)
constexpr uint32_t kWBytes = kH * kH * 2;            // 32 KB per hidden layer (2 K-blocks x 128 rows x 128 B)
constexpr uint32_t kHeadRows = 16;
constexpr uint32_t kHeadBytes = kHeadRows * kH * 2;  // 4 KB
constexpr uint32_t kOffW = 0;                        // W1 | W2 | W3
constexpr uint32_t kOffHead = 3 * kWBytes;           // 98304
// Hidden-layer biases ride on the tensor core as one more K = 16 step: A is a
// block of ones (columns 0 and 1), B holds bias = hi + lo in BF16 (columns 0
// and 1), both K-major without swizzle (core matrices 8 rows x 16 B, K step
// 128 B, 8-row step 256 B).
constexpr uint32_t kBiasBytes = kRows * 32;              // 4096 per block
constexpr uint32_t kBiasLbo = 128, kBiasSbo = 256;
constexpr uint32_t kOffBias = kOffHead + kHeadBytes;     // 102400: b1 | b2 | b3
constexpr uint32_t kOffOnes = kOffBias + 3 * kBiasBytes; // 114688
constexpr uint32_t kOffTail = kOffOnes + kBiasBytes;     // 118784: fp32 b1 b2 b3 [384], b4 [4], B [128], M [12]
constexpr uint32_t kTailFloats = 3 * kH + 4 + 2 * kF + 12;
constexpr uint32_t kImageBytes = kOffTail + kTailFloats * 4;  // 120896
constexpr uint32_t kOffA = 121856;                   // 1024-aligned, three 32 KB activation buffers
constexpr uint32_t kABytes = kRows * kH * 2;
constexpr uint32_t kOffBar = kOffA + kSlots * kABytes;  // 203776
constexpr uint32_t kSmemBytes = kOffBar + 128 + 1024;   // barriers + alignment slack

static_assert(kImageBytes % 16 == 0, "bulk copy size");
static_assert(kImageBytes <= kOffA && kSmemBytes <= 227 * 1024, "shared-memory budget");
static_assert(kOffA % 1024 == 0 && kOffHead % 1024 == 0, "swizzle atoms need 1024-byte alignment");

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

// 25 warps: the busiest SM sub-partition holds seven of them (16K registers), so at most 72 per thread
__global__ void __maxnreg__(72) k_nif_tc(const TcParams p, int mode)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar_a = sbase + kOffBar;            // [kSlots] operand ready (count 128)
    const uint32_t bar_acc = bar_a + 8 * kSlots;        // [kSlots] accumulator ready (commit)
    const uint32_t bar_w = bar_acc + 8 * kSlots;        // weights loaded
    const uint32_t bar_drain = bar_w + 8;               // final drain after an abort
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 64);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + kOffBar + 68);
    const float* tail = reinterpret_cast<const float*>(smem + kOffTail);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t count = mode == 0 ? p.n : (int64_t)min(*p.esc_count, p.esc_cap);
    const int64_t n_tiles = (count + kRows - 1) / kRows;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(bar_a + 8 * s, 2 * kRows);   // both halves of the slot arrive
            mbar_init(bar_acc + 8 * s, 1);
        }
        mbar_init(bar_w, 1);
        mbar_init(bar_drain, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // one bulk copy per 32 KB piece of the weight image, all on bar_w
        mbar_expect_tx(bar_w, kImageBytes);
        for (uint32_t off = 0; off < kImageBytes; off += 32768u) {
            const uint32_t sz = min(32768u, kImageBytes - off);
            bulk_g2s(sbase + off, p.image + off, sz, bar_w);
        }
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    mbar_wait(bar_w, 0, abort, p.err);

    if (warp == kMmaWarp) {
        // ------------------------------------------------------------- MMA issuer
        if (lane == 0 && !*abort) {
            const uint32_t id_h = idesc_bf16(128, 128), id_o = idesc_bf16(128, kHeadRows);
            // Event loop: serve whichever slot has its operand ready, so a slow
            // epilogue in one slot never holds back the MMAs of the others.
            uint32_t ph[kSlots] = {0, 0, 0};
            int stage[kSlots] = {0, 0, 0};
            int64_t it[kSlots] = {0, 0, 0};
            int live = 0;
            bool done[kSlots];
            for (int s = 0; s < kSlots; ++s) {
                done[s] = ((int64_t)blockIdx.x * kSlots + s) >= n_tiles;
                live += done[s] ? 0 : 1;
            }
            uint64_t last = global_ns();
            while (live > 0 && !*abort) {
                bool progressed = false;
                for (int s = 0; s < kSlots; ++s) {
                    if (done[s] || !mbar_test_wait(bar_a + 8 * s, ph[s])) continue;
                    progressed = true;
                    ph[s] ^= 1;
                    tc_fence_after();
                    const uint32_t a_base = sbase + kOffA + s * kABytes;
                    if (stage[s] < 3) {
                        const uint32_t w_base = sbase + kOffW + stage[s] * kWBytes;
                        const uint32_t d = tmem + s * 128;
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const uint32_t koff = (kk >> 2) * (kRows * 128) + (kk & 3) * 32;
                            mma_bf16(d, sw128_desc(a_base + koff), sw128_desc(w_base + koff), id_h, kk > 0);
                        }
                        // + bias: ones x (hi, lo)
                        mma_bf16(d, plain_desc(sbase + kOffOnes, kBiasLbo, kBiasSbo),
                                 plain_desc(sbase + kOffBias + stage[s] * kBiasBytes, kBiasLbo, kBiasSbo), id_h, 1);
                    } else {
                        const uint32_t d = tmem + 384 + 32 * s;
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const uint32_t aoff = (kk >> 2) * (kRows * 128) + (kk & 3) * 32;
                            const uint32_t boff = (kk >> 2) * (kHeadRows * 128) + (kk & 3) * 32;
                            mma_bf16(d, sw128_desc(a_base + aoff), sw128_desc(sbase + kOffHead + boff), id_o, kk > 0);
                        }
                    }
                    mma_commit(bar_acc + 8 * s);
                    if (++stage[s] == 4) {
                        stage[s] = 0;
                        ++it[s];
                        if ((it[s] * gridDim.x + blockIdx.x) * kSlots + s >= n_tiles) {
                            done[s] = true;
                            --live;
                        }
                    }
                }
                if (progressed) {
                    last = global_ns();
                } else {
                    __nanosleep(32);   // nothing ready: yield the issue slots to the epilogue warps
                }
                if (!progressed && global_ns() - last > kWaitBudgetNs) {
                    atomicOr(p.err, PT_ERR_TIMEOUT);
                    *abort = 1;
                }
            }
            if (*abort) {
                // make sure no MMA is still writing TMEM before it is freed
                mma_commit(bar_drain);
                const uint64_t t0 = global_ns();
                while (!mbar_try_wait(bar_drain, 0) && global_ns() - t0 < kWaitBudgetNs) {
                }
            }
        }
    } else {
        // ------------------------------------------------------- epilogue warps
        const int s = warp >> 3;                       // tile slot (8 warps each)
        const int half = (warp >> 2) & 1;              // which 64 columns / 32 frequencies of the row
        const uint32_t row = (warp & 3) * 32 + lane;   // row in tile == TMEM lane
        const uint32_t lane_base = ((uint32_t)(warp & 3) * 32u) << 16;
        const uint32_t a_base = sbase + kOffA + s * kABytes;
        const float* Bm = tail + 3 * kH + 4;
        const float* Mm = Bm + 2 * kF;
        uint32_t ph = 0;
        // inputs of this thread's row of a tile, loaded one tile ahead so the
        // global-memory latency hides behind the previous tile's MMA chain
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
        TileIn in = load_inputs(((int64_t)0 * gridDim.x + blockIdx.x) * kSlots + s);
        for (int64_t i = 0;; ++i) {
            const int64_t tile = ((int64_t)i * gridDim.x + blockIdx.x) * kSlots + s;
            if (tile >= n_tiles) break;
            if (__any_sync(0xFFFFFFFFu, *abort != 0)) break;  // warp-uniform exit
            const int64_t g = tile * kRows + row;
            const bool valid = g < count;
            const float u = in.u, v = in.v, tr = in.tr, tg = in.tg, tb = in.tb;
            const uint32_t slot = in.slot;
            // Fourier features [sin 2 pi (Bx)_i, cos 2 pi (Bx)_i]: phase reduced to one turn in FP32,
            // then the hardware sine / cosine (the result is rounded to BF16)
            const uint64_t uu = pack_f32x2(u, u), vv = pack_f32x2(v, v);
            const uint64_t two_pi = pack_f32x2(6.28318530717958648f, 6.28318530717958648f);
#pragma unroll 1
            for (int c8 = half * 4; c8 < half * 4 + 4; ++c8) {
                uint32_t sp[4], cp[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // frequencies f, f + 1 in packed FP32 pairs: t = B0 u + B1 v, r = t - rint(t)
                    const int f = c8 * 8 + 2 * j;
                    const float4 bq = *reinterpret_cast<const float4*>(Bm + 2 * f);   // B0 B1 of f, f + 1
                    const uint64_t t = fma_f32x2(pack_f32x2(bq.x, bq.z), uu, mul_f32x2(pack_f32x2(bq.y, bq.w), vv));
                    const uint64_t r = sub_f32x2(t, pack_f32x2(rintf(lo_f32(t)), rintf(hi_f32(t))));
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
            fence_proxy_async();
            mbar_arrive(bar_a + 8 * s);
            const TileIn next = load_inputs(((int64_t)(i + 1) * gridDim.x + blockIdx.x) * kSlots + s);

            bool ok = true;
            for (int layer = 0; layer < 3; ++layer) {
                const bool got = mbar_wait(bar_acc + 8 * s, ph, abort, p.err);
                if (!__all_sync(0xFFFFFFFFu, got)) { ok = false; break; }  // tcgen05.ld needs the whole warp
                ph ^= 1;
                tc_fence_after();
                // this half-row's 64 accumulator columns in four groups of 16, the TMEM load of
                // group g + 1 in flight while group g is packed (the bias is already in the
                // accumulator: ReLU while rounding to BF16) and stored
                const uint32_t tcol = tmem + lane_base + s * 128 + half * 64;
                uint32_t ra[16], rb[16];
                auto put16 = [&](const uint32_t (&x)[16], int g) {
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) pk[j] = pack_relu_bf16(__uint_as_float(x[2 * j]), __uint_as_float(x[2 * j + 1]));
                    const int c8 = half * 8 + 2 * g;
                    st_shared_v4(a_base + sw128_chunk(row, c8), pk[0], pk[1], pk[2], pk[3]);
                    st_shared_v4(a_base + sw128_chunk(row, c8 + 1), pk[4], pk[5], pk[6], pk[7]);
                };
                tmem_ld16(tcol, ra);
                tmem_wait_ld();
                tmem_ld16(tcol + 16, rb);
                put16(ra, 0);
                tmem_wait_ld();
                tmem_ld16(tcol + 32, ra);
                put16(rb, 1);
                tmem_wait_ld();
                tmem_ld16(tcol + 48, rb);
                put16(ra, 2);
                tmem_wait_ld();
                put16(rb, 3);
                tc_fence_before();
                fence_proxy_async();
                mbar_arrive(bar_a + 8 * s);
            }
            if (!ok) break;
            const bool got_head = mbar_wait(bar_acc + 8 * s, ph, abort, p.err);
            if (!__all_sync(0xFFFFFFFFu, got_head)) break;
            ph ^= 1;
            tc_fence_after();
            if (half == 1) {  // the other half of the slot owns the output
                in = next;
                continue;
            }
            uint32_t yr[4];
            tmem_ld4(tmem + lane_base + 384 + 32 * s, yr);
            tmem_wait_ld();
            const float* b4 = tail + 3 * kH;
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
                    if (p.accumulate) { a += L[0]; b += L[1]; c += L[2]; }  // radiance gathered before the escape
                    if (!(isfinite(a) && isfinite(b) && isfinite(c))) atomicOr(p.err, PT_ERR_NONFINITE);
                    L[0] = a; L[1] = b; L[2] = c;
                }
            }
            tc_fence_before();
            in = next;
        }
    }
    if (mode == 1 && blockIdx.x == 0 && threadIdx.x == 0 && p.stats) atomicAdd(p.stats, (unsigned long long)count);
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

}  // namespace

// Host-side packing of the weight image for k_nif_tc (see the offsets above).
// W[l] are PyTorch-layout [out][in] float matrices.
bool pack_nif_tc_image(const float* params, int F, int H, int L, std::vector<unsigned char>& out)
{
    if (F != kF || H != kH || L != 3) return false;
    out.assign(kImageBytes, 0);
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
        put_plain(kOffOnes + bias_elem(r, 0), 1.f);
        put_plain(kOffOnes + bias_elem(r, 1), 1.f);
    }
    const float* p = params;
    const float* Bsrc = p;
    p += 2 * F;
    float* tail = reinterpret_cast<float*>(&out[kOffTail]);
    for (int l = 0; l <= L; ++l) {
        const int in = l == 0 ? 2 * F : H, o = l == L ? 3 : H;
        if (l < L) {
            for (int j = 0; j < o; ++j)
                for (int k = 0; k < in; ++k) put(kOffW + l * kWBytes, kRows, j, k, p[(size_t)j * in + k]);
            p += (size_t)in * o;
            for (int j = 0; j < o; ++j) {
                tail[l * kH + j] = p[j];
                const float hi = from_bf16(to_bf16(p[j]));
                put_plain(kOffBias + l * kBiasBytes + bias_elem(j, 0), hi);
                put_plain(kOffBias + l * kBiasBytes + bias_elem(j, 1), p[j] - hi);
            }
            p += o;
        } else {
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < in; ++k) put(kOffHead, kHeadRows, j, k, p[(size_t)j * in + k]);
            p += (size_t)in * 3;
            for (int j = 0; j < 3; ++j) tail[3 * kH + j] = p[j];
            p += 3;
        }
    }
    for (int i = 0; i < 2 * F; ++i) tail[3 * kH + 4 + i] = Bsrc[i];
    for (int i = 0; i < 9; ++i) tail[3 * kH + 4 + 2 * F + i] = p[i];
    return true;
}

cudaError_t launch_nif_tc(const unsigned char* image, const NifEvalParams& np, int mode, int sm_count, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_nif_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
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
    k_nif_tc<<<sm_count, kThreads, kSmemBytes, s>>>(p, mode);
    return cudaGetLastError();
}

size_t nif_tc_image_bytes() { return kImageBytes; }

}  // namespace ptk

namespace ptk {
namespace {
// Flat master weights -> the tensor-core kernel's shared-memory image (same
// layout as pack_nif_tc_image builds on the host; BF16 round-to-nearest-even).
__global__ void k_repack_tc(const float* __restrict__ params, unsigned char* __restrict__ image)
{
    const float* W[4];
    const float* b[4];
    const float* p = params + 2 * kF;
    for (int l = 0; l < 4; ++l) {
        const int in = l == 0 ? 2 * kF : kH, o = l == 3 ? 3 : kH;
        W[l] = p;
        p += (size_t)in * o;
        b[l] = p;
        p += o;
    }
    const float* Mp = p;
    // bias blocks (hi, lo in columns 0, 1) and the block of ones; the rest of those blocks stays zero
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 4 * kRows; idx += gridDim.x * blockDim.x) {
        const int l = idx / kRows, r = idx % kRows;
        unsigned short* hi = reinterpret_cast<unsigned short*>(image + kOffBias + l * kBiasBytes + bias_elem(r, 0));
        unsigned short* lo = reinterpret_cast<unsigned short*>(image + kOffBias + l * kBiasBytes + bias_elem(r, 1));
        if (l < 3) {
            const float x = b[l][r];
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            *hi = __bfloat16_as_ushort(h);
            *lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
        } else {   // l == 3: the ones block directly follows the bias blocks
            *hi = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
            *lo = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
        }
    }
    const int n_hidden = 3 * kH * kH, n_head = kHeadRows * kH;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_hidden + n_head + (int)kTailFloats;
         idx += gridDim.x * blockDim.x) {
        if (idx < n_hidden + n_head) {
            uint32_t base, rows, r, k;
            float x;
            if (idx < n_hidden) {
                const int l = idx / (kH * kH);
                r = (idx / kH) % kH;
                k = idx % kH;
                base = kOffW + l * kWBytes;
                rows = kRows;
                x = W[l][(size_t)r * kH + k];
            } else {
                const int q = idx - n_hidden;
                r = q / kH;
                k = q % kH;
                base = kOffHead;
                rows = kHeadRows;
                x = r < 3 ? W[3][(size_t)r * kH + k] : 0.f;
            }
            const uint32_t off = base + (k >> 6) * (rows * 128) + r * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) + (k & 7) * 2;
            const unsigned short bits = __bfloat16_as_ushort(__float2bfloat16_rn(x));
            *reinterpret_cast<unsigned short*>(image + off) = bits;
        } else {
            const int t = idx - n_hidden - n_head;
            float val = 0.f;
            if (t < 3 * kH) val = b[t / kH][t % kH];
            else if (t < 3 * kH + 4) val = (t - 3 * kH) < 3 ? b[3][t - 3 * kH] : 0.f;
            else if (t < 3 * kH + 4 + 2 * kF) val = params[t - 3 * kH - 4];
            else if (t < 3 * kH + 4 + 2 * kF + 9) val = Mp[t - 3 * kH - 4 - 2 * kF];
            reinterpret_cast<float*>(image + kOffTail)[t] = val;
        }
    }
}
}  // namespace

cudaError_t repack_nif_tc_image(const float* params, unsigned char* image, cudaStream_t s)
{
    k_repack_tc<<<128, 256, 0, s>>>(params, image);
    return cudaGetLastError();
}
}  // namespace ptk
