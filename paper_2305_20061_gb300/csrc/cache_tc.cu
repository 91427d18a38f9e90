// Radiance-cache queries on tcgen05 tensor cores (BF16 operands, FP32
// accumulation) for the production shape: 12 frequencies per axis (78
// inputs), five hidden FC-64 ReLU layers, FC-3 (Mueller et al. 2021, which
// Section 2.1 cites).
//
// One persistent CTA per SM keeps the BF16 weights in shared memory and
// streams 128-row tiles through four tile slots:
//
//   warps 0..15  four per slot; warp w owns TMEM lanes / tile rows
//                32 (w % 4) .. + 31 of slot w / 4.  Each thread encodes its
//                row (sin/cos of 2^j pi p per axis, direction, normal) into
//                the slot's operand buffer, and after every MMA reads its
//                row's 64 accumulator columns (bias included), applies ReLU
//                while packing to BF16 and writes them back as the next
//                layer's operand (UMMA SWIZZLE_128B, K-major).
//   warp 16      allocates TMEM (4 x 64 columns); lane 0 issues the MMAs of
//                every slot (layer 0: K = 80 in five K = 16 steps, layers
//                1-4: K = 64; each plus one K = 16 step multiplying a block
//                of ones with the layer's bias as BF16 hi + lo; the head:
//                N = 16 into the slot's first accumulator columns).
//
// Every wait is bounded (2 s, abort flag, drain, TMEM freed).
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "tc_ptx.cuh"

namespace ptk {

namespace {

using namespace tc;

constexpr int kJ = 12, kIn = 6 * kJ + 6, kH = 64, kL = 5, kRows = 128;
constexpr int kSlots = 4;
constexpr int kThreads = (kSlots * 4 + 1) * 32;   // 544
constexpr int kMmaWarp = kSlots * 4;
constexpr uint32_t kTmemCols = kSlots * kH;     // 256
constexpr int kK0Steps = (kIn + 15) / 16;       // 5

// shared-memory image (offsets from a 1024-byte aligned base)
constexpr uint32_t kOffW0 = 0;                          // [64 rows][K 128]: 2 K-blocks x 8 KB
constexpr uint32_t kOffW = kOffW0 + 2 * kH * 128;        // 16384: layers 1-4, [64][64] = 8 KB each
constexpr uint32_t kOffHead = kOffW + (kL - 1) * kH * 128;   // 49152: [16 rows][64] = 2 KB
constexpr uint32_t kHeadRows = 16;
constexpr uint32_t kBiasLbo = 128, kBiasSbo = 256;       // no-swizzle K = 16 blocks
constexpr uint32_t kBiasBytes = kH * 32;                 // 2 KB per layer (64 rows)
constexpr uint32_t kOffBias = kOffHead + kHeadRows * 128;    // 51200: 5 bias blocks
constexpr uint32_t kOffOnes = kOffBias + kL * kBiasBytes;    // 61440: [128 rows][16] ones block, 4 KB
constexpr uint32_t kOffTail = kOffOnes + kRows * 32;     // 65536: fp32 head bias [4]
constexpr uint32_t kImageBytes = kOffTail + 16;          // 65552
constexpr uint32_t kOffA = 66560;                        // 1024-aligned, four 32 KB operand buffers
constexpr uint32_t kABytes = kRows * 128 * 2;            // 2 K-blocks of [128 rows][64]
constexpr uint32_t kOffBar = kOffA + kSlots * kABytes;   // 197632
constexpr uint32_t kSmemBytes = kOffBar + 128 + 1024;

static_assert(kImageBytes % 16 == 0 && kImageBytes <= kOffA, "image layout");
static_assert(kOffA % 1024 == 0 && kOffW % 1024 == 0 && kOffHead % 1024 == 0, "swizzle atoms");
static_assert(kSmemBytes <= 227 * 1024, "shared-memory budget");

// byte offset of element (row r, k) of an R-row BF16 operand, SWIZZLE_128B K-major
__host__ __device__ constexpr uint32_t sw128_elem(uint32_t R, uint32_t r, uint32_t k)
{
    return (k >> 6) * (R * 128) + r * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) + (k & 7) * 2;
}
// 16-byte chunk c (elements 8c .. 8c + 7) of row r of a 128-row operand
__device__ __forceinline__ uint32_t sw128_chunk(uint32_t r, uint32_t c)
{
    return (c >> 3) * (kRows * 128) + r * 128 + (((c & 7) ^ (r & 7)) << 4);
}
// element (row r, k < 16) of a no-swizzle K = 16 block
__host__ __device__ constexpr uint32_t bias_elem(uint32_t r, uint32_t k)
{
    return (r >> 3) * kBiasSbo + (k >> 3) * kBiasLbo + (r & 7) * 16 + (k & 7) * 2;
}

struct CacheTcParams {
    const unsigned char* image;
    CacheBox box;
    const float* rows;       // [cap][stride]
    int stride;              // 9: plain evaluation (raw outputs), 16: render queries
    int64_t cap;
    const uint32_t* n_dev;   // nullable
    float* out;              // stride 9: [n][3]
    float* slot_L;           // stride 16
    int accumulate;
    uint32_t* err;
    unsigned long long* stats;
};

// sin / cos(2^j pi p) for j < 12 of one position coordinate, packed as BF16
// pairs in encoding order (sin 0..11 then cos 0..11): 12 words
__device__ __forceinline__ void axis_words(float q, float lo, float eh, float el, uint32_t (&w)[12])
{
    // p = (q - lo) / (hi - lo) as a float pair ph + pl (TwoSum, one division correction step)
    const float d = q - lo;
    const float bv = d - q;
    const float e = (q - (d - bv)) + (-lo - bv);
    const float ph = __fdiv_rn(d, eh);
    const float pl = __fdiv_rn(fmaf(-ph, eh, d) + e - ph * el, eh);
    float sc = 1.f;
#pragma unroll
    for (int j = 0; j < kJ; j += 2) {   // two frequencies at a time, packed straight away
        float sv[2], cv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float x = ph * sc;
            const float xr = x - 2.f * rintf(0.5f * x);    // whole turns removed exactly: xr in [-1, 1]
            __sincosf(3.14159265358979324f * (xr + pl * sc), &sv[h], &cv[h]);
            sc *= 2.f;
        }
        w[j / 2] = pack_bf16(sv[0], sv[1]);
        w[kJ / 2 + j / 2] = pack_bf16(cv[0], cv[1]);
    }
}

// 17 warps: the busiest SM sub-partition holds five of them, so at most 96 registers per thread
__global__ void __launch_bounds__(kThreads, 1) k_cache_tc(const CacheTcParams p)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar_a = sbase + kOffBar;             // [kSlots] operand ready (count 128)
    const uint32_t bar_acc = bar_a + 8 * kSlots;         // [kSlots] accumulator ready (commit)
    const uint32_t bar_w = bar_acc + 8 * kSlots;         // weights loaded
    const uint32_t bar_drain = bar_w + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 80);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + kOffBar + 84);
    const float* tail = reinterpret_cast<const float*>(smem + kOffTail);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t count = p.n_dev ? min((int64_t)*p.n_dev, p.cap) : p.cap;
    const int64_t n_tiles = (count + kRows - 1) / kRows;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(bar_a + 8 * s, kRows);
            mbar_init(bar_acc + 8 * s, 1);
        }
        mbar_init(bar_w, 1);
        mbar_init(bar_drain, 1);
        *abort = 0;
        if (p.stats && blockIdx.x == 0) atomicAdd(p.stats, (unsigned long long)count);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar_w, kImageBytes);
        for (uint32_t off = 0; off < kImageBytes; off += 32768u)
            bulk_g2s(sbase + off, p.image + off, min(32768u, kImageBytes - off), bar_w);
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
            const uint32_t id_h = idesc_bf16(128, kH), id_o = idesc_bf16(128, kHeadRows);
            const uint64_t ones = plain_desc(sbase + kOffOnes, kBiasLbo, kBiasSbo);
            uint32_t ph[kSlots] = {0, 0, 0, 0};
            int stage[kSlots] = {0, 0, 0, 0};
            int64_t it[kSlots] = {0, 0, 0, 0};
            bool done[kSlots];
            int live = 0;
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
                    const uint32_t a = sbase + kOffA + s * kABytes;
                    const uint32_t d = tmem + s * kH;
                    const int st = stage[s];
                    if (st == 0) {          // layer 0: K = 80 (K-block 0, then the first 16 of K-block 1)
#pragma unroll
                        for (int kk = 0; kk < kK0Steps; ++kk) {
                            const uint32_t ka = (kk >> 2) * (kRows * 128) + (kk & 3) * 32;
                            const uint32_t kb = (kk >> 2) * (kH * 128) + (kk & 3) * 32;
                            mma_bf16(d, sw128_desc(a + ka), sw128_desc(sbase + kOffW0 + kb), id_h, kk > 0);
                        }
                        mma_bf16(d, ones, plain_desc(sbase + kOffBias, kBiasLbo, kBiasSbo), id_h, 1);
                    } else if (st < kL) {   // layers 1-4: K = 64
                        const uint32_t w = sbase + kOffW + (st - 1) * (kH * 128);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_bf16(d, sw128_desc(a + kk * 32), sw128_desc(w + kk * 32), id_h, kk > 0);
                        mma_bf16(d, ones, plain_desc(sbase + kOffBias + st * kBiasBytes, kBiasLbo, kBiasSbo), id_h, 1);
                    } else {                // head: N = 16 into the slot's first columns
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_bf16(d, sw128_desc(a + kk * 32), sw128_desc(sbase + kOffHead + kk * 32), id_o, kk > 0);
                    }
                    mma_commit(bar_acc + 8 * s);
                    if (++stage[s] == kL + 1) {
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
                    __nanosleep(32);
                }
                if (!progressed && global_ns() - last > kWaitBudgetNs) {
                    atomicOr(p.err, PT_ERR_TIMEOUT);
                    *abort = 1;
                }
            }
            if (*abort) {
                mma_commit(bar_drain);
                const uint64_t t0 = global_ns();
                while (!mbar_try_wait(bar_drain, 0) && global_ns() - t0 < kWaitBudgetNs) {
                }
            }
        }
    } else {
        // ------------------------------------------------------- epilogue warps
        const int s = warp >> 2;
        const uint32_t row = (warp & 3) * 32 + lane;
        const uint32_t lane_base = ((uint32_t)(warp & 3) * 32u) << 16;
        const uint32_t a_base = sbase + kOffA + s * kABytes;
        const uint32_t tcol = tmem + lane_base + s * kH;
        uint32_t ph = 0;
        for (int64_t i = 0;; ++i) {
            const int64_t tile = ((int64_t)i * gridDim.x + blockIdx.x) * kSlots + s;
            if (tile >= n_tiles) break;
            if (__any_sync(0xFFFFFFFFu, *abort != 0)) break;
            const int64_t g = tile * kRows + row;
            const bool valid = g < count;
            // ---- encoding of this row (zeros past the end)
            {
                float q[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (valid) {
                    const float* r = p.rows + g * p.stride;
#pragma unroll
                    for (int t = 0; t < 9; ++t) q[t] = r[t];
                }
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    uint32_t w[12];
                    if (valid) {
                        axis_words(q[ax], p.box.lo[ax], p.box.eh[ax], p.box.el[ax], w);
                    } else {
#pragma unroll
                        for (int t = 0; t < 12; ++t) w[t] = 0u;
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        st_shared_v4(a_base + sw128_chunk(row, 3 * ax + c), w[4 * c], w[4 * c + 1], w[4 * c + 2],
                                     w[4 * c + 3]);
                }
                st_shared_v4(a_base + sw128_chunk(row, 9), pack_bf16(q[3], q[4]), pack_bf16(q[5], q[6]),
                             pack_bf16(q[7], q[8]), 0u);
            }
            fence_proxy_async();
            mbar_arrive(bar_a + 8 * s);
            bool ok = true;
            for (int layer = 0; layer < kL; ++layer) {
                const bool got = mbar_wait(bar_acc + 8 * s, ph, abort, p.err);
                if (!__all_sync(0xFFFFFFFFu, got)) { ok = false; break; }
                ph ^= 1;
                tc_fence_after();
                uint32_t ra[16], rb[16];
                auto put16 = [&](const uint32_t (&x)[16], int gq) {
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        pk[j] = pack_relu_bf16(__uint_as_float(x[2 * j]), __uint_as_float(x[2 * j + 1]));
                    st_shared_v4(a_base + sw128_chunk(row, 2 * gq), pk[0], pk[1], pk[2], pk[3]);
                    st_shared_v4(a_base + sw128_chunk(row, 2 * gq + 1), pk[4], pk[5], pk[6], pk[7]);
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
            uint32_t yr[4];
            tmem_ld4(tcol, yr);
            tmem_wait_ld();
            tc_fence_before();
            if (valid) {
                const float y0 = __uint_as_float(yr[0]) + tail[0];
                const float y1 = __uint_as_float(yr[1]) + tail[1];
                const float y2 = __uint_as_float(yr[2]) + tail[2];
                if (p.stride == 16) {
                    const float4 tq = *reinterpret_cast<const float4*>(p.rows + g * 16 + 8);   // n.z tp.xyz
                    const float4 lq = *reinterpret_cast<const float4*>(p.rows + g * 16 + 12);  // L.xyz slot
                    float a = tq.y * fmaxf(y0, 0.f), b = tq.z * fmaxf(y1, 0.f), c = tq.w * fmaxf(y2, 0.f);
                    if (p.accumulate) { a += lq.x; b += lq.y; c += lq.z; }
                    if (!(isfinite(a) && isfinite(b) && isfinite(c))) atomicOr(p.err, PT_ERR_NONFINITE);
                    float* L = p.slot_L + 3 * (size_t)__float_as_uint(lq.w);
                    L[0] = a; L[1] = b; L[2] = c;
                } else {
                    p.out[3 * g] = y0;
                    p.out[3 * g + 1] = y1;
                    p.out[3 * g + 2] = y2;
                }
            }
        }
    }
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Flat FP32 master weights (W0 [64][78], b0, W1..W4 [64][64], b1..b4, W5 [3][64], b5) -> the image.
__global__ void k_repack_cache_tc(const float* __restrict__ params, unsigned char* __restrict__ image)
{
    const float* W[kL + 1];
    const float* b[kL + 1];
    const float* q = params;
    for (int l = 0; l <= kL; ++l) {
        const int in = l == 0 ? kIn : kH, o = l == kL ? 3 : kH;
        W[l] = q;
        q += in * o;
        b[l] = q;
        q += o;
    }
    const int n0 = kH * 128, nh = (kL - 1) * kH * kH, nhead = kHeadRows * kH, nb = kL * kH, nones = kRows;
    const int total = n0 + nh + nhead + nb + nones + 4;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        if (idx < n0) {                                   // layer 0, K padded to 128 with zeros
            const int r = idx / 128, k = idx % 128;
            const float x = k < kIn ? W[0][r * kIn + k] : 0.f;
            *reinterpret_cast<unsigned short*>(image + kOffW0 + sw128_elem(kH, r, k)) =
                __bfloat16_as_ushort(__float2bfloat16_rn(x));
        } else if (idx < n0 + nh) {                       // layers 1-4
            const int t = idx - n0, l = 1 + t / (kH * kH), r = (t / kH) % kH, k = t % kH;
            *reinterpret_cast<unsigned short*>(image + kOffW + (l - 1) * (kH * 128) + sw128_elem(kH, r, k)) =
                __bfloat16_as_ushort(__float2bfloat16_rn(W[l][r * kH + k]));
        } else if (idx < n0 + nh + nhead) {               // head rows 0-2, zero rows 3-15
            const int t = idx - n0 - nh, r = t / kH, k = t % kH;
            const float x = r < 3 ? W[kL][r * kH + k] : 0.f;
            *reinterpret_cast<unsigned short*>(image + kOffHead + sw128_elem(kHeadRows, r, k)) =
                __bfloat16_as_ushort(__float2bfloat16_rn(x));
        } else if (idx < n0 + nh + nhead + nb) {          // bias blocks: (hi, lo) in K columns 0, 1
            const int t = idx - n0 - nh - nhead, l = t / kH, r = t % kH;
            const float x = b[l][r];
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            unsigned char* blk = image + kOffBias + l * kBiasBytes;
            *reinterpret_cast<unsigned short*>(blk + bias_elem(r, 0)) = __bfloat16_as_ushort(h);
            *reinterpret_cast<unsigned short*>(blk + bias_elem(r, 1)) =
                __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
        } else if (idx < n0 + nh + nhead + nb + nones) {  // ones block
            const int r = idx - n0 - nh - nhead - nb;
            const unsigned short one = __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
            *reinterpret_cast<unsigned short*>(image + kOffOnes + bias_elem(r, 0)) = one;
            *reinterpret_cast<unsigned short*>(image + kOffOnes + bias_elem(r, 1)) = one;
        } else {                                          // head bias (FP32)
            const int t = idx - (n0 + nh + nhead + nb + nones);
            reinterpret_cast<float*>(image + kOffTail)[t] = t < 3 ? b[kL][t] : 0.f;
        }
    }
}

cudaError_t launch(const CacheTcParams& p, int sm_count, cudaStream_t s)
{
    if (p.cap <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_cache_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    k_cache_tc<<<sm_count, kThreads, kSmemBytes, s>>>(p); count_launch();
    return cudaGetLastError();
}

}  // namespace

bool cache_tc_supported(int J, int H, int L) { return J == kJ && H == kH && L == kL; }
size_t cache_tc_image_bytes() { return kImageBytes; }

// Rebuild the BF16 image from the master weights.  The image must start zeroed
// (the zero padding of the blocks is never rewritten).
cudaError_t repack_cache_tc(const float* params, unsigned char* image, cudaStream_t s)
{
    k_repack_cache_tc<<<64, 256, 0, s>>>(params, image); count_launch();
    return cudaGetLastError();
}

cudaError_t cache_eval_tc(const unsigned char* image, CacheBox box, int64_t n, const float* q, float* out,
                          uint32_t* err, int sm_count, cudaStream_t s)
{
    CacheTcParams p = {};
    p.image = image; p.box = box; p.rows = q; p.stride = 9; p.cap = n; p.out = out; p.err = err;
    return launch(p, sm_count, s);
}

cudaError_t cache_query_tc(const unsigned char* image, CacheBox box, int64_t cap, const uint32_t* n_dev,
                           const float* rows, float* slot_L, int accumulate, uint32_t* err, unsigned long long* stats,
                           int sm_count, cudaStream_t s)
{
    CacheTcParams p = {};
    p.image = image; p.box = box; p.rows = rows; p.stride = 16; p.cap = cap; p.n_dev = n_dev;
    p.slot_L = slot_L; p.accumulate = accumulate; p.err = err; p.stats = stats;
    return launch(p, sm_count, s);
}

}  // namespace ptk
