// FP8 (E4M3) variant of the fused tensor-core NIF for F = 64, three hidden
// FC-128 ReLU layers and the FC-3 head (Section 3.2; the paper lists FP8
// weights as future work, Section 5), on sm_103a tcgen05 tensor cores with
// FP32 accumulation.
//
// Quantisation: features are scaled by 448 (|f| <= 1); hidden weights and
// the head carry one scale per output row (row max / 448); hidden
// activations carry one scale per layer, calibrated on the host from the FP32
// network over a fixed 32 x 32 grid of (u, v) pixel centres (layer max /
// 448, values beyond saturate).  Dequantisation, bias, ReLU and the next
// layer's quantisation fold into one FMA per value:
//   q_out = relu(acc * (s_in * s_w[j] / s_out) + b[j] / s_out)
// done as packed FP32x2 FMAs and a saturating ReLU conversion to E4M3.
//
// A 128-element E4M3 row is exactly one 128-byte swizzle row, so operands
// are half the size of the BF16 kernel's: four tile slots fit beside the
// weights.  One warpgroup per slot (thread t = row t = TMEM lane t), warp 16
// allocates TMEM and issues the MMAs (128x128x32, head 128x16x32); the head
// reuses the slot's accumulator columns after the last hidden epilogue has
// read them.  All waits are bounded as in the BF16 kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "tc_ptx.cuh"

namespace ptk {

namespace {

using namespace tc;

constexpr int kF = 64, kH = 128, kRows = 128;
constexpr int kSlots = 4;
constexpr int kThreads = (4 * kSlots + 1) * 32;   // 4 warps per slot + the MMA warp
constexpr int kMmaWarp = 4 * kSlots;
constexpr uint32_t kTmemCols = 512;

constexpr uint32_t kWBytes = kH * kH;              // 16 KB per hidden layer
constexpr uint32_t kHeadRows = 16;
constexpr uint32_t kOffHead = 3 * kWBytes;         // 49152
constexpr uint32_t kOffTail = kOffHead + kHeadRows * kH;  // 51200
// tail floats: mul [3][128], add [3][128], head mul [4], head add [4], B [128], M [12]
constexpr uint32_t kTailFloats = 6 * kH + 8 + 2 * kF + 12;
constexpr uint32_t kImageBytes = kOffTail + kTailFloats * 4;   // 54864
constexpr uint32_t kOffA = 55296;                  // 1024-aligned, four 16 KB operand buffers
constexpr uint32_t kABytes = kRows * kH;
constexpr uint32_t kOffBar = kOffA + kSlots * kABytes;
constexpr uint32_t kSmemBytes = kOffBar + 128 + 1024;
constexpr float kE4M3Max = 448.f;

static_assert(kImageBytes % 16 == 0, "bulk copy size");
static_assert(kOffA % 1024 == 0 && kOffHead % 1024 == 0 && kOffA >= kImageBytes, "layout");

// 16-byte chunk c (elements [16c, 16c+16)) of row r of a 128 x 128 E4M3 operand, SWIZZLE_128B K-major
__device__ __forceinline__ uint32_t chunk8(uint32_t r, uint32_t c) { return r * 128 + (((c & 7) ^ (r & 7)) << 4); }

struct In8 {
    float u, v, tr, tg, tb;
    uint32_t slot;
};

struct Fp8Params {
    const unsigned char* image;
    const float* uv;
    float* rgb;
    int64_t n;
    const EscapeRec* esc;
    const uint32_t* esc_count;
    uint32_t esc_cap;
    float* slot_L;
    int accumulate;
    uint32_t* err;
    unsigned long long* stats;
};

__global__ void __launch_bounds__(kThreads, 1) k_nif_fp8(const Fp8Params p, int mode)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar_a = sbase + kOffBar;
    const uint32_t bar_acc = bar_a + 8 * kSlots;
    const uint32_t bar_w = bar_acc + 8 * kSlots;
    const uint32_t bar_drain = bar_w + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 96);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + kOffBar + 100);
    const float* tail = reinterpret_cast<const float*>(smem + kOffTail);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t count = mode == 0 ? p.n : (int64_t)min(*p.esc_count, p.esc_cap);
    const int64_t n_tiles = (count + kRows - 1) / kRows;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(bar_a + 8 * s, kRows);
            mbar_init(bar_acc + 8 * s, 1);
        }
        mbar_init(bar_w, 1);
        mbar_init(bar_drain, 1);
        *abort = 0;
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
        if (lane == 0 && !*abort) {
            const uint32_t id_h = idesc_e4m3(128, 128), id_o = idesc_e4m3(128, kHeadRows);
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
                    const uint32_t a_base = sbase + kOffA + s * kABytes;
                    const uint32_t d = tmem + s * 128;
                    const bool head = stage[s] == 3;
                    const uint32_t b_base = head ? sbase + kOffHead : sbase + stage[s] * kWBytes;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_e4m3(d, sw128_desc(a_base + 32 * kk), sw128_desc(b_base + 32 * kk), head ? id_o : id_h, kk > 0);
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
                mma_commit(bar_drain);
                const uint64_t t0 = global_ns();
                while (!mbar_try_wait(bar_drain, 0) && global_ns() - t0 < kWaitBudgetNs) {
                }
            }
        }
    } else {
        const int s = warp >> 2;
        const uint32_t row = (warp & 3) * 32 + lane;
        const uint32_t lane_base = ((uint32_t)(warp & 3) * 32u) << 16;
        const uint32_t a_base = sbase + kOffA + s * kABytes;
        const float* Bm = tail + 6 * kH + 8;
        const float* Mm = Bm + 2 * kF;
        uint32_t ph = 0;
        auto load_inputs = [&](int64_t tile) {
            In8 t = {};
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
        In8 in = load_inputs((int64_t)blockIdx.x * kSlots + s);
        for (int64_t i = 0;; ++i) {
            const int64_t tile = ((int64_t)i * gridDim.x + blockIdx.x) * kSlots + s;
            if (tile >= n_tiles) break;
            if (__any_sync(0xFFFFFFFFu, *abort != 0)) break;
            const int64_t g = tile * kRows + row;
            const bool valid = g < count;
            // features x 448 -> E4M3: sin of frequencies 0..63 in chunks 0..3, cos in chunks 4..7
#pragma unroll 1
            for (int c16 = 0; c16 < 4; ++c16) {
                uint32_t sw[4], cw[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float sv[4], cv[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int f = c16 * 16 + 4 * j + h;
                        const float t = fmaf(Bm[2 * f], in.u, Bm[2 * f + 1] * in.v);
                        const float r = t - rintf(t);
                        __sincosf(6.28318530717958648f * r, &sv[h], &cv[h]);
                    }
                    sw[j] = pack_e4m3x2(sv[0] * kE4M3Max, sv[1] * kE4M3Max) |
                            (pack_e4m3x2(sv[2] * kE4M3Max, sv[3] * kE4M3Max) << 16);
                    cw[j] = pack_e4m3x2(cv[0] * kE4M3Max, cv[1] * kE4M3Max) |
                            (pack_e4m3x2(cv[2] * kE4M3Max, cv[3] * kE4M3Max) << 16);
                }
                st_shared_v4(a_base + chunk8(row, c16), sw[0], sw[1], sw[2], sw[3]);
                st_shared_v4(a_base + chunk8(row, 4 + c16), cw[0], cw[1], cw[2], cw[3]);
            }
            fence_proxy_async();
            mbar_arrive(bar_a + 8 * s);
            const In8 next = load_inputs(((int64_t)(i + 1) * gridDim.x + blockIdx.x) * kSlots + s);

            bool ok = true;
            for (int layer = 0; layer < 3; ++layer) {
                const bool got = mbar_wait(bar_acc + 8 * s, ph, abort, p.err);
                if (!__all_sync(0xFFFFFFFFu, got)) { ok = false; break; }
                ph ^= 1;
                tc_fence_after();
                const uint64_t* mul2 = reinterpret_cast<const uint64_t*>(tail + layer * kH);
                const uint64_t* add2 = reinterpret_cast<const uint64_t*>(tail + (3 + layer) * kH);
#pragma unroll 1
                for (int c32 = 0; c32 < 4; ++c32) {
                    uint32_t r[32];
                    TMEM_LD32(tmem + lane_base + s * 128 + c32 * 32, r);
                    tmem_wait_ld();
                    uint32_t q[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const uint64_t v0 = fma_f32x2(pack_u64(r[4 * j], r[4 * j + 1]), mul2[c32 * 16 + 2 * j],
                                                      add2[c32 * 16 + 2 * j]);
                        const uint64_t v1 = fma_f32x2(pack_u64(r[4 * j + 2], r[4 * j + 3]), mul2[c32 * 16 + 2 * j + 1],
                                                      add2[c32 * 16 + 2 * j + 1]);
                        q[j] = pack_relu_e4m3x2(__uint_as_float((uint32_t)v0), __uint_as_float((uint32_t)(v0 >> 32))) |
                               (pack_relu_e4m3x2(__uint_as_float((uint32_t)v1), __uint_as_float((uint32_t)(v1 >> 32)))
                                << 16);
                    }
                    st_shared_v4(a_base + chunk8(row, 2 * c32), q[0], q[1], q[2], q[3]);
                    st_shared_v4(a_base + chunk8(row, 2 * c32 + 1), q[4], q[5], q[6], q[7]);
                }
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
            tmem_ld4(tmem + lane_base + s * 128, yr);
            tmem_wait_ld();
            const float* hm = tail + 6 * kH;
            const float* ha = hm + 4;
            const float y0 = fmaf(__uint_as_float(yr[0]), hm[0], ha[0]);
            const float y1 = fmaf(__uint_as_float(yr[1]), hm[1], ha[1]);
            const float y2 = fmaf(__uint_as_float(yr[2]), hm[2], ha[2]);
            const float r0 = expf(Mm[0] * y0 + Mm[1] * y1 + Mm[2] * y2);
            const float r1 = expf(Mm[3] * y0 + Mm[4] * y1 + Mm[5] * y2);
            const float r2 = expf(Mm[6] * y0 + Mm[7] * y1 + Mm[8] * y2);
            if (valid) {
                if (mode == 0) {
                    p.rgb[3 * g] = r0; p.rgb[3 * g + 1] = r1; p.rgb[3 * g + 2] = r2;
                } else {
                    float* L = p.slot_L + 3 * (size_t)in.slot;
                    float a = in.tr * r0, b = in.tg * r1, c = in.tb * r2;
                    if (p.accumulate) { a += L[0]; b += L[1]; c += L[2]; }
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

uint8_t to_e4m3(float x)
{
    return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

}  // namespace

// Host packing of the FP8 image; scales_out (nullable) receives the four
// activation scales [features, h1, h2, h3] (value = scale x E4M3 code).
bool pack_nif_fp8_image(const float* params, int F, int H, int L, std::vector<unsigned char>& out, float* scales_out)
{
    if (F != kF || H != kH || L != 3) return false;
    const float* Bsrc = params;
    const float* W[4];
    const float* b[4];
    const float* p = params + 2 * F;
    for (int l = 0; l < 4; ++l) {
        const int in = l == 0 ? 2 * F : H, o = l == 3 ? 3 : H;
        W[l] = p;
        p += (size_t)in * o;
        b[l] = p;
        p += o;
    }
    const float* M = p;
    // activation scales from the FP32 network on a 32 x 32 grid of pixel centres
    float amax[3] = {0.f, 0.f, 0.f};
    std::vector<float> x(kH), y(kH);
    for (int gi = 0; gi < 32 * 32; ++gi) {
        const double u = (gi % 32 + 0.5) / 32.0, v = (gi / 32 + 0.5) / 32.0;
        for (int f = 0; f < kF; ++f) {
            const double t = (double)Bsrc[2 * f] * u + (double)Bsrc[2 * f + 1] * v;
            x[f] = (float)std::sin(6.283185307179586 * t);
            x[kF + f] = (float)std::cos(6.283185307179586 * t);
        }
        for (int l = 0; l < 3; ++l) {
            for (int j = 0; j < kH; ++j) {
                float acc = b[l][j];
                for (int k = 0; k < kH; ++k) acc += W[l][(size_t)j * kH + k] * x[k];
                y[j] = acc > 0.f ? acc : 0.f;
                amax[l] = std::max(amax[l], y[j]);
            }
            std::swap(x, y);
        }
    }
    float s_act[4] = {1.f / kE4M3Max, 0, 0, 0};
    for (int l = 0; l < 3; ++l) s_act[l + 1] = amax[l] > 0.f ? amax[l] / kE4M3Max : 1.f;
    if (scales_out)
        for (int i = 0; i < 4; ++i) scales_out[i] = s_act[i];

    out.assign(kImageBytes, 0);
    float* tail = reinterpret_cast<float*>(&out[kOffTail]);
    auto put = [&](uint32_t base, uint32_t r, uint32_t k, uint8_t q) {
        out[base + r * 128 + ((((k >> 4) & 7) ^ (r & 7)) << 4) + (k & 15)] = q;
    };
    for (int l = 0; l < 4; ++l) {
        const int rows = l == 3 ? 3 : kH;
        for (int j = 0; j < rows; ++j) {
            float wmax = 0.f;
            for (int k = 0; k < kH; ++k) wmax = std::max(wmax, std::fabs(W[l][(size_t)j * kH + k]));
            const float sw = wmax > 0.f ? wmax / kE4M3Max : 1.f;
            for (int k = 0; k < kH; ++k)
                put(l == 3 ? kOffHead : l * kWBytes, j, k, to_e4m3(W[l][(size_t)j * kH + k] / sw));
            if (l < 3) {
                tail[l * kH + j] = s_act[l] * sw / s_act[l + 1];     // folded dequant + requant
                tail[(3 + l) * kH + j] = b[l][j] / s_act[l + 1];
            } else {
                tail[6 * kH + j] = s_act[3] * sw;                    // head dequant
                tail[6 * kH + 4 + j] = b[3][j];
            }
        }
    }
    for (int i = 0; i < 2 * kF; ++i) tail[6 * kH + 8 + i] = Bsrc[i];
    for (int i = 0; i < 9; ++i) tail[6 * kH + 8 + 2 * kF + i] = M[i];
    return true;
}

cudaError_t launch_nif_fp8(const unsigned char* image, const NifEvalParams& np, int mode, int sm_count, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_nif_fp8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    Fp8Params p = {};
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
    k_nif_fp8<<<sm_count, kThreads, kSmemBytes, s>>>(p, mode); count_launch();
    return cudaGetLastError();
}

}  // namespace ptk
