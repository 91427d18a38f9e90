// Tensor-core GEMMs of MLP training: the HDR NIF (Section 3.2.1) and the
// online radiance cache (Section 3.3).  BF16 operands, FP32 accumulation in
// TMEM (tcgen05), FP32 activations and gradients in HBM ([sample][128] rows),
// FP32 master weights.
//
//   forward   X[l+1] = relu(X[l] W_l^T + b_l), l = 0 .. L-1.  A CTA holds
//             every hidden layer's weights in shared memory and takes each
//             128-row tile through all layers: the ReLU output of one layer,
//             rounded to BF16, is the A operand of the next.
//   backward  G[l-1] = (G[l] W_l) * [X[l] > 0], l = L-1 .. 1, chained the
//             same way from the output layer's gradient G[L-1].
//   weights   dW_l = G[l]^T X[l] and db_l = the column sums of G[l].  The
//             batch is the reduction, so both operands are staged transposed
//             (operand rows = features, K = samples), and a row of ones
//             appended to X[l]^T yields db_l in the same MMA.  A CTA
//             accumulates its share of the batch for one layer in TMEM and
//             writes one partial; partials are summed in a fixed order, so
//             the gradient is deterministic.
//
// Operands use the K-major SWIZZLE_NONE layout (8-row x 16-byte core
// matrices) with strides chosen so that the staging stores are free of
// shared-memory bank conflicts.  Every mbarrier wait is bounded; a CTA that
// gives up sets PT_ERR_TIMEOUT, waits (bounded) for its MMAs and frees TMEM.
#include <cstdint>

#include <cuda_runtime.h>

#include "tc_ptx.cuh"

namespace ptk {

namespace {

using namespace tc;

constexpr int kRows = 128;                   // samples per tile (M of the row GEMMs, K of the weight GEMM)
constexpr int kThreads = 256;                // two warps per TMEM lane quarter
constexpr int kMaxLayers = 8;
constexpr uint32_t kActLbo = 16 * 128 + 16;  // activation tile: byte step between 8-column core blocks
constexpr uint32_t kTSbo = 144;              // transposed tile: byte step between 8-feature groups
constexpr uint32_t kTLboA = 16 * kTSbo;      // G^T tile (128 features): byte step between 8-sample blocks
constexpr int kSmemPerSm = 233472;           // 228 KiB of shared memory per SM
constexpr int kSmemReserved = 1024;          // reserved per CTA

__host__ __device__ constexpr int pad16(int n) { return (n + 15) & ~15; }

struct FwdParams {
    int64_t B;
    int L, in0, K0, H;
    const float* X0;
    float* X[kMaxLayers + 1];        // X[1 .. L] written
    const float* W[kMaxLayers];
    const float* b[kMaxLayers];
    unsigned int* err;
};

struct DxParams {
    int64_t B;
    int L, H;
    const float* Gtop;               // G[L-1]
    const float* X[kMaxLayers];      // X[1 .. L-1]: the ReLU masks
    float* G[kMaxLayers];            // G[0 .. L-2] written
    const float* W[kMaxLayers];      // W[1 .. L-1]
    unsigned int* err;
};

struct DwParams {
    int64_t B;
    int L, H, in0, Gl, stride;       // Gl CTAs per layer, stride floats per partial
    const float* G[kMaxLayers];
    const float* X[kMaxLayers];
    float* partial;                  // [L * Gl][stride]: [H][pad16(in)] dW, then [H] db
    unsigned int* err;
};

struct Bars {
    uint32_t bar, drain;
    uint32_t* tmem_slot;
    volatile int* abort;
};

__device__ __forceinline__ Bars bars_at(unsigned char* smem, uint32_t off)
{
    Bars b;
    b.bar = smem_u32(smem + off);
    b.drain = b.bar + 8;
    b.tmem_slot = reinterpret_cast<uint32_t*>(smem + off + 16);
    b.abort = reinterpret_cast<volatile int*>(smem + off + 20);
    return b;
}

// barrier init (thread 0) and TMEM allocation (warp 0); the caller then stages
// its constant operands and calls tc_begin_finish
__device__ __forceinline__ void tc_begin(const Bars& b, uint32_t cols)
{
    if (threadIdx.x == 0) {
        mbar_init(b.bar, 1);
        mbar_init(b.drain, 1);
        *b.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(b.tmem_slot)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
}
__device__ __forceinline__ uint32_t tc_begin_finish(const Bars& b)
{
    fence_proxy_async();   // generic-proxy operand stores -> visible to the MMA
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *b.tmem_slot;
}
// after the last MMA wait: on failure wait (bounded) for MMAs in flight, then free TMEM
__device__ __forceinline__ void tc_end(const Bars& b, uint32_t tmem, uint32_t cols, bool ok)
{
    if (!ok && threadIdx.x == 0) {
        mma_commit(b.drain);
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(b.drain, 0) && global_ns() - t0 < kWaitBudgetNs) {
        }
    }
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
    }
}

// the whole CTA waits for the MMA commit; true when every thread saw it
__device__ __forceinline__ bool wait_all(const Bars& b, uint32_t ph, unsigned int* err)
{
    const bool got = mbar_wait(b.bar, ph, b.abort, err);
    const bool ok = __syncthreads_and(got) != 0;
    if (ok) tc_fence_after();
    return ok;
}

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// columns >= width are zeroed
__device__ __forceinline__ float4 mask4(float4 v, int c, int width)
{
    if (c + 3 >= width) {
        v.x = c < width ? v.x : 0.f;
        v.y = c + 1 < width ? v.y : 0.f;
        v.z = c + 2 < width ? v.z : 0.f;
        v.w = 0.f;
    }
    return v;
}

// Rows [tile*128, +128) x columns [0, K) of a [B][128] FP32 matrix -> BF16
// activation tile: byte (r>>3)*128 + (c>>3)*kActLbo + (r&7)*16 + (c&7)*2.
// Columns >= width and rows >= B are zeros.  Warp w takes rows 16w .. 16w+15,
// lane l columns 4l .. 4l+3 (one coalesced row per load).
__device__ __forceinline__ void stage_rows(uint32_t a, const float* __restrict__ X, int64_t tile, int64_t B, int width,
                                           int K)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = 4 * lane;
    if (c >= K) return;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float4 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t g = tile * kRows + warp * 16 + h * 8 + i;
            v[i] = (g < B && c < width) ? mask4(ld4(X + g * 128 + c), c, width) : z;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t r = warp * 16 + h * 8 + i;
            const uint32_t addr = a + (r >> 3) * 128 + (c >> 3) * kActLbo + (r & 7) * 16 + (c & 7) * 2;
            asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(pack_bf16(v[i].x, v[i].y)),
                         "r"(pack_bf16(v[i].z, v[i].w))
                         : "memory");
        }
    }
}

// Rows [tile*128, +128) x columns [0, Kc) of a [B][128] FP32 matrix,
// transposed into a K-major operand whose rows are the columns c and whose K
// is the sample: byte (c>>3)*kTSbo + (r>>3)*lbo + (c&7)*16 + (r&7)*2.  Warp w
// takes the 8-sample blocks w and w + 8; lane l loads columns 4l .. 4l+3 of
// the block's 8 rows and stores each column's 8 samples as one 16-byte row.
__device__ __forceinline__ void stage_cols(uint32_t t, uint32_t lbo, const float* __restrict__ X, int64_t tile,
                                           int64_t B, int width, int Kc)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = 4 * lane;
    if (c >= Kc) return;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int rb = warp + 8 * h;
        float4 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t g = tile * kRows + rb * 8 + i;
            v[i] = (g < B && c < width) ? mask4(ld4(X + g * 128 + c), c, width) : z;
        }
        const uint32_t base = t + (c >> 3) * kTSbo + rb * lbo + (c & 7) * 16;
        st_shared_v4(base, pack_bf16(v[0].x, v[1].x), pack_bf16(v[2].x, v[3].x), pack_bf16(v[4].x, v[5].x),
                     pack_bf16(v[6].x, v[7].x));
        st_shared_v4(base + 16, pack_bf16(v[0].y, v[1].y), pack_bf16(v[2].y, v[3].y), pack_bf16(v[4].y, v[5].y),
                     pack_bf16(v[6].y, v[7].y));
        st_shared_v4(base + 32, pack_bf16(v[0].z, v[1].z), pack_bf16(v[2].z, v[3].z), pack_bf16(v[4].z, v[5].z),
                     pack_bf16(v[6].z, v[7].z));
        st_shared_v4(base + 48, pack_bf16(v[0].w, v[1].w), pack_bf16(v[2].w, v[3].w), pack_bf16(v[4].w, v[5].w),
                     pack_bf16(v[6].w, v[7].w));
    }
}

// K-major B operand [N rows n][K columns k] from a row-major FP32 matrix:
// value(n, k) = src[n * ld_n + k * ld_k] for n < rows_valid and k < cols_valid,
// else 0.  Byte (n>>3)*128 + (k>>3)*(N*16) + (n&7)*16 + (k&7)*2.
__device__ __forceinline__ void stage_weights(uint32_t w, int N, int K, const float* __restrict__ src, int ld_n,
                                              int ld_k, int rows_valid, int cols_valid)
{
    for (int idx = threadIdx.x; idx < N * (K / 8); idx += kThreads) {
        const int n = idx % N, kb = idx / N;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = 8 * kb + e;
            v[e] = (n < rows_valid && k < cols_valid) ? __ldg(&src[(size_t)n * ld_n + (size_t)k * ld_k]) : 0.f;
        }
        st_shared_v4(w + (n >> 3) * 128 + kb * (N * 16) + (n & 7) * 16, pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]),
                     pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    }
}

__device__ __forceinline__ void store16(float* dst, const float (&v)[16])
{
    float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
// 16 columns c0 .. c0+15 of activation-tile row `row` (two core blocks)
__device__ __forceinline__ void put_act16(uint32_t a_row, int c0, const float (&v)[16])
{
    const uint32_t p = a_row + (uint32_t)(c0 >> 3) * kActLbo;
    st_shared_v4(p, pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    st_shared_v4(p + kActLbo, pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                 pack_bf16(v[14], v[15]));
}

// ---------------------------------------------------------------------------
// forward through the hidden layers
template <int NH>
__host__ __device__ constexpr uint32_t fwd_bar_offset(int L, int K0)
{
    const uint32_t wbytes = (uint32_t)NH * K0 * 2 + (uint32_t)(L - 1) * NH * NH * 2;
    const uint32_t a = (wbytes + (uint32_t)L * NH * 4 + 127) & ~127u;
    return a + (uint32_t)((K0 > NH ? K0 : NH) / 8) * kActLbo;
}

template <int NH>
__global__ void __launch_bounds__(kThreads, NH <= 64 ? 2 : 1) k_tc_fwd(const FwdParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t sbase = smem_u32(smem);
    const int L = p.L, K0 = p.K0;
    const uint32_t w0_bytes = (uint32_t)NH * K0 * 2, wl_bytes = (uint32_t)NH * NH * 2;
    const uint32_t off_bias = w0_bytes + (uint32_t)(L - 1) * wl_bytes;
    float* bias = reinterpret_cast<float*>(smem + off_bias);
    const uint32_t a = sbase + ((off_bias + (uint32_t)L * NH * 4 + 127) & ~127u);
    const Bars bs = bars_at(smem, fwd_bar_offset<NH>(L, K0));
    constexpr uint32_t kCols = NH < 32 ? 32 : NH;

    tc_begin(bs, kCols);
    stage_weights(sbase, NH, K0, p.W[0], p.in0, 1, p.H, p.in0);
    for (int l = 1; l < L; ++l) stage_weights(sbase + w0_bytes + (l - 1) * wl_bytes, NH, NH, p.W[l], p.H, 1, p.H, p.H);
    for (int i = threadIdx.x; i < L * NH; i += kThreads) {
        const int l = i / NH, c = i % NH;
        bias[i] = c < p.H ? __ldg(&p.b[l][c]) : 0.f;
    }
    const uint32_t tmem = tc_begin_finish(bs);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, grp = warp >> 2;
    const uint32_t row = q * 32 + lane;
    const uint32_t tl = tmem + ((q * 32u) << 16);
    const uint32_t a_row = a + (row >> 3) * 128 + (row & 7) * 16;
    const uint32_t idesc = idesc_bf16(128, NH);
    const int64_t n_tiles = (p.B + kRows - 1) / kRows;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        stage_rows(a, p.X0, tile, p.B, p.in0, K0);
        fence_proxy_async();
        __syncthreads();
        const int64_t g = tile * kRows + row;
        for (int l = 0; l < L; ++l) {
            if (threadIdx.x == 0 && !*bs.abort) {
                tc_fence_after();
                const int K = l == 0 ? K0 : NH;
                const uint32_t w = sbase + (l == 0 ? 0u : w0_bytes + (uint32_t)(l - 1) * wl_bytes);
                for (int ks = 0; ks < K / 16; ++ks)
                    mma_bf16(tmem, plain_desc(a + ks * 2 * kActLbo, kActLbo, 128),
                             plain_desc(w + ks * 2 * (NH * 16), NH * 16, 128), idesc, ks > 0);
                mma_commit(bs.bar);
            }
            ok = wait_all(bs, ph, p.err);
            if (!ok) break;
            ph ^= 1;
            float* dst = p.X[l + 1] + g * 128;
#pragma unroll
            for (int cc = grp; cc < NH / 16; cc += 2) {
                uint32_t r[16];
                tmem_ld16(tl + cc * 16, r);
                tmem_wait_ld();
                float v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int c = cc * 16 + e;
                    v[e] = c < p.H ? fmaxf(__uint_as_float(r[e]) + bias[l * NH + c], 0.f) : 0.f;
                }
                if (g < p.B) store16(dst + cc * 16, v);
                if (l + 1 < L) put_act16(a_row, cc * 16, v);
            }
            tc_fence_before();
            fence_proxy_async();
            __syncthreads();
        }
    }
    tc_end(bs, tmem, kCols, ok);
}

// ---------------------------------------------------------------------------
// backward through the hidden layers (input gradients)
template <int NH>
__host__ __device__ constexpr uint32_t dx_bar_offset(int L)
{
    return (uint32_t)(L - 1) * NH * NH * 2 + (uint32_t)(NH / 8) * kActLbo;
}

template <int NH>
__global__ void __launch_bounds__(kThreads, NH <= 64 ? 2 : 1) k_tc_dx(const DxParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t sbase = smem_u32(smem);
    const int L = p.L;
    const uint32_t wl_bytes = (uint32_t)NH * NH * 2;
    const uint32_t a = sbase + (uint32_t)(L - 1) * wl_bytes;   // a multiple of 128
    const Bars bs = bars_at(smem, dx_bar_offset<NH>(L));
    constexpr uint32_t kCols = NH < 32 ? 32 : NH;

    tc_begin(bs, kCols);
    // image l-1 = W_l^T as a K-major B operand: row n = input feature k, K = output feature j
    for (int l = 1; l < L; ++l) stage_weights(sbase + (l - 1) * wl_bytes, NH, NH, p.W[l], 1, p.H, p.H, p.H);
    const uint32_t tmem = tc_begin_finish(bs);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, grp = warp >> 2;
    const uint32_t row = q * 32 + lane;
    const uint32_t tl = tmem + ((q * 32u) << 16);
    const uint32_t a_row = a + (row >> 3) * 128 + (row & 7) * 16;
    const uint32_t idesc = idesc_bf16(128, NH);
    constexpr int kMine = (NH / 16 + 1) / 2;   // column chunks per thread
    const int64_t n_tiles = (p.B + kRows - 1) / kRows;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        stage_rows(a, p.Gtop, tile, p.B, p.H, NH);
        fence_proxy_async();
        __syncthreads();
        const int64_t g = tile * kRows + row;
        for (int l = L - 1; l >= 1; --l) {
            if (threadIdx.x == 0 && !*bs.abort) {
                tc_fence_after();
                const uint32_t w = sbase + (uint32_t)(l - 1) * wl_bytes;
                for (int ks = 0; ks < NH / 16; ++ks)
                    mma_bf16(tmem, plain_desc(a + ks * 2 * kActLbo, kActLbo, 128),
                             plain_desc(w + ks * 2 * (NH * 16), NH * 16, 128), idesc, ks > 0);
                mma_commit(bs.bar);
            }
            // the ReLU mask of this row while the MMA runs
            float4 xm[kMine][4];
#pragma unroll
            for (int i = 0; i < kMine; ++i) {
                const int cc = grp + 2 * i;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    xm[i][u] = (g < p.B && cc < NH / 16) ? ld4(p.X[l] + g * 128 + cc * 16 + 4 * u)
                                                        : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            ok = wait_all(bs, ph, p.err);
            if (!ok) break;
            ph ^= 1;
            float* dst = p.G[l - 1] + g * 128;
#pragma unroll
            for (int i = 0; i < kMine; ++i) {
                const int cc = grp + 2 * i;
                if (cc >= NH / 16) break;
                uint32_t r[16];
                tmem_ld16(tl + cc * 16, r);
                tmem_wait_ld();
                float v[16];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float xs[4] = {xm[i][u].x, xm[i][u].y, xm[i][u].z, xm[i][u].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = cc * 16 + 4 * u + e;
                        v[4 * u + e] = (c < p.H && xs[e] > 0.f) ? __uint_as_float(r[4 * u + e]) : 0.f;
                    }
                }
                if (g < p.B) store16(dst + cc * 16, v);
                if (l > 1) put_act16(a_row, cc * 16, v);
            }
            tc_fence_before();
            fence_proxy_async();
            __syncthreads();
        }
    }
    tc_end(bs, tmem, kCols, ok);
}

// ---------------------------------------------------------------------------
// weight and bias gradients: CTA b handles layer b / Gl, tiles (b % Gl) + i Gl
__host__ __device__ constexpr uint32_t dw_lbo_b(int N) { return (uint32_t)(N / 8) * kTSbo; }
__host__ __device__ constexpr uint32_t dw_bar_offset(int Nmax) { return 16 * kTLboA + 16 * dw_lbo_b(Nmax); }

template <int NH>
__global__ void __launch_bounds__(kThreads, NH <= 64 ? 3 : 2) k_tc_dw(const DwParams p, uint32_t cols)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t sbase = smem_u32(smem);
    const int l = blockIdx.x / p.Gl, part = blockIdx.x % p.Gl;
    const int in = l == 0 ? p.in0 : p.H;
    const int Kin = pad16(in), N = Kin + 16;
    const int Nmax = (pad16(p.in0) > NH ? pad16(p.in0) : NH) + 16;
    const uint32_t at = sbase, bt = sbase + 16 * kTLboA, lbo_b = dw_lbo_b(N);
    const Bars bs = bars_at(smem, dw_bar_offset(Nmax));

    tc_begin(bs, cols);
    // G^T rows (features) NH .. 127 stay zero; X^T gets a ones row at feature Kin (the bias gradient)
    for (int i = threadIdx.x; i < (int)(16 * kTLboA / 16); i += kThreads) st_shared_v4(at + 16 * i, 0u, 0u, 0u, 0u);
    {
        const int rb = threadIdx.x >> 4, f = threadIdx.x & 15;   // 16 sample blocks x 16 feature rows
        const uint32_t one = f == 0 ? 0x3F803F80u : 0u;
        st_shared_v4(bt + ((Kin + f) >> 3) * kTSbo + rb * lbo_b + ((Kin + f) & 7) * 16, one, one, one, one);
    }
    const uint32_t tmem = tc_begin_finish(bs);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, grp = warp >> 2;
    const uint32_t idesc = idesc_bf16(128, N);
    const int64_t n_tiles = (p.B + kRows - 1) / kRows;
    uint32_t ph = 0;
    int it = 0;
    bool ok = true;
    for (int64_t tile = part; tile < n_tiles; tile += p.Gl, ++it) {
        stage_cols(at, kTLboA, p.G[l], tile, p.B, p.H, NH);
        stage_cols(bt, lbo_b, p.X[l], tile, p.B, in, Kin);
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0 && !*bs.abort) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < kRows / 16; ++ks)
                mma_bf16(tmem, plain_desc(at + ks * 2 * kTLboA, kTLboA, kTSbo), plain_desc(bt + ks * 2 * lbo_b, lbo_b, kTSbo),
                         idesc, (it > 0 || ks > 0) ? 1u : 0u);
            mma_commit(bs.bar);
        }
        ok = wait_all(bs, ph, p.err);
        if (!ok) break;
        ph ^= 1;
    }
    if (ok) {
        // TMEM lane j = row j of dW_l; columns k < Kin are dW_l[j][k], column Kin is db_l[j]
        const int j = q * 32 + lane;
        const uint32_t tl = tmem + ((q * 32u) << 16);
        float* P = p.partial + (size_t)blockIdx.x * p.stride;
        for (int cc = grp; cc < N / 16; cc += 2) {
            float v[16];
            if (it > 0) {
                uint32_t r[16];
                tmem_ld16(tl + cc * 16, r);
                tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
            } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = 0.f;
            }
            if (j < p.H) {
                if (cc * 16 < Kin)
                    store16(P + (size_t)j * Kin + cc * 16, v);
                else
                    P[(size_t)p.H * Kin + j] = v[0];
            }
        }
    }
    tc_end(bs, tmem, cols, ok);
}

// ---------------------------------------------------------------------------
int tmem_cols_for(int n)
{
    int c = 32;
    while (c < n) c <<= 1;
    return c;
}
// dynamic shared memory that keeps (CTAs per SM) x cols within the 512 TMEM columns
int smem_for_tmem(int need, int cols)
{
    const int m = 512 / cols;
    const int floor_bytes = (kSmemPerSm + m) / (m + 1) - kSmemReserved + 16;
    return ((need > floor_bytes ? need : floor_bytes) + 15) & ~15;
}

// grid of a persistent launch: as many CTAs as fit at once; error when the
// residency would oversubscribe TMEM
cudaError_t resident_grid(const void* fn, int smem, int cols, int sm_count, int64_t want, int* grid)
{
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1 || occ * cols > 512) return cudaErrorInvalidConfiguration;
    const int64_t g = (int64_t)occ * sm_count;
    *grid = (int)(want < g ? want : g);
    return cudaSuccess;
}

template <int NH>
cudaError_t forward_nh(const TrainNet& net, int64_t B, TrainWork& wk, unsigned int* err, cudaStream_t s)
{
    FwdParams p = {};
    p.B = B;
    p.L = net.L;
    p.in0 = net.in0;
    p.K0 = pad16(net.in0);
    p.H = net.H;
    p.X0 = wk.X[0];
    for (int l = 1; l <= net.L; ++l) p.X[l] = wk.X[l];
    for (int l = 0; l < net.L; ++l) {
        p.W[l] = net.W[l];
        p.b[l] = net.b[l];
    }
    p.err = err;
    constexpr int kCols = NH < 32 ? 32 : NH;
    const int smem = smem_for_tmem((int)fwd_bar_offset<NH>(net.L, p.K0) + 32, kCols);
    int grid = 0;
    cudaError_t e = resident_grid((const void*)k_tc_fwd<NH>, smem, kCols, wk.sm_count, (B + kRows - 1) / kRows, &grid);
    if (e != cudaSuccess) return e;
    k_tc_fwd<NH><<<grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int NH>
cudaError_t backward_nh(const TrainNet& net, int64_t B, TrainWork& wk, unsigned int* err, int* Gl_out, int* stride_out,
                        cudaStream_t s)
{
    const int64_t n_tiles = (B + kRows - 1) / kRows;
    constexpr int kCols = NH < 32 ? 32 : NH;
    cudaError_t e;
    if (net.L > 1) {
        DxParams p = {};
        p.B = B;
        p.L = net.L;
        p.H = net.H;
        p.Gtop = wk.G[net.L - 1];
        for (int l = 1; l < net.L; ++l) {
            p.X[l] = wk.X[l];
            p.W[l] = net.W[l];
        }
        for (int l = 0; l + 1 < net.L; ++l) p.G[l] = wk.G[l];
        p.err = err;
        const int smem = smem_for_tmem((int)dx_bar_offset<NH>(net.L) + 32, kCols);
        int grid = 0;
        e = resident_grid((const void*)k_tc_dx<NH>, smem, kCols, wk.sm_count, n_tiles, &grid);
        if (e != cudaSuccess) return e;
        k_tc_dx<NH><<<grid, kThreads, smem, s>>>(p);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    DwParams p = {};
    p.B = B;
    p.L = net.L;
    p.H = net.H;
    p.in0 = net.in0;
    for (int l = 0; l < net.L; ++l) {
        p.G[l] = wk.G[l];
        p.X[l] = wk.X[l];
    }
    const int Kmax = pad16(net.in0) > NH ? pad16(net.in0) : NH;
    const int Nmax = Kmax + 16;
    p.stride = (NH * Kmax + NH + 3) & ~3;
    p.partial = wk.partial;
    p.err = err;
    const int cols = tmem_cols_for(Nmax);
    const int smem = smem_for_tmem((int)dw_bar_offset(Nmax) + 32, cols);
    int resident = 0;
    e = resident_grid((const void*)k_tc_dw<NH>, smem, cols, wk.sm_count, (int64_t)1 << 30, &resident);
    if (e != cudaSuccess) return e;
    int Gl = resident / net.L;
    if (Gl > wk.n_blocks / net.L) Gl = wk.n_blocks / net.L;   // partial slots
    if ((int64_t)Gl > n_tiles) Gl = (int)n_tiles;
    if (Gl < 1) Gl = 1;
    if ((int64_t)Gl * net.L * p.stride > (int64_t)wk.n_blocks * (128 * 128 + 128)) return cudaErrorInvalidValue;
    p.Gl = Gl;
    k_tc_dw<NH><<<Gl * net.L, kThreads, smem, s>>>(p, (uint32_t)cols);
    *Gl_out = Gl;
    *stride_out = p.stride;
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
bool train_tc_supported(const TrainNet& net)
{
    return net.L >= 1 && net.L <= kMaxLayers && net.H >= 1 && net.H <= 128 && net.in0 >= 1 && net.in0 <= 128;
}

cudaError_t train_tc_forward(const TrainNet& net, int64_t B, TrainWork& wk, unsigned int* err, cudaStream_t s)
{
    if (!train_tc_supported(net)) return cudaErrorInvalidValue;
    if (net.H <= 32) return forward_nh<32>(net, B, wk, err, s);
    if (net.H <= 64) return forward_nh<64>(net, B, wk, err, s);
    return forward_nh<128>(net, B, wk, err, s);
}

cudaError_t train_tc_backward(const TrainNet& net, int64_t B, TrainWork& wk, unsigned int* err, int* Gl, int* stride,
                              cudaStream_t s)
{
    if (!train_tc_supported(net)) return cudaErrorInvalidValue;
    if (net.H <= 32) return backward_nh<32>(net, B, wk, err, Gl, stride, s);
    if (net.H <= 64) return backward_nh<64>(net, B, wk, err, Gl, stride, s);
    return backward_nh<128>(net, B, wk, err, Gl, stride, s);
}

}  // namespace ptk
