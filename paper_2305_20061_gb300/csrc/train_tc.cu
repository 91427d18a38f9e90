// Tensor-core GEMMs of MLP training: the HDR NIF (Section 3.2.1) and the
// online radiance cache (Section 3.3).  BF16 operands, FP32 accumulation in
// TMEM (tcgen05), FP32 activations in HBM ([sample][128] rows), FP32 master
// weights.
//
//   forward   X[l+1] = relu(X[l] W_l^T + b_l), l = 0 .. L-1.  A CTA holds
//             every hidden layer's weights in shared memory and takes each
//             128-row tile through all layers: the ReLU output of one layer,
//             rounded to BF16, is the A operand of the next.  Only X[L], the
//             output layer's input, is written in FP32.
//   backward  G[l-1] = (G[l] W_l) * [X[l] > 0], l = L-1 .. 1, chained the
//             same way from the output layer's gradient G[L-1]; the ReLU
//             masks come from the BF16 tiles of X[l].
//   weights   dW_l = G[l]^T X[l] and db_l = the column sums of G[l].  The
//             batch is the reduction.  The two chains also write every BF16
//             operand tile they build (X[0 .. L-1], G[0 .. L-1]) to HBM in
//             the MMA's core-matrix layout; read back as MN-major operands
//             (rows = samples = K) they need no transposition, so the weight
//             kernel is a TMA bulk-copy pipeline feeding the MMA.  A constant
//             ones column appended to X[l] yields db_l in the same MMA.  A CTA
//             accumulates its share of the batch for one layer in TMEM and
//             writes one partial; partials are summed in a fixed order, so
//             the gradient is deterministic.
//
// Shared-memory operands use the SWIZZLE_NONE core-matrix layout (8 rows x
// 16 bytes); the strides of the activation tiles keep the staging stores free
// of bank conflicts.  Every mbarrier wait is bounded; a CTA that gives up
// sets PT_ERR_TIMEOUT, waits (bounded) for its MMAs and frees TMEM.
#include <cstdint>

#include <cuda_runtime.h>

#include "tc_ptx.cuh"

namespace ptk {

namespace {

using namespace tc;

constexpr int kRows = 128;                   // samples per tile (M of the row GEMMs, K of the weight GEMM)
constexpr int kThreads = 512;                // 16 warps: four per TMEM lane quarter; warp w stages rows 8w .. 8w+7
constexpr int kGroups = kThreads / 128;      // warps sharing a lane quarter (they split the columns)
constexpr int kMaxLayers = 8;
constexpr uint32_t kActLbo = 16 * 128 + 16;  // activation tile: byte step between 8-column core blocks
constexpr uint32_t kTileCb = 2048;           // HBM operand tile: byte step between 8-column blocks (128 rows x 16 B)
constexpr uint32_t kBarBytes = 32;           // two MMA barriers, the drain barrier, TMEM address, abort flag
constexpr int kDwThreads = 128;              // weight kernel: one thread drives the pipeline, four warps drain TMEM
constexpr int kDwMaxStages = 4;
constexpr uint32_t kDwBarBytes = 128;        // full / empty per stage, done, drain, TMEM address, abort flag
constexpr int kSmemPerSm = 233472;           // 228 KiB of shared memory per SM
constexpr int kSmemLimit = 227 * 1024;       // dynamic shared memory of one CTA
constexpr int kSmemReserved = 1024;          // reserved per CTA

__host__ __device__ constexpr int pad16(int n) { return (n + 15) & ~15; }

struct FwdParams {
    int64_t B;
    int L, in0, K0, H;
    const float* X0;
    float* XL;                       // X[L] (the output layer's input) written in FP32, tiled: element (r, c)
                                     // of tile t at t * 16384 + (c >> 2) * 512 + r * 4 + (c & 3)
    unsigned char* Xb[kMaxLayers];   // BF16 operand tiles of X[0 .. L-1] written
    const float* W[kMaxLayers];
    const float* b[kMaxLayers];
    unsigned int* err;
};

struct DxParams {
    int64_t B;
    int L, H;
    const float* Gtop;               // G[L-1]
    const unsigned char* Xb[kMaxLayers];   // BF16 tiles of X[1 .. L-1]: the ReLU masks (BF16 > 0 iff FP32 > 0
                                           // for every value above 2^-134)
    unsigned char* Gb[kMaxLayers];   // BF16 operand tiles of G[0 .. L-1] written
    const float* W[kMaxLayers];      // W[1 .. L-1]
    unsigned int* err;
};

struct DwParams {
    int64_t B;
    int L, H, in0, Gl, stride;       // Gl CTAs per layer, stride floats per partial
    int stages;                      // pipeline depth
    const unsigned char* Gb[kMaxLayers];
    const unsigned char* Xb[kMaxLayers];
    float* partial;                  // [L * Gl][stride]: [H][pad16(in)] dW, then [H] db
    unsigned int* err;
};

struct Bars {
    uint32_t bar[2], drain;
    uint32_t* tmem_slot;
    volatile int* abort;
};

__device__ __forceinline__ Bars bars_at(unsigned char* smem, uint32_t off)
{
    Bars b;
    b.bar[0] = smem_u32(smem + off);
    b.bar[1] = b.bar[0] + 8;
    b.drain = b.bar[0] + 16;
    b.tmem_slot = reinterpret_cast<uint32_t*>(smem + off + 24);
    b.abort = reinterpret_cast<volatile int*>(smem + off + 28);
    return b;
}

// barrier init (thread 0) and TMEM allocation (warp 0); the caller then stages
// its constant operands and calls tc_begin_finish
__device__ __forceinline__ void tc_begin(const Bars& b, uint32_t cols)
{
    if (threadIdx.x == 0) {
        mbar_init(b.bar[0], 1);
        mbar_init(b.bar[1], 1);
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

// the whole CTA waits for a commit on `bar`; true when every thread saw it
__device__ __forceinline__ bool wait_all(const Bars& b, uint32_t bar, uint32_t ph, unsigned int* err)
{
    const bool got = mbar_wait(bar, ph, b.abort, err);
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

// This warp's 8 rows (8w .. 8w+7) of rows [tile*128, +128) of a [B][128]
// FP32 matrix, columns 4l .. 4l+3 for lane l (one coalesced row per load).
// Rows >= B and lanes with 4l >= min(K, width) load nothing (their values are
// left as they are); nothing here waits for the loads, so the registers can
// fill while the caller works on the previous tile.
__device__ __forceinline__ void load_rows8(float4 (&v)[8], const float* __restrict__ X, int64_t tile, int64_t B,
                                           int width, int K)
{
    const int warp = threadIdx.x >> 5, c = 4 * (threadIdx.x & 31);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t g = tile * kRows + warp * 8 + i;
        if (c < K && c < width && g < B) v[i] = ld4(X + g * 128 + c);
    }
}

// ... as BF16 into the activation tile: byte (r>>3)*128 + (c>>3)*kActLbo +
// (r&7)*16 + (c&7)*2 (the A operand of the row GEMMs, K = columns); rows >= B
// and columns >= width become zeros
__device__ __forceinline__ void store_rows8(uint32_t a, const float4 (&v)[8], int64_t tile, int64_t B, int width,
                                            int K)
{
    const int warp = threadIdx.x >> 5, c = 4 * (threadIdx.x & 31);
    if (c >= K) return;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t g = tile * kRows + warp * 8 + i;
        const float4 x = (g < B && c < width) ? mask4(v[i], c, width) : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t addr = a + warp * 128 + (c >> 3) * kActLbo + i * 16 + (c & 7) * 2;
        asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(pack_bf16(x.x, x.y)), "r"(pack_bf16(x.z, x.w))
                     : "memory");
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
__device__ __forceinline__ void pack16(const float (&v)[16], uint32_t (&w)[8])
{
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = pack_bf16(v[2 * i], v[2 * i + 1]);
}
// 16 columns c0 .. c0+15 of activation-tile row `row` (two core blocks)
__device__ __forceinline__ void put_act16(uint32_t a_row, int c0, const uint32_t (&w)[8])
{
    const uint32_t p = a_row + (uint32_t)(c0 >> 3) * kActLbo;
    st_shared_v4(p, w[0], w[1], w[2], w[3]);
    st_shared_v4(p + kActLbo, w[4], w[5], w[6], w[7]);
}
// ... and of the HBM operand tile: byte (r>>3)*128 + (c>>3)*kTileCb + (r&7)*16 + (c&7)*2 (a warp's 32 rows
// are 512 contiguous bytes)
__device__ __forceinline__ void put_tile16(unsigned char* tile, int row, int c0, const uint32_t (&w)[8])
{
    uint4* d = reinterpret_cast<uint4*>(tile + (size_t)(c0 >> 3) * kTileCb + row * 16);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[kTileCb / 16] = make_uint4(w[4], w[5], w[6], w[7]);
}
// the activation tile's columns [0, C) -> the HBM operand tile (16-byte units, coalesced)
__device__ __forceinline__ void copy_act_to_tile(unsigned char* tile, uint32_t a, int C)
{
    for (int u = threadIdx.x; u < kRows * (C / 8); u += kThreads) {
        const int r = u & (kRows - 1), cb = u >> 7;
        uint32_t x0, x1, x2, x3;
        asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(x0), "=r"(x1), "=r"(x2), "=r"(x3)
                     : "r"(a + cb * kActLbo + r * 16)
                     : "memory");
        *reinterpret_cast<uint4*>(tile + (size_t)cb * kTileCb + r * 16) = make_uint4(x0, x1, x2, x3);
    }
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
__global__ void __launch_bounds__(kThreads, 1) k_tc_fwd(const FwdParams p)
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
    float4 pf[8] = {};   // the next tile's input rows, loaded while this tile runs through the layers
    load_rows8(pf, p.X0, blockIdx.x, p.B, p.in0, K0);
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        store_rows8(a, pf, tile, p.B, p.in0, K0);
        fence_proxy_async();
        __syncthreads();
        if (tile + gridDim.x < n_tiles) load_rows8(pf, p.X0, tile + gridDim.x, p.B, p.in0, K0);
        copy_act_to_tile(p.Xb[0] + (size_t)tile * kRows * K0 * 2, a, K0);   // read before layer 0's epilogue
        const int64_t g = tile * kRows + row;
        for (int l = 0; l < L; ++l) {
            if (threadIdx.x == 0 && !*bs.abort) {
                tc_fence_after();
                const int K = l == 0 ? K0 : NH;
                const uint32_t w = sbase + (l == 0 ? 0u : w0_bytes + (uint32_t)(l - 1) * wl_bytes);
                for (int ks = 0; ks < K / 16; ++ks)
                    mma_bf16(tmem, plain_desc(a + ks * 2 * kActLbo, kActLbo, 128),
                             plain_desc(w + ks * 2 * (NH * 16), NH * 16, 128), idesc, ks > 0);
                mma_commit(bs.bar[0]);
            }
            ok = wait_all(bs, bs.bar[0], ph, p.err);
            if (!ok) break;
            ph ^= 1;
            float* dst = p.XL + tile * (kRows * 128) + row * 4;
#pragma unroll
            for (int cc = grp; cc < NH / 16; cc += kGroups) {
                uint32_t r[16];
                tmem_ld16(tl + cc * 16, r);
                tmem_wait_ld();
                float v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int c = cc * 16 + e;
                    v[e] = c < p.H ? fmaxf(__uint_as_float(r[e]) + bias[l * NH + c], 0.f) : 0.f;
                }
                if (l + 1 == L && g < p.B) {
                    // four 16-byte column groups; a warp's 32 rows of one group are 512 contiguous bytes
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        *reinterpret_cast<float4*>(dst + (cc * 4 + u) * (kRows * 4)) =
                            make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
                }
                if (l + 1 < L) {
                    uint32_t w[8];
                    pack16(v, w);
                    put_act16(a_row, cc * 16, w);
                    put_tile16(p.Xb[l + 1] + (size_t)tile * kRows * NH * 2, row, cc * 16, w);
                }
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
__global__ void __launch_bounds__(kThreads, 1) k_tc_dx(const DxParams p)
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
    constexpr int kMine = (NH / 16 + kGroups - 1) / kGroups;   // column chunks per thread
    const int64_t n_tiles = (p.B + kRows - 1) / kRows;
    uint32_t ph = 0;
    bool ok = true;
    float4 pf[8] = {};
    load_rows8(pf, p.Gtop, blockIdx.x, p.B, p.H, NH);
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        store_rows8(a, pf, tile, p.B, p.H, NH);
        fence_proxy_async();
        __syncthreads();
        if (tile + gridDim.x < n_tiles) load_rows8(pf, p.Gtop, tile + gridDim.x, p.B, p.H, NH);
        copy_act_to_tile(p.Gb[L - 1] + (size_t)tile * kRows * NH * 2, a, NH);
        if (L == 1) __syncthreads();   // no layer step below: the next tile's staging must wait for the copy
        const int64_t g = tile * kRows + row;
        for (int l = L - 1; l >= 1; --l) {
            if (threadIdx.x == 0 && !*bs.abort) {
                tc_fence_after();
                const uint32_t w = sbase + (uint32_t)(l - 1) * wl_bytes;
                for (int ks = 0; ks < NH / 16; ++ks)
                    mma_bf16(tmem, plain_desc(a + ks * 2 * kActLbo, kActLbo, 128),
                             plain_desc(w + ks * 2 * (NH * 16), NH * 16, 128), idesc, ks > 0);
                mma_commit(bs.bar[0]);
            }
            // the ReLU mask of this row (16 BF16 values per chunk) while the MMA runs
            uint4 xm[kMine][2];
            const unsigned char* xt = p.Xb[l] + (size_t)tile * kRows * NH * 2 + row * 16;
#pragma unroll
            for (int i = 0; i < kMine; ++i) {
                const int cc = grp + kGroups * i;
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    xm[i][u] = cc < NH / 16 ? __ldg(reinterpret_cast<const uint4*>(xt + (size_t)(2 * cc + u) * kTileCb))
                                            : make_uint4(0u, 0u, 0u, 0u);
            }
            ok = wait_all(bs, bs.bar[0], ph, p.err);
            if (!ok) break;
            ph ^= 1;
            unsigned char* gt = p.Gb[l - 1] + (size_t)tile * kRows * NH * 2;
#pragma unroll
            for (int i = 0; i < kMine; ++i) {
                const int cc = grp + kGroups * i;
                if (cc >= NH / 16) break;
                uint32_t r[16];
                tmem_ld16(tl + cc * 16, r);
                tmem_wait_ld();
                float v[16];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const uint32_t xw[4] = {xm[i][u].x, xm[i][u].y, xm[i][u].z, xm[i][u].w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int c = cc * 16 + 8 * u + e;
                        const float x = __uint_as_float((e & 1) ? (xw[e >> 1] & 0xFFFF0000u) : (xw[e >> 1] << 16));
                        v[8 * u + e] = (c < p.H && x > 0.f) ? __uint_as_float(r[8 * u + e]) : 0.f;
                    }
                }
                uint32_t w[8];
                pack16(v, w);
                if (l > 1) put_act16(a_row, cc * 16, w);
                put_tile16(gt, row, cc * 16, w);
            }
            tc_fence_before();
            fence_proxy_async();
            __syncthreads();
        }
    }
    tc_end(bs, tmem, kCols, ok);
}

// ---------------------------------------------------------------------------
// weight and bias gradients: CTA b handles layer b / Gl, tiles (b % Gl) + i Gl.
// Stage s of the pipeline: the G tile as the MN-major A operand (128 feature
// rows; features >= NH stay zero), then the X tile followed by a ones column
// (feature Kin) as the MN-major B operand.  Both are copied by TMA straight
// from the HBM operand tiles, which have the same layout.
__host__ __device__ constexpr uint32_t dw_a_bytes() { return 16 * kTileCb; }
__host__ __device__ constexpr uint32_t dw_b_bytes(int Kmax)
{
    return (uint32_t)((Kmax / 8 + 2) > 16 ? (Kmax / 8 + 2) : 16) * kTileCb;   // >= 16 blocks: see the launch
}
__host__ __device__ constexpr uint32_t dw_stage_bytes(int Kmax) { return dw_a_bytes() + dw_b_bytes(Kmax); }

template <int NH>
__global__ void __launch_bounds__(kDwThreads, 1) k_tc_dw(const DwParams p, uint32_t cols)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t sbase = smem_u32(smem);
    const int l = blockIdx.x / p.Gl, part = blockIdx.x % p.Gl;
    const int Kin = l == 0 ? pad16(p.in0) : NH;   // the X tile's width (as the chains wrote it)
    const int N = Kin + 16;
    const int Kmax = pad16(p.in0) > NH ? pad16(p.in0) : NH;
    const uint32_t stage = dw_stage_bytes(Kmax);
    const int S = p.stages;
    const uint32_t bars = S * stage;
    const uint32_t full0 = sbase + bars, empty0 = full0 + 8 * kDwMaxStages, done = empty0 + 8 * kDwMaxStages;
    const uint32_t drain = done + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + bars + 16 * kDwMaxStages + 16);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + bars + 16 * kDwMaxStages + 20);

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(full0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, 1);
        }
        mbar_init(done, 1);
        mbar_init(drain, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // constant parts of every stage: A feature blocks NH/8 .. 15 zero; B block Kin/8 = [1, 0 .. 0] per
    // sample row (the ones column), block Kin/8 + 1 zero
    for (int i = 0; i < S; ++i) {
        const uint32_t st = sbase + i * stage;
        for (int u = threadIdx.x; u < (int)((16 - NH / 8) * (kTileCb / 16)); u += kDwThreads)
            st_shared_v4(st + (NH / 8) * kTileCb + 16 * u, 0u, 0u, 0u, 0u);
        for (int u = threadIdx.x; u < 2 * kRows; u += kDwThreads) {
            const int blk = u >> 7, r = u & (kRows - 1);
            st_shared_v4(st + dw_a_bytes() + (Kin / 8 + blk) * kTileCb + r * 16, blk == 0 ? 0x3F80u : 0u, 0u, 0u, 0u);
        }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int64_t n_tiles = (p.B + kRows - 1) / kRows;
    const int n_my = part < n_tiles ? (int)((n_tiles - 1 - part) / p.Gl + 1) : 0;
    if (threadIdx.x == 0) {
        // MN-major A and B (transpose bits 15 and 16): core matrices of 8 samples x 16 bytes (8 features);
        // K (samples) steps 128 bytes per 8 samples, features step kTileCb per 8
        const uint32_t idesc = idesc_bf16(128, N) | (1u << 15) | (1u << 16);
        const uint32_t gbytes = kRows * NH * 2, xbytes = kRows * Kin * 2;
        const unsigned char* gsrc = p.Gb[l];
        const unsigned char* xsrc = p.Xb[l];
        bool ok = true;
        for (int i = 0; i < n_my + S - 1 && ok; ++i) {
            if (i < n_my) {   // TMA of tile i into stage i % S once the MMAs of tile i - S are done with it
                const int s = i % S;
                const int64_t tile = part + (int64_t)i * p.Gl;
                if (i >= S) ok = mbar_wait(empty0 + 8 * s, (uint32_t)((i / S - 1) & 1), abort, p.err);
                if (!ok) break;
                const uint32_t st = sbase + s * stage;
                mbar_expect_tx(full0 + 8 * s, gbytes + xbytes);
                bulk_g2s(st, gsrc + (size_t)tile * gbytes, gbytes, full0 + 8 * s);
                bulk_g2s(st + dw_a_bytes(), xsrc + (size_t)tile * xbytes, xbytes, full0 + 8 * s);
            }
            const int j = i - (S - 1);
            if (j >= 0) {     // MMAs of tile j
                const int s = j % S;
                ok = mbar_wait(full0 + 8 * s, (uint32_t)((j / S) & 1), abort, p.err);
                if (!ok) break;
                tc_fence_after();
                const uint32_t st = sbase + s * stage;
#pragma unroll
                for (int ks = 0; ks < kRows / 16; ++ks)
                    mma_bf16(tmem, plain_desc(st + ks * 256, 128, kTileCb),
                             plain_desc(st + dw_a_bytes() + ks * 256, 128, kTileCb), idesc,
                             (j > 0 || ks > 0) ? 1u : 0u);
                mma_commit(empty0 + 8 * s);
            }
        }
        if (ok) {
            mma_commit(done);
            ok = mbar_wait(done, 0, abort, p.err);
        }
        if (!ok) {
            *abort = 1;
            mma_commit(drain);
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait(drain, 0) && global_ns() - t0 < kWaitBudgetNs) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (!*abort) {
        // TMEM lane j = row j of dW_l; columns k < Kin are dW_l[j][k], column Kin is db_l[j]
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int j = warp * 32 + lane;
        const uint32_t tl = tmem + ((warp * 32u) << 16);
        float* P = p.partial + (size_t)blockIdx.x * p.stride;
        for (int cc = 0; cc < N / 16; ++cc) {
            float v[16];
            if (n_my > 0) {
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
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
    }
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
cudaError_t resident_grid(const void* fn, int threads, int smem, int cols, int sm_count, int64_t want, int* grid)
{
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
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
    p.XL = wk.X[net.L];
    for (int l = 0; l < net.L; ++l) {
        p.Xb[l] = wk.Xb[l];
        p.W[l] = net.W[l];
        p.b[l] = net.b[l];
    }
    p.err = err;
    constexpr int kCols = NH < 32 ? 32 : NH;
    const int smem = smem_for_tmem((int)(fwd_bar_offset<NH>(net.L, p.K0) + kBarBytes), kCols);
    int grid = 0;
    cudaError_t e = resident_grid((const void*)k_tc_fwd<NH>, kThreads, smem, kCols, wk.sm_count,
                                  (B + kRows - 1) / kRows, &grid);
    if (e != cudaSuccess) return e;
    k_tc_fwd<NH><<<grid, kThreads, smem, s>>>(p); count_launch();
    return cudaGetLastError();
}

template <int NH>
cudaError_t backward_nh(const TrainNet& net, int64_t B, TrainWork& wk, unsigned int* err, int* Gl_out, int* stride_out,
                        int* pitch, cudaStream_t s)
{
    const int64_t n_tiles = (B + kRows - 1) / kRows;
    constexpr int kCols = NH < 32 ? 32 : NH;
    cudaError_t e;
    {
        DxParams p = {};
        p.B = B;
        p.L = net.L;
        p.H = net.H;
        p.Gtop = wk.dX[0];
        for (int l = 1; l < net.L; ++l) {
            p.Xb[l] = wk.Xb[l];
            p.W[l] = net.W[l];
        }
        for (int l = 0; l < net.L; ++l) p.Gb[l] = wk.Gb[l];
        p.err = err;
        const int smem = smem_for_tmem((int)(dx_bar_offset<NH>(net.L) + kBarBytes), kCols);
        int grid = 0;
        e = resident_grid((const void*)k_tc_dx<NH>, kThreads, smem, kCols, wk.sm_count, n_tiles, &grid);
        if (e != cudaSuccess) return e;
        k_tc_dx<NH><<<grid, kThreads, smem, s>>>(p); count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    DwParams p = {};
    p.B = B;
    p.L = net.L;
    p.H = net.H;
    p.in0 = net.in0;
    for (int l = 0; l < net.L; ++l) {
        p.Gb[l] = wk.Gb[l];
        p.Xb[l] = wk.Xb[l];
    }
    const int Kmax = pad16(net.in0) > NH ? pad16(net.in0) : NH;
    const int Nmax = Kmax + 16;
    p.stride = (NH * Kmax + NH + 3) & ~3;
    p.partial = wk.partial;
    p.err = err;
    // B regions of at least 16 feature blocks and A regions of exactly 16: every operand read stays inside
    // its stage for either assignment of the two descriptor strides to the two directions
    const int budget = 227 * 1024 - (int)kDwBarBytes;
    int stages = budget / (int)dw_stage_bytes(Kmax);
    if (stages > kDwMaxStages) stages = kDwMaxStages;
    if (stages < 2) return cudaErrorInvalidConfiguration;
    p.stages = stages;
    const int cols = tmem_cols_for(Nmax);
    const int smem = smem_for_tmem(stages * (int)dw_stage_bytes(Kmax) + (int)kDwBarBytes, cols);
    int resident = 0;
    e = resident_grid((const void*)k_tc_dw<NH>, kDwThreads, smem, cols, wk.sm_count, (int64_t)1 << 30, &resident);
    if (e != cudaSuccess) return e;
    int Gl = resident / net.L;
    if (Gl > wk.n_blocks / net.L) Gl = wk.n_blocks / net.L;   // partial slots
    if ((int64_t)Gl > n_tiles) Gl = (int)n_tiles;
    if (Gl < 1) Gl = 1;
    if ((int64_t)Gl * net.L * p.stride > (int64_t)wk.n_blocks * (128 * 128 + 128)) return cudaErrorInvalidValue;
    p.Gl = Gl;
    k_tc_dw<NH><<<Gl * net.L, kDwThreads, smem, s>>>(p, (uint32_t)cols); count_launch();
    *Gl_out = Gl;
    *stride_out = p.stride;
    for (int l = 0; l < net.L; ++l) pitch[l] = l == 0 ? pad16(net.in0) : NH;
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
namespace {
// the chains keep every layer's weights in shared memory: the shapes whose images fit
template <int NH>
bool fits(int L, int in0)
{
    const int K0 = pad16(in0);
    return (int)(fwd_bar_offset<NH>(L, K0) + kBarBytes) <= kSmemLimit &&
           (int)(dx_bar_offset<NH>(L) + kBarBytes) <= kSmemLimit;
}
}  // namespace

bool train_tc_supported(const TrainNet& net)
{
    if (!(net.L >= 1 && net.L <= kMaxLayers && net.H >= 1 && net.H <= 128 && net.in0 >= 1 && net.in0 <= 128))
        return false;
    if (net.H <= 32) return fits<32>(net.L, net.in0);
    if (net.H <= 64) return fits<64>(net.L, net.in0);
    return fits<128>(net.L, net.in0);
}

cudaError_t train_tc_forward(const TrainNet& net, int64_t B, TrainWork& wk, unsigned int* err, cudaStream_t s)
{
    if (!train_tc_supported(net)) return cudaErrorInvalidValue;
    if (net.H <= 32) return forward_nh<32>(net, B, wk, err, s);
    if (net.H <= 64) return forward_nh<64>(net, B, wk, err, s);
    return forward_nh<128>(net, B, wk, err, s);
}

cudaError_t train_tc_backward(const TrainNet& net, int64_t B, TrainWork& wk, unsigned int* err, int* Gl, int* stride,
                              int* pitch, cudaStream_t s)
{
    if (!train_tc_supported(net)) return cudaErrorInvalidValue;
    if (net.H <= 32) return backward_nh<32>(net, B, wk, err, Gl, stride, pitch, s);
    if (net.H <= 64) return backward_nh<64>(net, B, wk, err, Gl, stride, pitch, s);
    return backward_nh<128>(net, B, wk, err, Gl, stride, pitch, s);
}

}  // namespace ptk
