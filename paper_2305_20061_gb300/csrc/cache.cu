// Neural radiance cache queries (Mueller et al. 2021, which Section 2.1
// cites as the way to end paths early): one fused kernel evaluates the whole
// MLP for a tile of 128 queries with every weight resident in shared memory.
//
// Network: frequency-encoded position (J sin/cos pairs per axis, position
// normalised to the scene box), raw direction and normal -> L hidden FC-64
// ReLU layers -> FC-3.  A query row holds x[3], wo[3], n[3] (evaluation) or
// the 16-float row the bounce kernel writes at the cache vertex:
// x, wo, n, throughput tp[3], radiance gathered before the vertex L[3] and
// the path's slot (bits).  For those the result is written as the path's
// radiance: L_slot = tp * max(cache, 0) (+ L when the scene emits).
//
// Persistent CTAs (one per SM, 256 threads).  A layer is a 128 x 64 output
// tile: warp w owns columns 8w..8w+7 (its weight reads are broadcasts) and
// lane l rows 4l..4l+3 (conflict-free float4 reads of the transposed
// activations), 32 FP32 accumulators per thread.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace ptk {

namespace {

constexpr int kThreads = 256;
constexpr int kRows = 128;
constexpr int kH = 64;

struct Layout {
    int k0p;      // layer-0 input width padded to a multiple of 8
    int w0, w, bias, wout, bout, act_a, act_b, total;   // float offsets / count
};

__host__ __device__ inline Layout cache_layout(int in0, int L)
{
    Layout s;
    s.k0p = (in0 + 7) & ~7;
    s.w0 = 0;                                   // [k0p][64], W0 transposed
    s.w = s.w0 + s.k0p * kH;                    // [L-1][64][64], transposed
    s.bias = s.w + (L - 1) * kH * kH;           // [L][64]
    s.wout = s.bias + L * kH;                   // [3][64]
    s.bout = s.wout + 3 * kH;                   // [4]
    s.act_a = s.bout + 4;                       // [max(k0p, 64)][128]
    s.act_b = s.act_a + (s.k0p > kH ? s.k0p : kH) * kRows;   // [64][128]
    s.total = s.act_b + kH * kRows;
    return s;
}

struct EvalParams {
    const float* params;     // flat: W0 [64][in0], b0, W1 [64][64], b1, ..., WL [3][64], bL
    int J, L, in0;
    CacheBox box;
    const float* rows;       // [cap][stride]
    int stride;              // 9 (plain evaluation) or 16 (render queries)
    int64_t cap;
    const uint32_t* n_dev;   // nullable: live row count
    float* out;              // stride 9: raw outputs [n][3]
    float* slot_L;           // stride 16: path radiance [slot][3]
    int accumulate;
    uint32_t* err;
    unsigned long long* stats;   // nullable: += queries evaluated
};

// acc[r][c] += sum_k X[k][4 lane + r] * Wt[k][8 warp + c]
__device__ __forceinline__ void layer_tile(const float* __restrict__ X, const float* __restrict__ Wt, int K, int lane,
                                           int warp, float acc[4][8])
{
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float4 x = *reinterpret_cast<const float4*>(&X[k * kRows + 4 * lane]);
        const float4 w0 = *reinterpret_cast<const float4*>(&Wt[k * kH + 8 * warp]);
        const float4 w1 = *reinterpret_cast<const float4*>(&Wt[k * kH + 8 * warp + 4]);
        const float xv[4] = {x.x, x.y, x.z, x.w};
        const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(xv[r], wv[c], acc[r][c]);
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_cache_eval(const EvalParams p)
{
    extern __shared__ float4 smem4[];
    float* sm = reinterpret_cast<float*>(smem4);
    const Layout lay = cache_layout(p.in0, p.L);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // weights -> shared memory, transposed to [in][out]
    {
        const float* src = p.params;
        for (int l = 0; l < p.L; ++l) {
            const int in = l == 0 ? p.in0 : kH, kp = l == 0 ? lay.k0p : kH;
            float* dst = sm + (l == 0 ? lay.w0 : lay.w + (l - 1) * kH * kH);
            for (int idx = tid; idx < kp * kH; idx += kThreads) {
                const int k = idx / kH, j = idx % kH;
                dst[idx] = k < in ? src[(size_t)j * in + k] : 0.f;
            }
            src += (size_t)in * kH;
            for (int j = tid; j < kH; j += kThreads) sm[lay.bias + l * kH + j] = src[j];
            src += kH;
        }
        for (int idx = tid; idx < 3 * kH; idx += kThreads) sm[lay.wout + idx] = src[idx];
        if (tid < 3) sm[lay.bout + tid] = src[3 * kH + tid];
    }
    const int64_t n = p.n_dev ? min((int64_t)*p.n_dev, p.cap) : p.cap;
    const int64_t n_tiles = (n + kRows - 1) / kRows;
    if (p.stats && blockIdx.x == 0 && tid == 0) atomicAdd(p.stats, (unsigned long long)n);
    float* A = sm + lay.act_a;
    float* Bf = sm + lay.act_b;
    const int J = p.J;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t row0 = tile * kRows;
        __syncthreads();   // previous tile's readers are done with A / Bf
        // encoding -> A [feature][row]
        for (int idx = tid; idx < 3 * kRows; idx += kThreads) {
            const int r = idx % kRows, a = idx / kRows;
            const int64_t g = row0 + r;
            float* s = A + (2 * J * a) * kRows + r;
            if (g < n) {
                cache_axis_features(p.rows[g * p.stride + a], p.box.lo[a], p.box.eh[a], p.box.el[a], J, s, kRows,
                                    s + J * kRows, kRows);
            } else {
                for (int j = 0; j < 2 * J; ++j) s[j * kRows] = 0.f;
            }
        }
        for (int idx = tid; idx < (lay.k0p - 6 * J) * kRows; idx += kThreads) {
            const int r = idx % kRows, f = idx / kRows;
            const int64_t g = row0 + r;
            A[(6 * J + f) * kRows + r] = (f < 6 && g < n) ? p.rows[g * p.stride + 3 + f] : 0.f;
        }
        __syncthreads();
        // hidden layers, ping-pong between A and Bf
        float* X = A;
        float* Y = Bf;
        for (int l = 0; l < p.L; ++l) {
            const float* Wt = sm + (l == 0 ? lay.w0 : lay.w + (l - 1) * kH * kH);
            const float* b = sm + lay.bias + l * kH + 8 * warp;
            float acc[4][8];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = b[c];
            layer_tile(X, Wt, l == 0 ? lay.k0p : kH, lane, warp, acc);
            // Y was last read as the previous layer's input, before that layer's barrier
#pragma unroll
            for (int c = 0; c < 8; ++c)
                *reinterpret_cast<float4*>(&Y[(8 * warp + c) * kRows + 4 * lane]) =
                    make_float4(fmaxf(acc[0][c], 0.f), fmaxf(acc[1][c], 0.f), fmaxf(acc[2][c], 0.f),
                                fmaxf(acc[3][c], 0.f));
            __syncthreads();
            float* t = X; X = Y; Y = t;
        }
        // output layer: thread r < 128 owns row r
        if (tid < kRows) {
            const int64_t g = row0 + tid;
            if (g < n) {
                float y0 = sm[lay.bout], y1 = sm[lay.bout + 1], y2 = sm[lay.bout + 2];
                const float* Wo = sm + lay.wout;
#pragma unroll 8
                for (int k = 0; k < kH; ++k) {
                    const float h = X[k * kRows + tid];
                    y0 = fmaf(Wo[k], h, y0);
                    y1 = fmaf(Wo[kH + k], h, y1);
                    y2 = fmaf(Wo[2 * kH + k], h, y2);
                }
                if (p.stride == 16) {
                    const float4 tq = *reinterpret_cast<const float4*>(p.rows + g * 16 + 8);   // n.z tp.xyz
                    const float4 lq = *reinterpret_cast<const float4*>(p.rows + g * 16 + 12);  // L.xyz slot
                    float a = tq.y * fmaxf(y0, 0.f), bb = tq.z * fmaxf(y1, 0.f), c = tq.w * fmaxf(y2, 0.f);
                    if (p.accumulate) { a += lq.x; bb += lq.y; c += lq.z; }
                    if (!(isfinite(a) && isfinite(bb) && isfinite(c))) atomicOr(p.err, PT_ERR_NONFINITE);
                    float* L = p.slot_L + 3 * (size_t)__float_as_uint(lq.w);
                    L[0] = a; L[1] = bb; L[2] = c;
                } else {
                    p.out[3 * g] = y0;
                    p.out[3 * g + 1] = y1;
                    p.out[3 * g + 2] = y2;
                }
            }
        }
    }
}

cudaError_t launch(const EvalParams& p, int sm_count, cudaStream_t s)
{
    if (p.cap <= 0) return cudaSuccess;
    const size_t bytes = (size_t)cache_layout(p.in0, p.L).total * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_cache_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (p.cap + kRows - 1) / kRows;
    k_cache_eval<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, sm_count)), kThreads, bytes, s>>>(p); count_launch();
    return cudaGetLastError();
}

}  // namespace

size_t cache_eval_smem_bytes(int in0, int L) { return (size_t)cache_layout(in0, L).total * sizeof(float); }

cudaError_t cache_eval(const float* params, int J, int L, CacheBox box, int64_t n, const float* q, float* out,
                       int sm_count, cudaStream_t s)
{
    EvalParams p = {};
    p.params = params; p.J = J; p.L = L; p.in0 = 6 * J + 6; p.box = box;
    p.rows = q; p.stride = 9; p.cap = n; p.out = out;
    return launch(p, sm_count, s);
}

cudaError_t cache_query(const float* params, int J, int L, CacheBox box, int64_t cap, const uint32_t* n_dev,
                        const float* rows, float* slot_L, int accumulate, uint32_t* err, unsigned long long* stats,
                        int sm_count, cudaStream_t s)
{
    EvalParams p = {};
    p.stats = stats;
    p.params = params; p.J = J; p.L = L; p.in0 = 6 * J + 6; p.box = box;
    p.rows = rows; p.stride = 16; p.cap = cap; p.n_dev = n_dev;
    p.slot_L = slot_L; p.accumulate = accumulate; p.err = err;
    return launch(p, sm_count, s);
}

}  // namespace ptk
