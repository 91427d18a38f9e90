// Training of the HDR neural image field (Section 3.2.1): uniform (u, v)
// samples with a bilinear sub-pixel lookup of the HDR image, log-compressed
// targets, Huber loss, backpropagation and Adam, all in hand-written CUDA.
//
// Layers are padded to 128 x 128.  Activations are kept in HBM as [sample]
// [128] FP32 rows.  With FP32 GEMMs (this file) every GEMM is a 128-row tile
// times a 128 x 128 matrix staged in shared memory with a 4 x 32 register
// tile per thread; with BF16 GEMMs the forward, input-gradient and weight-
// gradient GEMMs run on the tensor cores (train_tc.cu) and only the output
// layer, the loss, the partial sums and Adam run here.  Either way weight
// gradients are split over the batch into one partial per CTA and summed in
// a fixed order, so a training step is deterministic.  The loss is summed in
// FP64.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "device_common.cuh"

namespace ptk {

namespace {

constexpr int kT = 128;           // rows per tile == threads per CTA
constexpr int kD = 128;           // padded width
constexpr size_t kGemmSmem = 2 * kD * kD * sizeof(float);

// Output tiles of MT rows x NT columns computed by the 128 threads of a CTA:
// MT / 4 row groups of 4 rows, the remaining thread index picks a group of
// NT / (128 / (MT / 4)) columns.  Row groups are spread within a warp so that
// each operand read is a broadcast or a conflict-free float4.
template <int MT, int NT>
struct TileMap {
    static constexpr int kRG = MT / 4;             // row groups
    static constexpr int kOG = kT / kRG;           // column groups
    static constexpr int kC = NT / kOG;            // columns per thread
    static_assert(kC % 4 == 0 && kRG % 4 == 0, "tile shape");
    int rg, og;
    __device__ TileMap()
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        rg = warp * (kRG / 4) + (lane % (kRG / 4));
        og = lane / (kRG / 4);
    }
};

// acc[r][c] += sum_{k < K} As[k][4 rg + r] * Bs[k][kC og + c]  (As: [k][MT], Bs: [k][NT])
template <int MT, int NT>
__device__ __forceinline__ void tile_mma(const float* As, const float* Bs, int K, const TileMap<MT, NT>& m,
                                         float (&acc)[4][TileMap<MT, NT>::kC])
{
    constexpr int C = TileMap<MT, NT>::kC;
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
        const float4 a = *reinterpret_cast<const float4*>(&As[k * MT + 4 * m.rg]);
        const float4* brow = reinterpret_cast<const float4*>(&Bs[k * NT + C * m.og]);
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
            const float4 b = brow[q];
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                acc[0][4 * q + e] = fmaf(a.x, bv[e], acc[0][4 * q + e]);
                acc[1][4 * q + e] = fmaf(a.y, bv[e], acc[1][4 * q + e]);
                acc[2][4 * q + e] = fmaf(a.z, bv[e], acc[2][4 * q + e]);
                acc[3][4 * q + e] = fmaf(a.w, bv[e], acc[3][4 * q + e]);
            }
        }
    }
}

// columns [0, K) of rows [tile*128, tile*128+128) of a [B][128] matrix -> smem [k][row] (zeros past B)
__device__ __forceinline__ void load_rows_transposed(float* S, const float* __restrict__ X, int64_t tile, int64_t B,
                                                     int K, int stride = kT)
{
    const int r = threadIdx.x;
    const int64_t g = tile * kT + r;
    const float4* src = reinterpret_cast<const float4*>(X + g * kD);
#pragma unroll 4
    for (int q = 0; q < K / 4; ++q) {
        const float4 v = g < B ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        S[(4 * q + 0) * stride + r] = v.x;
        S[(4 * q + 1) * stride + r] = v.y;
        S[(4 * q + 2) * stride + r] = v.z;
        S[(4 * q + 3) * stride + r] = v.w;
    }
}

// padded width (64 or 128) of a layer dimension
__host__ __device__ inline int pad_width(int n) { return n <= 64 ? 64 : 128; }
// reduction length rounded up to a multiple of 4 (the float4 row loads)
__host__ __device__ inline int pad_k(int n) { return (n + 3) & ~3; }

// ---------------------------------------------------------------------------
// training inputs: Philox key (seed, 1), counter (i, step, 0, 0) -> (u, v);
// bilinear lookup (u wraps, v clamps, pixel centres at (i + 0.5) / w) and
// target = log(max(rgb, 1e-6))
__global__ void k_train_inputs(uint32_t seed, uint32_t step, int64_t B, const float* __restrict__ sky, int w, int h,
                               float* __restrict__ uv, float* __restrict__ target)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 wd = philox4x32_10(make_uint4((uint32_t)i, step, 0u, 0u), seed, 1u);
        const float u = u01(wd.x), v = u01(wd.y);
        uv[2 * i] = u;
        uv[2 * i + 1] = v;
        const float x = u * (float)w - 0.5f, y = v * (float)h - 0.5f;
        const float x0 = floorf(x), y0 = floorf(y);
        const float fx = x - x0, fy = y - y0;
        int ix0 = (int)x0, iy0 = (int)y0;
        const int xa = ((ix0 % w) + w) % w, xb = (((ix0 + 1) % w) + w) % w;
        const int ya = min(max(iy0, 0), h - 1), yb = min(max(iy0 + 1, 0), h - 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float p00 = sky[((size_t)ya * w + xa) * 3 + c], p10 = sky[((size_t)ya * w + xb) * 3 + c];
            const float p01 = sky[((size_t)yb * w + xa) * 3 + c], p11 = sky[((size_t)yb * w + xb) * 3 + c];
            const float val = (1.f - fy) * ((1.f - fx) * p00 + fx * p10) + fy * ((1.f - fx) * p01 + fx * p11);
            target[3 * i + c] = logf(fmaxf(val, 1e-6f));
        }
    }
}

// X0[i] = [sin 2 pi (B uv_i), cos 2 pi (B uv_i)] padded to 128; one thread per (sample, frequency)
__global__ void k_train_features(int64_t B, const float* __restrict__ uv, const float* __restrict__ Bm, int F,
                                 float* __restrict__ X0)
{
    const int64_t n = B * F, npad = B * (kD - 2 * F);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n + npad;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < n) {
            const int64_t i = idx / F;
            const int f = (int)(idx - i * F);
            float sv, cv;
            fourier_feature(__ldg(&Bm[2 * f]), __ldg(&Bm[2 * f + 1]), uv[2 * i], uv[2 * i + 1], sv, cv);
            X0[i * kD + f] = sv;
            X0[i * kD + F + f] = cv;
        } else {
            const int64_t q = idx - n, i = q / (kD - 2 * F);
            X0[i * kD + 2 * F + (q - i * (kD - 2 * F))] = 0.f;
        }
    }
}

// Xout = relu(Xin W^T + b) for columns [0, NT); W is [out][in] row-major
// (PyTorch layout); the reduction runs over K >= in padded columns of Xin.
template <int NT>
__global__ void __launch_bounds__(kT, 1) k_layer_fwd(int64_t B, const float* __restrict__ Xin, float* __restrict__ Xout,
                                                     const float* __restrict__ W, const float* __restrict__ b, int in,
                                                     int out, int K)
{
    extern __shared__ float4 smem4[];
    float* Ws = reinterpret_cast<float*>(smem4);   // [k][j] = W[j][k]
    float* Xs = Ws + K * NT;                        // [k][row]
    for (int idx = threadIdx.x; idx < K * NT; idx += kT) {
        const int k = idx / NT, j = idx % NT;
        Ws[idx] = (j < out && k < in) ? W[(size_t)j * in + k] : 0.f;
    }
    using Map = TileMap<kT, NT>;
    constexpr int C = Map::kC;
    const Map m;
    const int64_t n_tiles = (B + kT - 1) / kT;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        __syncthreads();
        load_rows_transposed(Xs, Xin, tile, B, K);
        __syncthreads();
        float acc[4][C];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < C; ++j) acc[r][j] = 0.f;
        tile_mma<kT, NT>(Xs, Ws, K, m, acc);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t g = tile * kT + 4 * m.rg + r;
            if (g >= B) continue;
            float4* dst = reinterpret_cast<float4*>(Xout + g * kD + C * m.og);
#pragma unroll
            for (int q = 0; q < C / 4; ++q) {
                float o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = C * m.og + 4 * q + e;
                    o[e] = j < out ? fmaxf(acc[r][4 * q + e] + __ldg(&b[j]), 0.f) : 0.f;
                }
                dst[q] = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
    }
}

// dXin = (dXout W) * [Xin > 0] for columns [0, NT) of dXin; the reduction
// runs over the K >= out padded columns of dXout; W is [out][in]
template <int NT>
__global__ void __launch_bounds__(kT, 1) k_layer_bwd_dx(int64_t B, const float* __restrict__ dXout,
                                                        const float* __restrict__ Xin, float* __restrict__ dXin,
                                                        const float* __restrict__ W, int in, int out, int K)
{
    extern __shared__ float4 smem4[];
    float* Ws = reinterpret_cast<float*>(smem4);   // [j][k] = W[j][k]
    float* Ds = Ws + K * NT;                        // [j][row]
    for (int idx = threadIdx.x; idx < K * NT; idx += kT) {
        const int j = idx / NT, k = idx % NT;
        Ws[idx] = (j < out && k < in) ? W[(size_t)j * in + k] : 0.f;
    }
    using Map = TileMap<kT, NT>;
    constexpr int C = Map::kC;
    const Map m;
    const int64_t n_tiles = (B + kT - 1) / kT;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        __syncthreads();
        load_rows_transposed(Ds, dXout, tile, B, K);
        __syncthreads();
        float acc[4][C];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < C; ++j) acc[r][j] = 0.f;
        tile_mma<kT, NT>(Ds, Ws, K, m, acc);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t g = tile * kT + 4 * m.rg + r;
            if (g >= B) continue;
            const float4* xin = reinterpret_cast<const float4*>(Xin + g * kD + C * m.og);
            float4* dst = reinterpret_cast<float4*>(dXin + g * kD + C * m.og);
#pragma unroll
            for (int q = 0; q < C / 4; ++q) {
                const float4 x = xin[q];
                dst[q] = make_float4(x.x > 0.f ? acc[r][4 * q] : 0.f, x.y > 0.f ? acc[r][4 * q + 1] : 0.f,
                                     x.z > 0.f ? acc[r][4 * q + 2] : 0.f, x.w > 0.f ? acc[r][4 * q + 3] : 0.f);
            }
        }
    }
}

// per-CTA partials of dW = dXout^T Xin ([MT rows j][NT columns k]) and
// db = sum dXout over the CTA's tiles: partial[block] = [MT x NT dW] [MT db]
template <int MT, int NT>
__global__ void __launch_bounds__(kT, 1) k_layer_bwd_dw(int64_t B, const float* __restrict__ dXout,
                                                        const float* __restrict__ Xin, float* __restrict__ partial)
{
    extern __shared__ float4 smem4[];
    float* Ds = reinterpret_cast<float*>(smem4);   // [i][j] (reduction index first)
    float* Xs = Ds + kT * MT;                       // [i][k]
    using Map = TileMap<MT, NT>;
    constexpr int C = Map::kC;
    const Map m;                                    // rows of dW: j = 4 rg + r, columns k = C og + c
    float acc[4][C];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < C; ++j) acc[r][j] = 0.f;
    float db[4] = {0.f, 0.f, 0.f, 0.f};
    const int64_t n_tiles = (B + kT - 1) / kT;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        __syncthreads();
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int idx = threadIdx.x; idx < kT * MT / 4; idx += kT) {
            const int i = idx / (MT / 4), q = idx % (MT / 4);
            const int64_t g = tile * kT + i;
            reinterpret_cast<float4*>(Ds)[idx] = g < B ? reinterpret_cast<const float4*>(dXout + g * kD)[q] : z;
        }
        for (int idx = threadIdx.x; idx < kT * NT / 4; idx += kT) {
            const int i = idx / (NT / 4), q = idx % (NT / 4);
            const int64_t g = tile * kT + i;
            reinterpret_cast<float4*>(Xs)[idx] = g < B ? reinterpret_cast<const float4*>(Xin + g * kD)[q] : z;
        }
        __syncthreads();
        tile_mma<MT, NT>(Ds, Xs, kT, m, acc);
        if (m.og == 0) {
            for (int i = 0; i < kT; ++i) {
                const float4 d = *reinterpret_cast<const float4*>(&Ds[i * MT + 4 * m.rg]);
                db[0] += d.x; db[1] += d.y; db[2] += d.z; db[3] += d.w;
            }
        }
    }
    float* P = partial + (size_t)blockIdx.x * (MT * NT + MT);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float4* dst = reinterpret_cast<float4*>(P + (4 * m.rg + r) * NT + C * m.og);
#pragma unroll
        for (int q = 0; q < C / 4; ++q)
            dst[q] = make_float4(acc[r][4 * q], acc[r][4 * q + 1], acc[r][4 * q + 2], acc[r][4 * q + 3]);
    }
    if (m.og == 0)
        for (int r = 0; r < 4; ++r) P[MT * NT + 4 * m.rg + r] = db[r];
}

// Output layer and loss: dXlast = relu-masked W4^T dy, partial head
// gradients and FP64 loss partials per CTA.  head partial[block] = [3 x 128
// dW4] [3 db4].
//   mode 0 (NIF): Huber(delta) between M y and the target (log space).
//   mode 1 (radiance cache): relative L2, (y - t)^2 / (sg(y)^2 + 0.01), on
//          the linear output; rows with mask == 0 contribute nothing.
// X layout: rows of 128 floats, or (x_tiled) 128-row tiles of 128 x 128 floats
// in which 16-byte groups of 4 columns of consecutive rows are contiguous
// (element (r, c) of tile t at t * 16384 + (c >> 2) * 512 + r * 4 + (c & 3)).
__device__ __forceinline__ int64_t x_off(int64_t g, int c, bool tiled)
{
    return tiled ? (g >> 7) * (kT * kD) + (int64_t)(c >> 2) * (kT * 4) + (g & (kT - 1)) * 4 + (c & 3) : g * kD + c;
}

__global__ void __launch_bounds__(kT, 1) k_head_loss(int64_t B, const float* __restrict__ X, const float* __restrict__ target,
                                                     const float* __restrict__ W4, const float* __restrict__ b4, int H,
                                                     const float* __restrict__ Mm, float delta, float inv_n,
                                                     float* __restrict__ dX, float* __restrict__ head_partial,
                                                     double* __restrict__ loss_partial, int mode,
                                                     const int32_t* __restrict__ mask, int x_tiled)
{
    extern __shared__ float4 smem4[];
    // the tile's last hidden layer, [k][row] with a padded row pitch: read along rows (thread = row) by the
    // forward pass and along columns (thread = k) by the gradient pass, without bank conflicts either way
    float* Xs = reinterpret_cast<float*>(smem4);
    constexpr int kXs = kT + 1;
    __shared__ float dys[kT][3];
    __shared__ double lsum[kT];
    const int Kh = pad_k(H);
    float gW[3] = {0.f, 0.f, 0.f};   // this thread's column k = threadIdx.x of dW4
    float gb[3] = {0.f, 0.f, 0.f};
    double loss = 0.0;
    float M[9];
    for (int i = 0; i < 9; ++i) M[i] = mode == 0 ? Mm[i] : (i % 4 == 0 ? 1.f : 0.f);
    const int k = threadIdx.x;
    const float w0 = k < H ? __ldg(&W4[k]) : 0.f, w1 = k < H ? __ldg(&W4[H + k]) : 0.f,
                w2 = k < H ? __ldg(&W4[2 * H + k]) : 0.f;
    const int64_t n_tiles = (B + kT - 1) / kT;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        __syncthreads();   // the previous tile's readers of Xs and dys are done
        if (x_tiled) {
            const int r = threadIdx.x;
            const int64_t gr = tile * kT + r;
#pragma unroll 4
            for (int q = 0; q < Kh / 4; ++q) {
                const float4 v = gr < B ? *reinterpret_cast<const float4*>(X + x_off(gr, 4 * q, true))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
                Xs[(4 * q + 0) * kXs + r] = v.x;
                Xs[(4 * q + 1) * kXs + r] = v.y;
                Xs[(4 * q + 2) * kXs + r] = v.z;
                Xs[(4 * q + 3) * kXs + r] = v.w;
            }
        } else {
            load_rows_transposed(Xs, X, tile, B, Kh, kXs);
        }
        __syncthreads();
        // thread = row: output, loss and dL/dy
        const int64_t g = tile * kT + threadIdx.x;
        float dy[3] = {0.f, 0.f, 0.f};
        if (g < B && !(mask && !mask[g])) {
            float y[3] = {__ldg(&b4[0]), __ldg(&b4[1]), __ldg(&b4[2])};
            for (int kk = 0; kk < H; ++kk) {
                const float xv = Xs[kk * kXs + threadIdx.x];
                y[0] = fmaf(__ldg(&W4[kk]), xv, y[0]);
                y[1] = fmaf(__ldg(&W4[H + kk]), xv, y[1]);
                y[2] = fmaf(__ldg(&W4[2 * H + kk]), xv, y[2]);
            }
            float dz[3];
            for (int c = 0; c < 3; ++c) {
                const float z = M[3 * c] * y[0] + M[3 * c + 1] * y[1] + M[3 * c + 2] * y[2];
                const float r = z - target[3 * g + c];
                if (mode == 0) {
                    const float a = fabsf(r);
                    loss += a <= delta ? 0.5 * (double)r * (double)r : (double)delta * ((double)a - 0.5 * (double)delta);
                    dz[c] = (a <= delta ? r : copysignf(delta, r)) * inv_n;
                } else {
                    const float den = z * z + 0.01f;   // held constant in the gradient
                    loss += (double)r * (double)r / (double)den;
                    dz[c] = 2.f * r / den * inv_n;
                }
            }
            for (int j = 0; j < 3; ++j) dy[j] = M[j] * dz[0] + M[3 + j] * dz[1] + M[6 + j] * dz[2];
        }
        dys[threadIdx.x][0] = dy[0]; dys[threadIdx.x][1] = dy[1]; dys[threadIdx.x][2] = dy[2];
        __syncthreads();
        // thread = column k: the tile's rows of dX = relu-masked W4^T dy (coalesced) and column k of dW4,
        // in sample order
        const int rows = (int)min((int64_t)kT, B - tile * kT);
#pragma unroll 8
        for (int i = 0; i < rows; ++i) {
            const int64_t gi = tile * kT + i;
            const float xv = k < Kh ? Xs[k * kXs + i] : 0.f;   // columns >= Kh >= H enter neither dX nor the
                                                                // head gradient
            const float v = dys[i][0] * w0 + dys[i][1] * w1 + dys[i][2] * w2;
            dX[gi * kD + k] = (k < H && xv > 0.f) ? v : 0.f;
            gW[0] = fmaf(dys[i][0], xv, gW[0]);
            gW[1] = fmaf(dys[i][1], xv, gW[1]);
            gW[2] = fmaf(dys[i][2], xv, gW[2]);
            if (k < 3) gb[k] += dys[i][k];
        }
    }
    float* P = head_partial + (size_t)blockIdx.x * (3 * kD + 3);
    P[threadIdx.x] = gW[0];
    P[kD + threadIdx.x] = gW[1];
    P[2 * kD + threadIdx.x] = gW[2];
    if (threadIdx.x < 3) P[3 * kD + threadIdx.x] = gb[threadIdx.x];
    lsum[threadIdx.x] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int i = 0; i < kT; ++i) sum += lsum[i];
        loss_partial[blockIdx.x] = sum;
    }
}

// Fixed-order sum of per-CTA partials into the flat gradient layout:
// dst_W[j * in + k] for j < out, k < in, then dst_b[j].  stride/wofs/bofs
// describe the partial layout ([block][stride], W block at wofs with row
// pitch pitch, bias at bofs).
__global__ void __launch_bounds__(256) k_sum_partials(const float* __restrict__ partial, int n_blocks, int stride,
                                                      int pitch, int bofs, int in, int out, float* __restrict__ dst_W,
                                                      float* __restrict__ dst_b)
{
    // 32 elements per CTA; warp w sums the partials b = w, w + 8, ... in order, then the eight
    // running sums are combined in a fixed tree (deterministic, independent of scheduling)
    __shared__ float part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = out * in + out;
    const int idx = blockIdx.x * 32 + lane;
    int src = 0;
    float* dst = nullptr;
    if (idx < out * in) {
        const int j = idx / in, k = idx % in;
        src = j * pitch + k;
        dst = dst_W + idx;
    } else if (idx < n) {
        src = bofs + (idx - out * in);
        dst = dst_b + (idx - out * in);
    }
    float acc = 0.f;
    if (idx < n)
        for (int b = w; b < n_blocks; b += 8) acc += partial[(size_t)b * stride + src];
    part[w][lane] = acc;
    __syncthreads();
    if (w == 0 && idx < n)
        *dst = ((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane])) +
               ((part[4][lane] + part[5][lane]) + (part[6][lane] + part[7][lane]));
}

// The same fixed-order sums for several layers in one launch: job j owns the
// CTAs [first[j], first[j + 1]) and sums exactly as k_sum_partials would.
constexpr int kMaxSumJobs = 8;
struct SumJobs {
    int n_jobs;
    int first[kMaxSumJobs + 1];
    const float* partial[kMaxSumJobs];
    int n_blocks, stride;
    int pitch[kMaxSumJobs], bofs[kMaxSumJobs], in[kMaxSumJobs], out[kMaxSumJobs];
    float* dst_W[kMaxSumJobs];
    float* dst_b[kMaxSumJobs];
};

__global__ void __launch_bounds__(256) k_sum_partials_jobs(const SumJobs jobs)
{
    int j = 0;
    while (j + 1 < jobs.n_jobs && (int)blockIdx.x >= jobs.first[j + 1]) ++j;
    __shared__ float part[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int in = jobs.in[j], out = jobs.out[j];
    const int n = out * in + out;
    const int idx = ((int)blockIdx.x - jobs.first[j]) * 32 + lane;
    int src = 0;
    float* dst = nullptr;
    if (idx < out * in) {
        const int r = idx / in, k = idx % in;
        src = r * jobs.pitch[j] + k;
        dst = jobs.dst_W[j] + idx;
    } else if (idx < n) {
        src = jobs.bofs[j] + (idx - out * in);
        dst = jobs.dst_b[j] + (idx - out * in);
    }
    float acc = 0.f;
    if (idx < n)
        for (int b = w; b < jobs.n_blocks; b += 8) acc += jobs.partial[j][(size_t)b * jobs.stride + src];
    part[w][lane] = acc;
    __syncthreads();
    if (w == 0 && idx < n)
        *dst = ((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane])) +
               ((part[4][lane] + part[5][lane]) + (part[6][lane] + part[7][lane]));
}

// one warp: lane l sums partials l, l + 32, ... in order, then a fixed shuffle tree
__global__ void k_sum_loss(const double* __restrict__ partial, int n, double scale, double* __restrict__ out_d,
                           float* __restrict__ out_f)
{
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += partial[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, off);
    if (threadIdx.x != 0) return;
    s *= scale;   // mean over samples and channels
    if (out_d) *out_d = s;
    if (out_f) *out_f = (float)s;
}

// Adam (Kingma & Ba 2015) with bias-corrected moments
__global__ void k_adam(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t train_inputs(uint32_t seed, uint32_t step, int64_t B, const float* sky, int w, int h, float* uv,
                         float* target, cudaStream_t s)
{
    k_train_inputs<<<(unsigned)std::min<int64_t>((B + 255) / 256, 152 * 16), 256, 0, s>>>(seed, step, B, sky, w, h, uv,
                                                                                           target); count_launch();
    return cudaGetLastError();
}

// Loss and gradient of a batch whose layer-0 inputs are already in X[0]:
// target [B][3] -> grad (flat trainable layout) and the loss (FP64 and/or
// FP32 copies).  mode 0: NIF (Huber, colour matrix); mode 1: radiance cache
// (relative L2, rows masked by mask).
namespace {

cudaError_t set_smem(const void* fn)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
}

// CTAs of a batch launch: as many as fit on the GPU at once (occupancy of
// the instance with its shared memory), no more than the tiles or the
// partial slots
int grid_of(const TrainWork& wk, int64_t B, const void* fn, size_t smem)
{
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kT, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
    const int64_t tiles = (B + kT - 1) / kT;
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(tiles, (int64_t)per_sm * wk.sm_count),
                                                       wk.n_blocks));
}

// launches of the three GEMM kernels with tile widths chosen per layer
// (64 when the dimension fits, else 128)
void layer_fwd(const TrainWork& wk, int64_t B, const float* Xin, float* Xout, const float* W, const float* b, int in, int out,
               cudaStream_t s)
{
    const int K = pad_k(in);
    if (pad_width(out) == 64) {
        const size_t sm = (size_t)K * (64 + kT) * sizeof(float);
        const int G = grid_of(wk, B, (const void*)k_layer_fwd<64>, sm);
        k_layer_fwd<64><<<G, kT, sm, s>>>(B, Xin, Xout, W, b, in, out, K); count_launch();
    } else {
        const size_t sm = (size_t)K * (128 + kT) * sizeof(float);
        const int G = grid_of(wk, B, (const void*)k_layer_fwd<128>, sm);
        k_layer_fwd<128><<<G, kT, sm, s>>>(B, Xin, Xout, W, b, in, out, K); count_launch();
    }
}

void layer_bwd_dx(const TrainWork& wk, int64_t B, const float* dXout, const float* Xin, float* dXin, const float* W, int in, int out,
                  cudaStream_t s)
{
    const int K = pad_k(out);
    if (pad_width(in) == 64) {
        const size_t sm = (size_t)K * (64 + kT) * sizeof(float);
        const int G = grid_of(wk, B, (const void*)k_layer_bwd_dx<64>, sm);
        k_layer_bwd_dx<64><<<G, kT, sm, s>>>(B, dXout, Xin, dXin, W, in, out, K); count_launch();
    } else {
        const size_t sm = (size_t)K * (128 + kT) * sizeof(float);
        const int G = grid_of(wk, B, (const void*)k_layer_bwd_dx<128>, sm);
        k_layer_bwd_dx<128><<<G, kT, sm, s>>>(B, dXout, Xin, dXin, W, in, out, K); count_launch();
    }
}

// returns the partial layout's column pitch (NT), row count (MT) and the CTAs (partials) used
int layer_bwd_dw(const TrainWork& wk, int64_t B, const float* dXout, const float* Xin, float* partial, int in, int out,
                 int* MT, int* NT, cudaStream_t s)
{
    *MT = pad_width(out);
    *NT = pad_width(in);
    const size_t sm = (size_t)kT * (*MT + *NT) * sizeof(float);
    const void* fn = (*MT == 64 && *NT == 64) ? (const void*)k_layer_bwd_dw<64, 64>
                     : (*MT == 64)            ? (const void*)k_layer_bwd_dw<64, 128>
                     : (*NT == 64)            ? (const void*)k_layer_bwd_dw<128, 64>
                                              : (const void*)k_layer_bwd_dw<128, 128>;
    const int G = grid_of(wk, B, fn, sm);
    if (*MT == 64 && *NT == 64) k_layer_bwd_dw<64, 64><<<G, kT, sm, s>>>(B, dXout, Xin, partial);
    else if (*MT == 64) k_layer_bwd_dw<64, 128><<<G, kT, sm, s>>>(B, dXout, Xin, partial);
    else if (*NT == 64) k_layer_bwd_dw<128, 64><<<G, kT, sm, s>>>(B, dXout, Xin, partial);
    else k_layer_bwd_dw<128, 128><<<G, kT, sm, s>>>(B, dXout, Xin, partial);
    count_launch();
    return G;
}

// dst[:, d0 + c] = src[:, s0 + c] for c < n (rows [B][128])
__global__ void k_copy_columns(int64_t B, const float* __restrict__ src, int s0, float* __restrict__ dst, int d0, int n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B * n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / n;
        const int c = (int)(i - r * n);
        dst[r * kD + d0 + c] = src[r * kD + s0 + c];
    }
}

}  // namespace

namespace {

// output layer, loss and the head's gradients (both precisions); writes the
// gradient at the last hidden layer's pre-activation to dX_last
cudaError_t head_loss(const TrainNet& net, int64_t B, const float* target, float delta, int mode, const int32_t* mask,
                      TrainWork& wk, float* dX_last, double* loss_d, float* loss_f, int x_tiled, cudaStream_t s)
{
    cudaError_t e = set_smem((const void*)k_head_loss);
    if (e != cudaSuccess) return e;
    const size_t hsm = (size_t)pad_k(net.H) * (kT + 1) * sizeof(float);
    const int Gh = grid_of(wk, B, (const void*)k_head_loss, hsm);
    k_head_loss<<<Gh, kT, hsm, s>>>(B, wk.X[net.L], target, net.W[net.L], net.b[net.L], net.H, net.M, delta,
                                    1.f / (3.f * (float)B), dX_last, wk.partial, wk.loss_partial, mode, mask,
                                    x_tiled); count_launch();
    k_sum_partials<<<(3 * net.H + 3 + 31) / 32, 256, 0, s>>>(wk.partial, Gh, 3 * kD + 3, kD, 3 * kD, net.H, 3,
                                                             net.gW[net.L], net.gb[net.L]); count_launch();
    k_sum_loss<<<1, 32, 0, s>>>(wk.loss_partial, Gh, 1.0 / (3.0 * (double)B), loss_d, loss_f); count_launch();
    return cudaGetLastError();
}

// BF16 operands on the tensor cores: forward and input-gradient chains and
// the weight-gradient partials in train_tc.cu, partial sums here
cudaError_t mlp_loss_grad_tc(const TrainNet& net, int64_t B, const float* target, float delta, int mode,
                             const int32_t* mask, TrainWork& wk, double* loss_d, float* loss_f, cudaStream_t s)
{
    cudaError_t e = train_tc_forward(net, B, wk, wk.err, s);
    if (e != cudaSuccess) return e;
    e = head_loss(net, B, target, delta, mode, mask, wk, wk.dX[0], loss_d, loss_f, 1, s);
    if (e != cudaSuccess) return e;
    int Gl = 0, stride = 0, pitch[8] = {};
    e = train_tc_backward(net, B, wk, wk.err, &Gl, &stride, pitch, s);
    if (e != cudaSuccess) return e;
    // every hidden layer's partials are summed by one launch
    SumJobs jobs = {};
    if (net.L > kMaxSumJobs) return cudaErrorInvalidValue;
    jobs.n_jobs = net.L;
    jobs.n_blocks = Gl;
    jobs.stride = stride;
    int blocks = 0;
    for (int l = 0; l < net.L; ++l) {
        const int in = l == 0 ? net.in0 : net.H;
        jobs.first[l] = blocks;
        jobs.partial[l] = wk.partial + (size_t)l * Gl * stride;
        jobs.pitch[l] = pitch[l];
        jobs.bofs[l] = net.H * pitch[l];
        jobs.in[l] = in;
        jobs.out[l] = net.H;
        jobs.dst_W[l] = net.gW[l];
        jobs.dst_b[l] = net.gb[l];
        blocks += (in * net.H + net.H + 31) / 32;
    }
    jobs.first[net.L] = blocks;
    k_sum_partials_jobs<<<blocks, 256, 0, s>>>(jobs); count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_loss_grad(const TrainNet& net, int64_t B, const float* target, float delta, int mode,
                          const int32_t* mask, int precision, TrainWork& wk, double* loss_d, float* loss_f,
                          cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    if (precision == PT_BF16) return mlp_loss_grad_tc(net, B, target, delta, mode, mask, wk, loss_d, loss_f, s);
    cudaError_t e;
    for (auto fn : {(const void*)k_layer_fwd<64>, (const void*)k_layer_fwd<128>, (const void*)k_layer_bwd_dx<64>,
                    (const void*)k_layer_bwd_dx<128>, (const void*)k_layer_bwd_dw<64, 64>,
                    (const void*)k_layer_bwd_dw<64, 128>, (const void*)k_layer_bwd_dw<128, 64>,
                    (const void*)k_layer_bwd_dw<128, 128>}) {
        e = set_smem(fn);
        if (e != cudaSuccess) return e;
    }
    // forward through the hidden layers
    for (int l = 0; l < net.L; ++l) {
        layer_fwd(wk, B, wk.X[l], wk.X[l + 1], net.W[l], net.b[l], net.in[l], net.out[l], s);
        if (net.skip > 0 && l == net.skip - 1) {
            // the skip layer's outputs are followed by the Fourier features (Section 3.2)
            k_copy_columns<<<(unsigned)std::min<int64_t>((B * net.in0 + 255) / 256, 152 * 32), 256, 0, s>>>(
                B, wk.X[0], 0, wk.X[l + 1], net.out[l], net.in0); count_launch();
        }
    }
    // head + loss
    e = head_loss(net, B, target, delta, mode, mask, wk, wk.dX[0], loss_d, loss_f, 0, s);
    if (e != cudaSuccess) return e;
    // backward through the hidden layers
    int cur = 0;
    // (at the layer after the skip layer the input gradient's feature columns are computed and not used)
    for (int l = net.L - 1; l >= 0; --l) {
        const int in = net.in[l], out = net.out[l];
        int MT = 0, NT = 0;
        const int Gw = layer_bwd_dw(wk, B, wk.dX[cur], wk.X[l], wk.partial, in, out, &MT, &NT, s);
        k_sum_partials<<<(in * out + out + 31) / 32, 256, 0, s>>>(wk.partial, Gw, MT * NT + MT, NT, MT * NT, in,
                                                                  out, net.gW[l], net.gb[l]); count_launch();
        if (l > 0) {
            layer_bwd_dx(wk, B, wk.dX[cur], wk.X[l], wk.dX[cur ^ 1], net.W[l], in, out, s);
            cur ^= 1;
        }
    }
    return cudaGetLastError();
}

cudaError_t nif_loss_grad(const TrainNet& net, int64_t B, const float* uv, const float* target, float delta,
                          int precision, TrainWork& wk, double* loss_d, float* loss_f, cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    k_train_features<<<(unsigned)std::min<int64_t>((B * 64 + 255) / 256, 152 * 32), 256, 0, s>>>(B, uv, net.B, net.F,
                                                                                                 wk.X[0]); count_launch();
    return mlp_loss_grad(net, B, target, delta, 0, nullptr, precision, wk, loss_d, loss_f, s);
}

// ---------------------------------------------------------------------------
// Radiance cache (Mueller et al. 2021, cited in Section 2.1)
namespace {

// query / record rows: 16 floats = x[3], wo[3], n[3], tp[3], L[3], slot or valid (bits).
// A CTA of 128 threads encodes 32 rows into shared memory (thread = (row,
// part): parts 0-2 one axis' 2J frequency features each, part 3 wo and n)
// and writes them out as whole 512-byte rows, zero-padded to 128 columns.
constexpr int kFeatRows = 32;
__global__ void __launch_bounds__(128) k_cache_features(int64_t cap, const uint32_t* __restrict__ n_dev,
                                                        const float* __restrict__ rows, CacheBox box,
                                                        float* __restrict__ X0)
{
    __shared__ float4 tile4[kFeatRows * kD / 4];
    float* tile = reinterpret_cast<float*>(tile4);
    const int64_t n = n_dev ? min((int64_t)*n_dev, cap) : cap;
    const int r = threadIdx.x >> 2, part = threadIdx.x & 3;
    for (int64_t base = (int64_t)blockIdx.x * kFeatRows; base < n; base += (int64_t)gridDim.x * kFeatRows) {
        __syncthreads();   // the previous rows are written out
        for (int i = threadIdx.x; i < kFeatRows * kD / 4; i += blockDim.x) tile4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        const int64_t i = base + r;
        if (i < n) {
            const float* q = rows + 16 * i;
            float* row = tile + r * kD;
            if (part < 3) {
                cache_axis_features(q[part], box.lo[part], box.eh[part], box.el[part], box.J, row + 2 * box.J * part, 1,
                                    row + 2 * box.J * part + box.J, 1);
            } else {
                for (int t = 0; t < 6; ++t) row[6 * box.J + t] = q[3 + t];
            }
        }
        __syncthreads();
        // warp w writes rows w, w + 4, ...: one coalesced 512-byte row per step
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int rr = warp; rr < kFeatRows; rr += 4) {
            const int64_t g = base + rr;
            if (g < n && 4 * lane < kD) reinterpret_cast<float4*>(X0 + g * kD)[lane] = tile4[rr * (kD / 4) + lane];
        }
    }
}

// training targets from vertex records: (L_path - L_before) / tp, masked where the path never got there
__global__ void k_cache_targets(int64_t n, const float* __restrict__ rec, const float* __restrict__ slot_L,
                                float* __restrict__ target, int32_t* __restrict__ mask)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float* r = rec + 16 * i;
        bool ok = r[15] != 0.f;
        float t[3];
        for (int c = 0; c < 3; ++c) {
            ok = ok && r[9 + c] > 0.f;
            t[c] = ok ? (slot_L[3 * i + c] - r[12 + c]) / r[9 + c] : 0.f;
        }
        mask[i] = ok ? 1 : 0;
        for (int c = 0; c < 3; ++c) target[3 * i + c] = ok ? t[c] : 0.f;
    }
}

// training pixels of a frame: Philox key (seed, 2), counter (i, frame, 0, 0), word 0 mod (W * H)
__global__ void k_train_pixels(uint32_t seed, uint32_t frame, int64_t n, uint32_t n_pix, int64_t* pixels)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pixels[i] = (int64_t)(philox4x32_10(make_uint4((uint32_t)i, frame, 0u, 0u), seed, 2u).x % n_pix);
}

}  // namespace

cudaError_t cache_train_inputs(int64_t n, const float* rec, const float* slot_L, CacheBox box, float* X0, float* target,
                               int32_t* mask, cudaStream_t s)
{
    const unsigned g = (unsigned)std::min<int64_t>((n + 127) / 128, 152 * 8);
    k_cache_features<<<(unsigned)std::min<int64_t>((n + kFeatRows - 1) / kFeatRows, 152 * 16), 128, 0, s>>>(
        n, nullptr, rec, box, X0); count_launch();
    if (slot_L) {
        k_cache_targets<<<g, 128, 0, s>>>(n, rec, slot_L, target, mask);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t cache_train_pixels(uint32_t seed, uint32_t frame, int64_t n, uint32_t n_pix, int64_t* pixels, cudaStream_t s)
{
    k_train_pixels<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(seed, frame, n, n_pix, pixels); count_launch();
    return cudaGetLastError();
}

cudaError_t adam_step(int64_t n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                      float c1, float c2, cudaStream_t s)
{
    k_adam<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(n, w, g, m, v, lr, b1, b2, eps, c1, c2); count_launch();
    return cudaGetLastError();
}

}  // namespace ptk
