// FP32 evaluation of the HDR neural image field (Section 3.2) on CUDA
// cores: the accuracy reference path of the renderer.
//
// One persistent CTA of 128 threads per SM walks tiles of queries (128 rows;
// 64 for networks wider than 128).  Activations live in shared memory as
// [feature][row]; each layer's transposed weights are staged into shared
// memory (in four K-chunks when 256 wide) and multiplied with a register
// tile of 4 rows x 32 outputs per thread.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace ptk {

namespace {

constexpr int kThreads = 128;

// Tile shape for a padded width D (128, or 256 for H = 256): R rows per
// tile, weights staged KC rows of K at a time (all of a 128-wide layer; a
// quarter of a 256-wide one), each thread owning 4 rows x 32 outputs.
template <int D>
struct Fp32Tile {
    static constexpr int R = D == 128 ? 128 : 64;
    static constexpr int KC = D == 128 ? 128 : 64;
    static constexpr int RG4 = R / 16;   // row groups per warp
    static constexpr size_t smem_bytes = ((size_t)KC * D + (size_t)D * R) * sizeof(float);
    static_assert((R / 4) * (D / 32) == kThreads, "one 4 x 32 block per thread");
};

template <int D>
__device__ __forceinline__ void stage_weights(float* Ws, const float* __restrict__ Wt)
{
    const float4* src = reinterpret_cast<const float4*>(Wt);
    float4* dst = reinterpret_cast<float4*>(Ws);
#pragma unroll 4
    for (int i = threadIdx.x; i < Fp32Tile<D>::KC * D / 4; i += kThreads) dst[i] = __ldg(&src[i]);
}

template <int D>
__global__ void __launch_bounds__(kThreads, 1) k_nif_fp32(const NifEvalParams p, int mode)
{
    using T = Fp32Tile<D>;
    constexpr int R = T::R, KC = T::KC;
    extern __shared__ float4 smem4[];
    float* Ws = reinterpret_cast<float*>(smem4);       // [k][j], KC rows of the current layer
    float* hs = Ws + KC * D;                            // [k][row]
    const DevNif& nf = p.nif;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = warp * T::RG4 + (lane % T::RG4);   // rows 4 rg .. 4 rg + 3
    const int og = lane / T::RG4;                      // outputs 32 og .. 32 og + 31
    const bool row_thread = tid < R;                   // threads that own a row for features and the head
    const int64_t count = mode == 0 ? p.n : (int64_t)min(*p.esc_count, p.esc_cap);
    const int64_t n_tiles = (count + R - 1) / R;

    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // ---- features of row `tid` ----
        const int64_t g = tile * R + tid;
        const bool valid = row_thread && g < count;
        float u = 0.f, v = 0.f, tr = 0.f, tg = 0.f, tb = 0.f;
        uint32_t slot = 0;
        if (valid) {
            if (mode == 0) {
                const float2 uv = reinterpret_cast<const float2*>(p.uv)[g];
                u = uv.x; v = uv.y;
            } else {
                const float2 uv = p.esc.uv[g];
                const float4 tp = p.esc.tp[g];
                slot = __float_as_uint(tp.w); u = uv.x; v = uv.y; tr = tp.x; tg = tp.y; tb = tp.z;
            }
        }
        if (row_thread) {
            for (int i = 0; i < nf.F; ++i) {
                float s, c;
                fourier_feature(__ldg(&nf.B[2 * i]), __ldg(&nf.B[2 * i + 1]), u, v, s, c);
                hs[i * R + tid] = s;
                hs[(nf.F + i) * R + tid] = c;
            }
            for (int i = 2 * nf.F; i < D; ++i) hs[i * R + tid] = 0.f;
        }

        for (int l = 0; l < nf.L; ++l) {
            float acc[4][32];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[r][j] = 0.f;
            for (int kc = 0; kc < D; kc += KC) {
                stage_weights<D>(Ws, nf.Wt + (size_t)l * D * D + (size_t)kc * D);
                __syncthreads();   // the chunk is staged and hs holds the layer's input
#pragma unroll 2
                for (int k = 0; k < KC; ++k) {
                    const float4 h = *reinterpret_cast<const float4*>(&hs[(kc + k) * R + 4 * rg]);
                    const float4* wrow = reinterpret_cast<const float4*>(&Ws[k * D + 32 * og]);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 w = wrow[q];
                        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            acc[0][4 * q + e] = fmaf(wv[e], h.x, acc[0][4 * q + e]);
                            acc[1][4 * q + e] = fmaf(wv[e], h.y, acc[1][4 * q + e]);
                            acc[2][4 * q + e] = fmaf(wv[e], h.z, acc[2][4 * q + e]);
                            acc[3][4 * q + e] = fmaf(wv[e], h.w, acc[3][4 * q + e]);
                        }
                    }
                }
                __syncthreads();  // every thread is done reading hs and this chunk of Ws
            }
            const float* bias = nf.bias + l * D;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float bj = __ldg(&bias[32 * og + j]);
                float4 o;
                o.x = fmaxf(acc[0][j] + bj, 0.f);
                o.y = fmaxf(acc[1][j] + bj, 0.f);
                o.z = fmaxf(acc[2][j] + bj, 0.f);
                o.w = fmaxf(acc[3][j] + bj, 0.f);
                *reinterpret_cast<float4*>(&hs[(32 * og + j) * R + 4 * rg]) = o;
            }
            if (nf.skip > 0 && l == nf.skip - 1) {
                __syncthreads();   // the padded outputs of other threads are written before the features
                // the skip layer's H - 2F outputs are followed by the Fourier features (Section 3.2)
                const int base = nf.H - 2 * nf.F;
                if (row_thread) {
                    for (int i = 0; i < nf.F; ++i) {
                        float sv, cv;
                        fourier_feature(__ldg(&nf.B[2 * i]), __ldg(&nf.B[2 * i + 1]), u, v, sv, cv);
                        hs[(base + i) * R + tid] = sv;
                        hs[(base + nf.F + i) * R + tid] = cv;
                    }
                }
            }
        }
        __syncthreads();   // the last layer's outputs are in hs

        // ---- output layer, colour matrix, exp (row `tid`) ----
        if (row_thread) {
            float y0 = __ldg(&nf.bout[0]), y1 = __ldg(&nf.bout[1]), y2 = __ldg(&nf.bout[2]);
            for (int k = 0; k < nf.H; ++k) {
                const float h = hs[k * R + tid];
                y0 = fmaf(__ldg(&nf.Wout[k]), h, y0);
                y1 = fmaf(__ldg(&nf.Wout[D + k]), h, y1);
                y2 = fmaf(__ldg(&nf.Wout[2 * D + k]), h, y2);
            }
            const float z0 = nf.M[0] * y0 + nf.M[1] * y1 + nf.M[2] * y2;
            const float z1 = nf.M[3] * y0 + nf.M[4] * y1 + nf.M[5] * y2;
            const float z2 = nf.M[6] * y0 + nf.M[7] * y1 + nf.M[8] * y2;
            const float r0 = expf(z0), r1 = expf(z1), r2 = expf(z2);
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
        __syncthreads();  // hs is overwritten by the next tile's features
    }
    if (mode == 1 && blockIdx.x == 0 && threadIdx.x == 0 && p.stats) atomicAdd(p.stats, (unsigned long long)count);
}

template <int D>
cudaError_t launch_d(const NifEvalParams& p, int mode, int sm_count, cudaStream_t s)
{
    constexpr size_t smem = Fp32Tile<D>::smem_bytes;
    cudaError_t e = cudaFuncSetAttribute(k_nif_fp32<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_nif_fp32<D><<<sm_count, kThreads, smem, s>>>(p, mode); count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_nif_fp32(const NifEvalParams& p, int mode, int sm_count, cudaStream_t s)
{
    return p.nif.D == 256 ? launch_d<256>(p, mode, sm_count, s) : launch_d<128>(p, mode, sm_count, s);
}

}  // namespace ptk

namespace ptk {
namespace {
// Flat master weights -> packed FP32 layout of k_nif_fp32 (D = 128, or 256
// for H > 128): [L][D][D] transposed hidden weights, [L][D] biases, [3][D]
// output weights, [3] output bias, [2F] frequencies (zero padding elsewhere,
// also beyond the skip layer's H - 2F outputs).
__global__ void k_repack_fp32(const float* __restrict__ params, int F, int H, int L, int skip, int D,
                              float* __restrict__ packed)
{
    float* Wt = packed;
    float* bias = Wt + (size_t)L * D * D;
    float* Wout = bias + (size_t)L * D;
    float* bout = Wout + 3 * D;
    float* Bc = bout + 3;
    // offset of linear layer l's weights in the flat layout
    auto layer_off = [&](int l) {
        size_t off = 2 * (size_t)F;
        for (int q = 0; q < l; ++q) {
            int in, out;
            nif_layer_dims(F, H, L, skip, q, &in, &out);
            off += (size_t)in * out + out;
        }
        return off;
    };
    const size_t DD = (size_t)D * D;
    const size_t total = (size_t)L * DD + (size_t)L * D + 3 * (size_t)D + 3 + 2 * F;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        float val = 0.f;
        if (idx < (size_t)L * DD) {
            const int l = (int)(idx / DD), k = (int)((idx / D) % D), j = (int)(idx % D);
            int in, out;
            nif_layer_dims(F, H, L, skip, l, &in, &out);
            if (j < out && k < in) val = params[layer_off(l) + (size_t)j * in + k];
            Wt[idx] = val;
        } else if (idx < (size_t)L * DD + (size_t)L * D) {
            const size_t r = idx - (size_t)L * DD;
            const int l = (int)(r / D), j = (int)(r % D);
            int in, out;
            nif_layer_dims(F, H, L, skip, l, &in, &out);
            if (j < out) val = params[layer_off(l) + (size_t)in * out + j];
            bias[r] = val;
        } else {
            const size_t off = layer_off(L);
            const size_t r = idx - (size_t)L * DD - (size_t)L * D;
            if (r < 3 * (size_t)D) {
                const int c = (int)(r / D), k = (int)(r % D);
                if (k < H) val = params[off + (size_t)c * H + k];
                Wout[r] = val;
            } else if (r < 3 * (size_t)D + 3) {
                bout[r - 3 * D] = params[off + 3 * (size_t)H + (r - 3 * D)];
            } else {
                Bc[r - 3 * D - 3] = params[r - 3 * D - 3];
            }
        }
    }
}
}  // namespace

cudaError_t repack_nif_fp32(const float* params, int F, int H, int L, int skip, float* packed, cudaStream_t s)
{
    k_repack_fp32<<<256, 256, 0, s>>>(params, F, H, L, skip, nif_fp32_width(H), packed); count_launch();
    return cudaGetLastError();
}
}  // namespace ptk
