// FP32 evaluation of the HDR neural image field (Section 3.2) on CUDA
// cores: the accuracy reference path of the renderer.
//
// One persistent CTA of 128 threads per SM walks 128-row tiles of queries.
// Activations live in shared memory as [feature][row]; each layer's
// transposed weights are staged into shared memory and multiplied with a
// register tile of 4 rows x 32 outputs per thread.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace ptk {

namespace {

constexpr int kRows = 128;      // rows (queries) per tile
constexpr int kDim = 128;       // padded layer width
constexpr int kThreads = 128;
constexpr size_t kSmemBytes = 2 * kDim * kDim * sizeof(float);

__device__ __forceinline__ void stage_weights(float* Ws, const float* __restrict__ Wt)
{
    const float4* src = reinterpret_cast<const float4*>(Wt);
    float4* dst = reinterpret_cast<float4*>(Ws);
#pragma unroll 4
    for (int i = threadIdx.x; i < kDim * kDim / 4; i += kThreads) dst[i] = __ldg(&src[i]);
}

__global__ void __launch_bounds__(kThreads, 1) k_nif_fp32(const NifEvalParams p, int mode)
{
    extern __shared__ float4 smem4[];
    float* Ws = reinterpret_cast<float*>(smem4);       // [k][j]
    float* hs = Ws + kDim * kDim;                       // [k][row]
    const DevNif& nf = p.nif;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = warp * 8 + (lane & 7);   // rows 4 rg .. 4 rg + 3
    const int og = lane >> 3;               // outputs 32 og .. 32 og + 31
    const int64_t count = mode == 0 ? p.n : (int64_t)min(*p.esc_count, p.esc_cap);
    const int64_t n_tiles = (count + kRows - 1) / kRows;

    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // ---- features of row `tid` ----
        const int64_t g = tile * kRows + tid;
        const bool valid = g < count;
        float u = 0.f, v = 0.f, tr = 0.f, tg = 0.f, tb = 0.f;
        uint32_t slot = 0;
        if (valid) {
            if (mode == 0) {
                const float2 uv = reinterpret_cast<const float2*>(p.uv)[g];
                u = uv.x; v = uv.y;
            } else {
                const float2* e = reinterpret_cast<const float2*>(p.esc + g);
                const float2 a = e[0], b = e[1], c = e[2];
                slot = __float_as_uint(a.x); u = a.y; v = b.x; tr = b.y; tg = c.x; tb = c.y;
            }
        }
        for (int i = 0; i < nf.F; ++i) {
            float s, c;
            fourier_feature(__ldg(&nf.B[2 * i]), __ldg(&nf.B[2 * i + 1]), u, v, s, c);
            hs[i * kRows + tid] = s;
            hs[(nf.F + i) * kRows + tid] = c;
        }
        for (int i = 2 * nf.F; i < kDim; ++i) hs[i * kRows + tid] = 0.f;
        stage_weights(Ws, nf.Wt);
        __syncthreads();

        for (int l = 0; l < nf.L; ++l) {
            float acc[4][32];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[r][j] = 0.f;
#pragma unroll 2
            for (int k = 0; k < kDim; ++k) {
                const float4 h = *reinterpret_cast<const float4*>(&hs[k * kRows + 4 * rg]);
                const float4* wrow = reinterpret_cast<const float4*>(&Ws[k * kDim + 32 * og]);
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
            __syncthreads();  // every thread is done reading hs and Ws
            const float* bias = nf.bias + l * kDim;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float bj = __ldg(&bias[32 * og + j]);
                float4 o;
                o.x = fmaxf(acc[0][j] + bj, 0.f);
                o.y = fmaxf(acc[1][j] + bj, 0.f);
                o.z = fmaxf(acc[2][j] + bj, 0.f);
                o.w = fmaxf(acc[3][j] + bj, 0.f);
                *reinterpret_cast<float4*>(&hs[(32 * og + j) * kRows + 4 * rg]) = o;
            }
            if (l + 1 < nf.L) stage_weights(Ws, nf.Wt + (size_t)(l + 1) * kDim * kDim);
            __syncthreads();
            if (nf.skip > 0 && l == nf.skip - 1) {
                // the skip layer's H - 2F outputs are followed by the Fourier features (Section 3.2)
                const int base = nf.H - 2 * nf.F;
                for (int i = 0; i < nf.F; ++i) {
                    float sv, cv;
                    fourier_feature(__ldg(&nf.B[2 * i]), __ldg(&nf.B[2 * i + 1]), u, v, sv, cv);
                    hs[(base + i) * kRows + tid] = sv;
                    hs[(base + nf.F + i) * kRows + tid] = cv;
                }
                __syncthreads();
            }
        }

        // ---- output layer, colour matrix, exp (row `tid`) ----
        float y0 = __ldg(&nf.bout[0]), y1 = __ldg(&nf.bout[1]), y2 = __ldg(&nf.bout[2]);
        for (int k = 0; k < nf.H; ++k) {
            const float h = hs[k * kRows + tid];
            y0 = fmaf(__ldg(&nf.Wout[k]), h, y0);
            y1 = fmaf(__ldg(&nf.Wout[kDim + k]), h, y1);
            y2 = fmaf(__ldg(&nf.Wout[2 * kDim + k]), h, y2);
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
        __syncthreads();  // hs is overwritten by the next tile's features
    }
    if (mode == 1 && blockIdx.x == 0 && threadIdx.x == 0 && p.stats) atomicAdd(p.stats, (unsigned long long)count);
}

}  // namespace

cudaError_t launch_nif_fp32(const NifEvalParams& p, int mode, int sm_count, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_nif_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    k_nif_fp32<<<sm_count, kThreads, kSmemBytes, s>>>(p, mode); count_launch();
    return cudaGetLastError();
}

}  // namespace ptk

namespace ptk {
namespace {
// Flat master weights -> packed FP32 layout of k_nif_fp32:
// [L][128][128] transposed hidden weights, [L][128] biases, [3][128] output
// weights, [3] output bias, [2F] frequencies (zero padding elsewhere, also
// beyond the skip layer's H - 2F outputs).
__global__ void k_repack_fp32(const float* __restrict__ params, int F, int H, int L, int skip, float* __restrict__ packed)
{
    float* Wt = packed;
    float* bias = Wt + (size_t)L * 128 * 128;
    float* Wout = bias + (size_t)L * 128;
    float* bout = Wout + 3 * 128;
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
    const size_t total = (size_t)L * 128 * 128 + (size_t)L * 128 + 3 * 128 + 3 + 2 * F;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        float val = 0.f;
        if (idx < (size_t)L * 128 * 128) {
            const int l = (int)(idx / (128 * 128)), k = (int)((idx / 128) % 128), j = (int)(idx % 128);
            int in, out;
            nif_layer_dims(F, H, L, skip, l, &in, &out);
            if (j < out && k < in) val = params[layer_off(l) + (size_t)j * in + k];
            Wt[idx] = val;
        } else if (idx < (size_t)L * 128 * 128 + (size_t)L * 128) {
            const size_t r = idx - (size_t)L * 128 * 128;
            const int l = (int)(r / 128), j = (int)(r % 128);
            int in, out;
            nif_layer_dims(F, H, L, skip, l, &in, &out);
            if (j < out) val = params[layer_off(l) + (size_t)in * out + j];
            bias[r] = val;
        } else {
            const size_t off = layer_off(L);
            const size_t r = idx - (size_t)L * 128 * 128 - (size_t)L * 128;
            if (r < 3 * 128) {
                const int c = (int)(r / 128), k = (int)(r % 128);
                if (k < H) val = params[off + (size_t)c * H + k];
                Wout[r] = val;
            } else if (r < 3 * 128 + 3) {
                bout[r - 3 * 128] = params[off + 3 * (size_t)H + (r - 3 * 128)];
            } else {
                Bc[r - 3 * 128 - 3] = params[r - 3 * 128 - 3];
            }
        }
    }
}
}  // namespace

cudaError_t repack_nif_fp32(const float* params, int F, int H, int L, int skip, float* packed, cudaStream_t s)
{
    k_repack_fp32<<<256, 256, 0, s>>>(params, F, H, L, skip, packed); count_launch();
    return cudaGetLastError();
}
}  // namespace ptk
