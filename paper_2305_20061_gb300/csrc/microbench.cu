// Measurement helper: the FP32 fused multiply-add rate of the device, the
// denominator of the traversal roofline (its slab, sphere, quad and triangle
// tests are FP32 arithmetic).  Each thread runs kChains independent FMA
// chains, enough to cover the FMA pipe's latency at full occupancy.
#include <cuda_runtime.h>

#include "pt_internal.h"

namespace ptk {
namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;
constexpr int kBlocksPerSM = 8;   // 2048 resident threads per SM

__global__ void __launch_bounds__(kBlock) k_ffma(float* __restrict__ sink, int64_t iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.f) sink[0] = s;   // never true for the arguments used; keeps the chains live
}

}  // namespace
}  // namespace ptk

using namespace ptk;

extern "C" PT_API pt_status pt_microbench_ffma(int64_t iters, float* d_sink, double* flop, void* stream)
{
    if (iters < 1 || !d_sink || !flop) return PT_EINVAL;
    int device = 0, sm_count = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return PT_ECUDA;
    const int blocks = sm_count * kBlocksPerSM;
    // x -> 0.999999 x + 1e-7 stays finite and positive for any iteration count
    k_ffma<<<blocks, kBlock, 0, (cudaStream_t)stream>>>(d_sink, iters, 0.999999f, 1e-7f);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return PT_ECUDA;
    *flop = 2.0 * kChains * (double)iters * (double)blocks * kBlock;
    return PT_OK;
}
