// Measurement helpers: the FP32 fused multiply-add rate of the device, the
// denominator of the traversal roofline (its slab, sphere, quad and triangle
// tests are FP32 arithmetic; each thread runs kChains independent FMA
// chains, enough to cover the FMA pipe's latency at full occupancy), and the
// L2 read bandwidth, the denominator of the large tree's L2 traffic (a
// buffer that fits L2 read again and again with loads that skip L1).
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

// XOR of every 16-byte word of buf, reps times over, grid-stride; L1 is bypassed (ld.global.cg) so that the
// reads after the first pass are served by L2
__global__ void __launch_bounds__(kBlock) k_l2_read(const uint4* __restrict__ buf, int64_t n_vec, int reps,
                                                    uint32_t* __restrict__ sink)
{
    uint32_t acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_vec; i += stride) {
            const uint4 v = __ldcg(&buf[i]);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    if (acc == 0x9E3779B9u && threadIdx.x == blockDim.x) sink[0] = acc;   // never true; keeps the loads live
}

}  // namespace
}  // namespace ptk

using namespace ptk;

extern "C" PT_API pt_status pt_microbench_l2_read(const void* d_buf, int64_t bytes, int32_t reps, uint32_t* d_sink,
                                                   double* bytes_read, void* stream)
{
    if (!d_buf || bytes < 16 || reps < 1 || !d_sink || !bytes_read || ((uintptr_t)d_buf & 15)) return PT_EINVAL;
    int device = 0, sm_count = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return PT_ECUDA;
    const int64_t n_vec = bytes / 16;
    k_l2_read<<<sm_count * kBlocksPerSM, kBlock, 0, (cudaStream_t)stream>>>((const uint4*)d_buf, n_vec, reps, d_sink);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return PT_ECUDA;
    *bytes_read = 16.0 * (double)n_vec * (double)reps;
    return PT_OK;
}

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
