// Self-test of the failure path of the device waits: one CTA waits, with the
// same bounded mbarrier wait the tensor-core kernels use, on a barrier that
// nothing ever arrives on.  The wait gives up after its budget, sets
// PT_ERR_TIMEOUT in the error word and the kernel returns normally, so the
// host sees the status at its next check and the context stays usable.  No
// trap, fault or unbounded loop is involved.
#include <cstdint>

#include <cuda_runtime.h>

#include "tc_ptx.cuh"

namespace ptk {

namespace {

__global__ void k_wait_selftest(uint32_t* err, uint64_t budget_ns, uint64_t* waited_ns)
{
    __shared__ uint64_t bar;
    __shared__ int abort;
    const uint32_t b = tc::smem_u32(&bar);
    if (threadIdx.x == 0) {
        tc::mbar_init(b, 1);
        abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint64_t t0 = tc::global_ns();
    const bool got = tc::mbar_wait_budget(b, 0, (volatile int*)&abort, err, budget_ns);   // nothing arrives
    __syncthreads();
    if (threadIdx.x == 0) *waited_ns = got ? 0ull : tc::global_ns() - t0;
}

}  // namespace

cudaError_t wait_selftest(uint32_t* err, uint64_t budget_ns, uint64_t* d_waited_ns, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(err, budget_ns, d_waited_ns); count_launch();
    return cudaGetLastError();
}

}  // namespace ptk
