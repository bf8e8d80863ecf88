// Failure-path self-test of the bounded device waits.
//
// One block whose first thread waits, through the same bounded mbarrier wait
// every pipeline of the library uses, on a barrier that nothing ever arrives
// at.  The wait runs out after `limit_ns`, sets the timeout bit in the status
// word and the kernel returns normally: the context stays usable and the host
// reads the failure as FMM_ERR_TIMEOUT.  No copy, tensor-memory allocation or
// other thread depends on the barrier.
#include "fmm_internal.h"
#include "ptx.cuh"

namespace fmm {

namespace {

__global__ void __launch_bounds__(32) wait_selftest_kernel(unsigned* status, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        // phase 0 of a fresh barrier with no arrivals never completes
        mbar_wait(smem_u32(&bar), 0u, &abort_flag, status, limit_ns);
    }
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned* status, unsigned long long limit_ns, cudaStream_t stream) {
    wait_selftest_kernel<<<1, 32, 0, stream>>>(status, limit_ns);
    return cudaGetLastError();
}

}  // namespace fmm
