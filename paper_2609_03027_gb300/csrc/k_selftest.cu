// Self-test of the bounded device waits (failure detection): one CTA that holds
// tensor memory, as the tensor-core kernels do, and waits on an mbarrier that
// nothing ever signals.  The wait runs out after the given budget, the kernel
// raises the plan's bounded-wait flag, frees its tensor memory and returns --
// the same path a tensor-core kernel takes when one of its waits runs out --
// so that epic_sync / epic_image_host can be seen to report EPIC_ERR_TIMEOUT
// and the plan to keep working afterwards.  Nothing traps or faults.
#include "epic_internal.h"
#include "tc_ptx.cuh"

namespace {

__global__ void __launch_bounds__(32, 1) k_bounded_wait_selftest(int* status, long long budget)
{
    __shared__ uint64_t never;  // initialised with one expected arrival that never comes
    __shared__ uint32_t tmem_sh;
    epic::tc::tmem_alloc(&tmem_sh, 32);
    epic::tc::tmem_relinquish();
    if (threadIdx.x == 0) {
        epic::tc::mbar_init(&never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    epic::tc::fence_before_sync();
    __syncwarp();
    epic::tc::fence_after_sync();
    const bool arrived = epic::tc::mbar_wait(&never, 0, budget);
    if (!arrived && threadIdx.x == 0) atomicExch(status, 1);
    epic::tc::fence_before_sync();
    __syncwarp();
    epic::tc::tmem_dealloc(tmem_sh, 32);
}

}  // namespace

extern "C" epic_status epic_selftest_bounded_wait(epic_plan_t p, long long budget_cycles, void* stream)
{
    if (!p) return EPIC_ERR_INVALID_ARG;
    if (budget_cycles < 1 || budget_cycles > 4000000000LL) {
        p->last_error = "selftest: budget_cycles must be in 1..4e9";
        return EPIC_ERR_INVALID_ARG;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    k_bounded_wait_selftest<<<1, 32, 0, s>>>(p->tc.status, budget_cycles);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "selftest launch");
    return EPIC_OK;
}
