// Fault-path self-test of the device-side timeout: one warp waits, with the
// bounded mbarrier wait of the tensor-core kernels (mbarrier.cuh), on a
// barrier that nothing ever arrives on.  The wait runs out after its limit,
// the warp records a timeout code in the context's status word and the kernel
// returns, so the context stays usable.  Nothing here faults or hangs a GPU.
#include "mbarrier.cuh"
#include "rt_internal.h"

namespace rtk {

namespace {

__global__ void __launch_bounds__(32) wait_never_kernel(uint32_t* status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // Phase 0 of a barrier expecting one arrival, with no arrival: never completes.
  const bool done = mbar_wait(b, 0u, limit_ns);
  if (!done && threadIdx.x == 0) atomicOr(status, kStatusTimeout | kWhereSelftest);
}

}  // namespace

cudaError_t launch_wait_never(uint32_t* status, uint64_t limit_ns, cudaStream_t s) {
  wait_never_kernel<<<1, 32, 0, s>>>(status, limit_ns);
  return cudaGetLastError();
}

}  // namespace rtk
