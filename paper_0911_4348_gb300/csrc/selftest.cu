// Self-test of the bounded device-side waits (the paper has no counterpart).
//
// Every mbarrier wait of the tensor-core kernels is bounded in wall time: on
// expiry the kernel records the timeout in a device flag and returns instead
// of hanging. This probe runs that wait helper on a barrier that the probe
// itself either releases first (the wait succeeds) or never releases (the wait
// must give up after the limit), so the give-up path can be exercised on a GPU
// without faulting or hanging it.
#include "common.cuh"
#include "tc.cuh"

namespace fedvr {
namespace {

__global__ void wait_probe_kernel(int release, unsigned long long limit_ns, int *flag) {
  __shared__ uint64_t bar;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (release && threadIdx.x == 0) tc::mbar_arrive(&bar);  // completes phase 0
  __syncwarp();
  // the same warp-collective bounded wait the tensor-core roles use
  if (!tc::warp_wait(&bar, 0, limit_ns) && lane == 0) atomicExch(flag, 1);
}

}  // namespace

cudaError_t launch_wait_probe(bool release, unsigned long long limit_ns, int *flag,
                              cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(release ? 1 : 0, limit_ns, flag);
  return cudaGetLastError();
}

}  // namespace fedvr
