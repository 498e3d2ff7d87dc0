// Self-test of the failure detection of the tensor-core kernels: every wait
// of those kernels on an mbarrier is bounded, and a wait that gives up sets
// the plan's error flag and lets the kernel end.  This kernel waits on a
// barrier that nothing completes, with a short bound, the same way.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sgl_internal.h"
#include "tc_ptx.cuh"

namespace sgl {
namespace {

__global__ void wait_selftest_kernel(int* flag, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tcx::mbar_init(&bar, 1);  // one arrival expected; none comes
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tcx::mbar_wait(&bar, 0, (volatile int*)&abort_flag, limit_ns)) atomicExch(flag, 1);
}

}  // namespace
}  // namespace sgl

extern "C" sgl_status sgl_selftest_wait(int64_t limit_ns, int* gave_up) {
  if (!gave_up || limit_ns <= 0 || limit_ns > 2000000000LL) return SGL_ERR_ARG;
  *gave_up = 0;
  int* d_flag = nullptr;
  if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess) return SGL_ERR_ALLOC;
  cudaError_t e = cudaMemset(d_flag, 0, sizeof(int));
  if (e == cudaSuccess) {
    sgl::wait_selftest_kernel<<<1, 32>>>(d_flag, (uint64_t)limit_ns);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(gave_up, d_flag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_flag);
  return e == cudaSuccess ? SGL_OK : SGL_ERR_CUDA;
}
