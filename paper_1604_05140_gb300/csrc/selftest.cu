// Self-test of the failure detection of the tensor-core kernels: every wait
// of those kernels on an mbarrier is bounded, and a wait that gives up sets
// the plan's error flag and lets the kernel end.  This kernel waits on a
// barrier that nothing completes, with a short bound, the same way, and then
// winds down as those kernels do after an abort: it waits, bounded, for an
// asynchronous copy it had issued and for its MMA commit, and frees the
// tensor memory it holds.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sgl_internal.h"
#include "tc_ptx.cuh"

namespace sgl {
namespace {

__global__ void wait_selftest_kernel(int* flag, const int4* src, uint64_t limit_ns) {
  __shared__ uint64_t bar, copied, mma_done;
  __shared__ int abort_flag;
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(16) int4 dst;
  if (threadIdx.x == 0) {
    tcx::mbar_init(&bar, 1);  // one arrival expected; none comes
    tcx::mbar_init(&copied, 1);
    tcx::mbar_init(&mma_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  tcx::tmem_alloc(&tmem_slot, 32);  // as the tensor-core kernels hold tensor memory
  tcx::tc_before();
  __syncthreads();
  tcx::tc_after();
  if (threadIdx.x == 0) {
    // an asynchronous copy is in flight when the wait gives up, as in a
    // producer that aborts; the wind-down waits for it, and for the MMAs of
    // an issuer (none here), before tensor memory is freed
    tcx::mbar_arrive_tx(&copied, 16);
    tcx::bulk_load(&dst, src, 16, &copied);
    if (!tcx::mbar_wait(&bar, 0, (volatile int*)&abort_flag, limit_ns)) {
      const bool drained = tcx::drain_ring(&copied, 1, 1) && tcx::drain_mma(&mma_done);
      atomicExch(flag, drained ? 1 : 2);
    }
  }
  tcx::tc_before();
  __syncthreads();
  tcx::tc_after();
  tcx::tmem_dealloc(tmem_slot, 32);
}

}  // namespace
}  // namespace sgl

extern "C" sgl_status sgl_selftest_wait(int64_t limit_ns, int* gave_up) {
  if (!gave_up || limit_ns <= 0 || limit_ns > 2000000000LL) return SGL_ERR_ARG;
  *gave_up = 0;
  int* d_buf = nullptr;  // the flag, then 16 bytes the kernel copies
  if (cudaMalloc(&d_buf, 32) != cudaSuccess) return SGL_ERR_ALLOC;
  cudaError_t e = cudaMemset(d_buf, 0, 32);
  if (e == cudaSuccess) {
    sgl::wait_selftest_kernel<<<1, 32>>>(d_buf, (const int4*)(d_buf + 4), (uint64_t)limit_ns);
    e = cudaGetLastError();
  }
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, d_buf, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_buf);
  *gave_up = flag == 1;
  return e == cudaSuccess ? SGL_OK : SGL_ERR_CUDA;
}
