// TF32x3 tensor-core stages (tcgen05) of the SGL transform.
#include <cuda_runtime.h>

#include "sgl_internal.h"

namespace sgl {

cudaError_t tc_prepare(Plan& P) {
  (void)P;
  return cudaErrorNotSupported;
}

void tc_release(Plan& P) { (void)P; }

int tc_launches(const Plan& P) {
  (void)P;
  return 4;
}

cudaError_t run_tc_stage(Plan& P, int prob, const void* x, void* y, int weighted, cudaStream_t s) {
  (void)P; (void)prob; (void)x; (void)y; (void)weighted; (void)s;
  return cudaErrorNotSupported;
}

}  // namespace sgl
