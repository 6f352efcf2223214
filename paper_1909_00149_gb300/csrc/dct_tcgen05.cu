// Placeholder: tensor-core (tcgen05) split-BF16 DCT GEMMs.
#include <cuda_runtime.h>

#include "../../include/otprox.h"
#include "otprox_internal.cuh"

namespace otp {
struct DctPlan;
int dct_tc_create(DctPlan*) { return fail(OT_EINVAL, "split-BF16 precision is not available yet"); }
void dct_tc_destroy(DctPlan*) {}
cudaError_t dct_tc_solve(DctPlan*, const float*, long long, float*, long long, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace otp
