// Tensor-core (tcgen05) path: not built yet.
#include "kernels.h"

namespace tn {
bool tc_supported() { return false; }
cudaError_t launch_contract_tc(const StepArgs&, int32_t, int32_t, bool, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace tn
