#include "lr_fused.cuh"

namespace lr {

bool fused_plan(const std::vector<TrajDev>&, lr_precision, FusedPlan* plan) {
  *plan = FusedPlan{};
  return false;
}
size_t fused_scratch_bytes(const FusedPlan&, int) { return 0; }
cudaError_t fused_integrate(const FusedPlan&, const DevPtrs&, const RunParams&, lr_precision, long, long,
                            cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace lr
