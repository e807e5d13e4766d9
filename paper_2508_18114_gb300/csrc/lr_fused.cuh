// FUSED engine: one persistent launch per integrate call.
#pragma once

#include <vector>

#include "lr_internal.cuh"

namespace lr {

struct FusedPlan {
  int team;        // CTAs per trajectory
  int threads;     // threads per CTA
  int smem;        // dynamic shared memory per CTA (bytes)
  int ok;
};

// Decide whether the fused engine supports this batch and with which shape.
bool fused_plan(const std::vector<TrajDev>& traj, lr_precision prec, FusedPlan* plan);
size_t fused_scratch_bytes(const FusedPlan& plan, int n_traj);
cudaError_t fused_integrate(const FusedPlan& plan, const DevPtrs& p, const RunParams& rp, lr_precision prec,
                            long step0, long n_steps, cudaStream_t s);

}  // namespace lr
