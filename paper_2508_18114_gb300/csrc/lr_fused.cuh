// FUSED engine: one persistent launch per integrate call.
//
// A trajectory is integrated by a team of C CTAs forming one thread-block
// cluster. Rows of Z are split between the team along the resonator index
// i_r (every CTA owns all transmon and filter indices of its i_r range), so
// both jump operators (filter and transmon lowering) stay inside a CTA and
// only the resonator couplings need the neighbouring CTAs' rows, read from
// their shared memory (DSMEM). The stage input Z_s lives in shared memory
// (double-buffered) for the whole launch; Z_n and the RK4 accumulator are
// touched once per stage element-wise and stay L2-resident.
#pragma once

#include <vector>

#include "lr_internal.cuh"

namespace lr {

struct FusedPlan {
  int ok;
  int C;           // CTAs per trajectory (cluster size)
  int n_clusters;  // resident clusters (persistent grid = n_clusters * C)
  int threads;
  int smem;        // dynamic shared memory per CTA (bytes)
  int zs_smem;     // 1: stage state in shared memory, 0: in global scratch (L2)
  int tc;          // tensor-core passes of the projection term: 0 (CUDA cores), 3 or 1
  int frame;       // 0 lab frame, 1 rotating frame with the rotating-wave approximation
  int Mp;          // padded rank (multiple of 4)
  int R;           // largest rows per CTA
  int Nmax;        // largest N in the batch
  int gram_mode;   // 0 native (bulk type), 1 double-word FP32 (FP64-class), 2 on the tensor cores (FP64-class)
  int es;          // bytes per complex state element
  std::vector<int> order;   // trajectories, largest work first
};

// Decide whether the fused engine supports this batch and with which shape.
// Needs a CUDA device (occupancy queries); returns false without one.
bool fused_plan(const std::vector<TrajDev>& traj, lr_precision prec, int frame, FusedPlan* plan);
size_t fused_scratch_bytes(const FusedPlan& plan, int n_traj);
// Once the workspace is bound: upload the trajectory order to the scratch and
// raise the kernel's shared-memory limit (synchronous), so that fused_integrate
// makes no host-to-device copy and can be captured in a CUDA graph.
cudaError_t fused_prepare(const FusedPlan& plan, lr_precision prec, void* scratch, int n_traj);
cudaError_t fused_integrate(const FusedPlan& plan, const DevPtrs& p, const RunParams& rp, lr_precision prec,
                            long step0, long n_steps, cudaStream_t s);

}  // namespace lr
