// FUSED engine: the instantiations for the frame rotating at w_d with the
// rotating-wave approximation (FRAME = 1), compiled in a translation unit of
// their own so that the two frames build in parallel.
#include "lr_fused_kernel.cuh"

namespace lr {
namespace fz {

const void* rwa_kernel_ptr(lr_precision prec, int zs_smem) {
  if (zs_smem) {
    if (prec == LR_PREC_FP64) return (const void*)fused_kernel<double2, 0, 1, 0, 1>;
    if (prec == LR_PREC_FP32) return (const void*)fused_kernel<float2, 0, 1, 0, 1>;
    return (const void*)fused_kernel<float2, 1, 1, 0, 1>;
  }
  if (prec == LR_PREC_FP64) return (const void*)fused_kernel<double2, 0, 0, 0, 1>;
  if (prec == LR_PREC_FP32) return (const void*)fused_kernel<float2, 0, 0, 0, 1>;
  return (const void*)fused_kernel<float2, 1, 0, 0, 1>;
}

cudaError_t rwa_launch(const cudaLaunchConfig_t& cfg, lr_precision prec, int zs_smem, const Args& a) {
  if (zs_smem) {
    if (prec == LR_PREC_FP64) return cudaLaunchKernelEx(&cfg, fused_kernel<double2, 0, 1, 0, 1>, a);
    if (prec == LR_PREC_FP32) return cudaLaunchKernelEx(&cfg, fused_kernel<float2, 0, 1, 0, 1>, a);
    return cudaLaunchKernelEx(&cfg, fused_kernel<float2, 1, 1, 0, 1>, a);
  }
  if (prec == LR_PREC_FP64) return cudaLaunchKernelEx(&cfg, fused_kernel<double2, 0, 0, 0, 1>, a);
  if (prec == LR_PREC_FP32) return cudaLaunchKernelEx(&cfg, fused_kernel<float2, 0, 0, 0, 1>, a);
  return cudaLaunchKernelEx(&cfg, fused_kernel<float2, 1, 0, 0, 1>, a);
}

}  // namespace fz
}  // namespace lr
