// lr_measure_peak: arithmetic-pipe microbenchmarks that give the roofline
// denominators of the integrator's kernels on the GPU it runs on.
//
//  kind 0  FP32 FMA: every thread runs 8 independent FFMA chains;
//  kind 1  FP64 FMA: the same with DFMA;
//  kind 2  TF32 tensor cores: one elected thread per CTA issues back-to-back
//          tcgen05.mma.kind::tf32 (M = 128, N = 256, K = 8) into one TMEM
//          accumulator from zero operand tiles in shared memory, then waits
//          (bounded) for the commit.
// Grids are a multiple of the SM count; the time is taken with CUDA events on
// the caller's stream after one warm-up launch.
#include <cuda_runtime.h>

#include "lr_internal.cuh"

namespace lr {
namespace pk {

__device__ unsigned g_sink;   // keeps the chains alive; written only for an impossible value

template <typename T>
__global__ void __launch_bounds__(256) fma_kernel(int iters, T seed) {
  T a[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) a[u] = seed + (T)(threadIdx.x + u);
  const T m = (T)0.999999, c = (T)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = fma(a[u], m, c);
  }
  T s = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += a[u];
  if (s == (T)-12345.678) g_sink = 1u;
}

constexpr int TC_M = 128, TC_N = 256, TC_K = 8;   // one kind::tf32 MMA
constexpr int TC_COLS = 256;                      // fp32 accumulator columns
constexpr long long WAIT_BUDGET = 2000000000LL;   // ~1 s of SM clock

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// K-major, no swizzle: 8-row x 16-byte core matrices, rows 16 B apart, row
// groups 128 B apart (stride offset), K halves rows*16 B apart (leading offset)
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | (uint64_t)((lbo >> 4) & 0x3FFF) << 16 |
         (uint64_t)((sbo >> 4) & 0x3FFF) << 32 | (uint64_t)1 << 46;
}

__global__ void __launch_bounds__(128, 1) tf32_kernel(int iters, unsigned* err) {
  __shared__ __align__(128) float A[TC_M * TC_K];
  __shared__ __align__(128) float B[TC_N * TC_K];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x;
  for (int e = tid; e < TC_M * TC_K; e += blockDim.x) A[e] = 0.0f;
  for (int e = tid; e < TC_N * TC_K; e += blockDim.x) B[e] = 0.0f;
  const uint32_t mb = smem_addr(&bar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tslot)),
                 "r"(TC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  if (tid == 0) {
    // D f32 (bit 4), A and B tf32 (bits 7, 10), N >> 3 at bit 17, M >> 4 at bit 24
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);
    const uint64_t ad = desc(smem_addr(A), TC_M * 16, 128), bd = desc(smem_addr(B), TC_N * 16, 128);
    for (int i = 0; i < iters; ++i) {
      const uint32_t acc = i > 0 ? 1u : 0u;
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
    // bounded wait for the MMAs; on timeout report it and keep waiting (again
    // bounded) before the accumulator is freed
    const long long t0 = clock64();
    bool done = false;
    for (int round = 0; round < 2 && !done; ++round) {
      for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(mb), "r"(0u)
            : "memory");
        if (ok) {
          done = true;
          break;
        }
        if (clock64() - t0 > (round + 1) * WAIT_BUDGET) break;
      }
      if (!done && round == 0) atomicCAS(err, 0u, (unsigned)DEV_TIMEOUT);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
}

__device__ unsigned g_err;

}  // namespace pk
}  // namespace lr

/* See include/lr.h. */
extern "C" lr_status lr_measure_peak(int kind, double* flops_per_s, double* seconds, void* stream) {
  using namespace lr;
  if (!flops_per_s || kind < 0 || kind > 2) return LR_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LR_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LR_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LR_ERR_CUDA;
  }
  unsigned* err = nullptr;
  lr_status st = LR_OK;
  double flops = 0.0;
  float ms = 0.0f;
  if (cudaGetSymbolAddress((void**)&err, pk::g_err) != cudaSuccess) st = LR_ERR_CUDA;
  if (st == LR_OK && cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess) st = LR_ERR_CUDA;
  for (int rep = 0; rep < 2 && st == LR_OK; ++rep) {   // rep 0: warm-up
    if (cudaEventRecord(e0, s) != cudaSuccess) st = LR_ERR_CUDA;
    if (kind == 0) {
      const int blocks = sms * 8, iters = 4096;
      pk::fma_kernel<float><<<blocks, 256, 0, s>>>(iters, 1.0f);
      flops = 2.0 * blocks * 256.0 * iters * 16 * 8;
    } else if (kind == 1) {
      const int blocks = sms * 8, iters = 64;
      pk::fma_kernel<double><<<blocks, 256, 0, s>>>(iters, 1.0);
      flops = 2.0 * blocks * 256.0 * iters * 16 * 8;
    } else {
      const int blocks = sms, iters = 16384;
      pk::tf32_kernel<<<blocks, 128, 0, s>>>(iters, err);
      flops = 2.0 * blocks * (double)pk::TC_M * pk::TC_N * pk::TC_K * iters;
    }
    if (cudaGetLastError() != cudaSuccess) st = LR_ERR_CUDA;
    if (st == LR_OK && cudaEventRecord(e1, s) != cudaSuccess) st = LR_ERR_CUDA;
    if (st == LR_OK && cudaEventSynchronize(e1) != cudaSuccess) st = LR_ERR_CUDA;
    if (st == LR_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = LR_ERR_CUDA;
  }
  unsigned herr = 0;
  if (st == LR_OK && cudaMemcpy(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) st = LR_ERR_CUDA;
  if (st == LR_OK && herr != 0) st = LR_ERR_TIMEOUT;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LR_OK) return st;
  *flops_per_s = flops / (ms * 1e-3);
  if (seconds) *seconds = ms * 1e-3;
  return LR_OK;
}
