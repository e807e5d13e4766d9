// tcgen05 / mbarrier helpers shared by the fused kernels, and the constants of
// the Gram matrix on the tensor cores (exact bf16 slices).
#pragma once

#include <stdint.h>

namespace lr {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | (uint64_t)((lbo >> 4) & 0x3FFF) << 16 |
         (uint64_t)((sbo >> 4) & 0x3FFF) << 32 | (uint64_t)1 << 46;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Gram matrix on the tensor cores (Mp = 20, at most 1024 rows per accumulation
// window). G = A^T A for A = [Re Z | Im Z] (rows x 40 reals) is formed
// exactly enough to be FP64-class from bf16 MMAs, by slicing (the error-free
// splitting of the Ozaki scheme): every column a is scaled by a power of two
// 2^-e_a with 2^e_a above its largest entry and cut into GS_N integer slices
// of 7 bits, x = sum_s k_s 2^(-7(s+1)), |k_0| <= 128, |k_s| <= 64 (round to
// nearest at each cut, the remainders exact in FP32). A k is exact in bf16,
// a product k_s k_t (< 2^14) exact in FP32, and a sum of at most 1024 of them
// stays below 2^24 units, so the FP32 accumulation of an MMA chain is exact.
// The slice pairs (s, t) with s + t <= 8 are added in double-word with their
// weights 2^(-7(s+t)); the dropped pairs and the cut after GS_N slices leave
// an error below ~2^-50 of |z_a| |z_b| over 1000 rows.
// Slice tile of a 128-row chunk: K-major bf16 core matrices (8 m-rows x 16
// bytes), m = 40 s + a (320 rows), m-groups 128 bytes apart, k-groups (8 Z
// rows) 320 x 16 bytes apart.
constexpr int GS_N = 8;                              // slices per value
constexpr int GS_CH = 32;                            // Z rows per chunk (two MMA K steps of 16)
constexpr int GS_MR = 40 * GS_N;                     // m-rows of a slice tile
constexpr int GS_LBO = GS_MR * 16;                   // bytes between k-groups
constexpr int GS_BUF = (GS_CH / 8) * GS_LBO;         // bytes of one chunk buffer (20480; two of them:
                                                     // the kernel keeps most of L1 for the stage rows)
constexpr int GS_MAXR = 1024;                        // rows per CTA whose sums stay exact
// TMEM columns of the three accumulators: D0 = slices 0-2 x 0-5 (N 240),
// D1 = slices 0-2 x 6-7 (N 80), D2 = slices 3-5 x 3-5 (N 128; 120 used)
constexpr int GS_D0 = 0, GS_D1 = 256, GS_D2 = 384;
__device__ __forceinline__ uint32_t gs_idesc(int n) {   // kind::f16, bf16 x bf16 -> f32, M = 128, K-major
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void gs_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// wait (at most `budget` SM cycles; ~1 s at the default) for the phase with
// the given parity; false on timeout
constexpr long long WAIT_BUDGET = 2000000000LL;
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long budget = WAIT_BUDGET) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}

}  // namespace lr
