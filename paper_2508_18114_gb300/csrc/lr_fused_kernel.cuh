#pragma once
// FUSED engine: persistent cluster kernel integrating whole pulses.
//
// Per RK4 stage of Eq. S5, for one trajectory on a team of C CTAs:
//   P  (local)  partial sums over the CTA's rows of the stage input Z_s:
//               G = Z^dag Z (upper tiles), T_r = Z^dag r Z, T_b = Z^dag b Z
//               (+ level populations and readout photons at recording steps);
//   B1          one cluster barrier: partials and the new Z_s are visible;
//   R  (every CTA, redundantly) reduce the C partial slots in rank order,
//               G = L D L^dag, L^-1, G^-1 = L^-dag D^-1 L^-1 and X_k = G^-1 T_k
//               (FP64 for the FP64 state; double-word FP32, ~2^-48, for the FP32
//               state), pre-scaled, conjugate-transposed and rounded to the bulk
//               precision: XT_r = kappa/2 X_r^dag, XT_b = gamma/2 X_b^dag;
//   F  (local + DSMEM halo) F = -i H_eff Z_s + (rZ_s) XT_r + (bZ_s) XT_b and the
//               RK4 stage update; the next stage input goes to the other Z_s
//               buffer, the accumulator and Z_n are updated in L2.
// Partial slots and Z_s buffers are double-buffered by stage parity, so the
// single barrier per stage separates every write from the reads of it.
//
// FRAME = 1 integrates the rotating-frame RWA Hamiltonian instead (detuned
// diagonal, excitation-conserving couplings, complex drive weight); the lab
// frame (FRAME = 0) compiles without any of it.
//
// Tensor-core projection (TC > 0, stage state in L2): the projection term of F
// is a real GEMM per 128-row tile, D[l][2m+c] = sum_K A[l][K] B[2m+c][K] with
// A[l] = (s_r rZ_s[l], s_b bZ_s[l]) as interleaved (re, im) floats (K = 4 Mp)
// and B the real 2x2-block embedding of XT. It runs as tcgen05.mma kind::tf32
// with both operands in shared memory (K-major, no swizzle) and D in tensor
// memory: 3 passes (big*big + big*small + small*big of a two-term TF32 split,
// FP32-class products) or 1 pass (plain TF32).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "lr_fused.cuh"
#include "lr_tc.cuh"

namespace cg = cooperative_groups;

namespace lr {
namespace fz {

constexpr int NT = 384;       // threads of the tensor-core variants (12 warps: 4 TMEM lane groups x 3)
constexpr int NWARP = NT / 32;
constexpr int NT_CC = 512;    // threads of the CUDA-core variants (16 warps at <= 128 registers)
__host__ __device__ constexpr int threads_for(int tc) { return tc > 0 ? NT : NT_CC; }
constexpr int TAB = 64;   // mode truncations handled by the fused engine: N_t, N_r, N_f < 64

struct Args {
  DevPtrs p;
  RunParams rp;
  long step0, n_steps;
  int C, n_clusters, Mp, R, Nmax;
  int zs_smem;
  // byte offsets in dynamic shared memory
  int o_zs, o_slot, slot_bytes, s_gp, s_tp, s_pop;   // s_*: offsets inside one slot
  int o_gd, o_w, o_tred, o_trd, o_xs, o_misc, o_tab;
  int o_ta, o_tb, npad;   // tensor-core operand tiles (TC > 0), B rows (2 Mp padded to 16)
  int o_gs;               // Gram on the tensor cores (GRAM_DW == 2): two slice buffers
  const int* order;
  void* zs_glob;      // global stage buffers, per cluster [C][2][R][Mp+1]
  void* acc_glob;     // RK4 accumulator, per cluster [Nmax*Mp]
  long long debug_wait;   // > 0: test hook, a wait of this many SM cycles that must run out
};

// ----------------------------------------------------------------- complex

template <typename T2> struct Real;
template <> struct Real<float2> { using t = float; };
template <> struct Real<double2> { using t = double; };

template <typename T2> __device__ __forceinline__ T2 cm(typename Real<T2>::t r, typename Real<T2>::t i) {
  T2 v;
  v.x = r;
  v.y = i;
  return v;
}

// ----------------------------------------------------------------- partition

struct Part {
  int r_lo, nr, st, R;
};

__device__ __forceinline__ Part part_of(const TrajDev& d, int C, int q) {
  Part P;
  const int base = d.Nr / C, rem = d.Nr % C;
  P.r_lo = q * base + min(q, rem);
  P.nr = base + (q < rem ? 1 : 0);
  P.st = P.nr * d.Nf;
  P.R = d.Nt * P.st;
  return P;
}

// ----------------------------------------------------------------- double-word accumulation
// Exact FP32 products (p + e = a*b via FMA) accumulated in an unevaluated
// sum of two floats (hi + lo): ~2^-48 relative, the FP64-class Gram matrix.
struct DW {
  float hi, lo;
};
__device__ __forceinline__ void dw_add_prod(DW& s, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}
__device__ __forceinline__ void dw_add(DW& s, const DW& o) {
  const float t = s.hi + o.hi;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (o.hi - bp);
  s.hi = t;
  s.lo += err + o.lo;
}
__device__ __forceinline__ double dw_value(const DW& s) { return (double)s.hi + (double)s.lo; }
__device__ __forceinline__ void dw_add_f(DW& s, float x) {   // s += x (Knuth's two-sum into hi)
  const float t = s.hi + x;
  const float bp = t - s.hi;
  s.lo += (s.hi - (t - bp)) + (x - bp);
  s.hi = t;
}

// Double-word arithmetic for the M x M phase (Dekker's product via FMA,
// Knuth's two-sum; results normalised, ~2^-48 relative).
__device__ __forceinline__ DW dw_make(double x) {
  DW r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ DW dw_sum(DW a, DW b) {
  const float s = a.hi + b.hi, bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  DW r;
  r.hi = s + e;
  r.lo = e - (r.hi - s);
  return r;
}
__device__ __forceinline__ DW dw_neg(DW a) {
  a.hi = -a.hi;
  a.lo = -a.lo;
  return a;
}
__device__ __forceinline__ DW dw_mul(DW a, DW b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  DW r;
  r.hi = p + e;
  r.lo = e - (r.hi - p);
  return r;
}
// 1/p for p > 0: Newton's iteration r <- r + r (1 - p r) once, in double-word,
// from the FP32 quotient (24 -> ~48 bits)
__device__ __forceinline__ DW dw_recip(DW p) {
  DW r0;
  r0.hi = 1.0f / p.hi;
  r0.lo = 0.0f;
  DW one;
  one.hi = 1.0f;
  one.lo = 0.0f;
  const DW e = dw_sum(one, dw_neg(dw_mul(p, r0)));
  return dw_sum(r0, dw_mul(r0, e));
}
struct DWC {
  DW re, im;
};
// x conj(y)
__device__ __forceinline__ DWC dwc_mul_conj(const DWC& x, const DWC& y) {
  DWC r;
  r.re = dw_sum(dw_mul(x.re, y.re), dw_mul(x.im, y.im));
  r.im = dw_sum(dw_mul(x.im, y.re), dw_neg(dw_mul(x.re, y.im)));
  return r;
}
// x y
__device__ __forceinline__ DWC dwc_mul(const DWC& x, const DWC& y) {
  DWC r;
  r.re = dw_sum(dw_mul(x.re, y.re), dw_neg(dw_mul(x.im, y.im)));
  r.im = dw_sum(dw_mul(x.re, y.im), dw_mul(x.im, y.re));
  return r;
}
__device__ __forceinline__ DWC dwc_sub(const DWC& a, const DWC& b) {
  DWC r;
  r.re = dw_sum(a.re, dw_neg(b.re));
  r.im = dw_sum(a.im, dw_neg(b.im));
  return r;
}
__device__ __forceinline__ DWC dwc_add(const DWC& a, const DWC& b) {
  DWC r;
  r.re = dw_sum(a.re, b.re);
  r.im = dw_sum(a.im, b.im);
  return r;
}
__device__ __forceinline__ DWC dwc_scale(const DWC& a, DW s) {
  DWC r;
  r.re = dw_mul(a.re, s);
  r.im = dw_mul(a.im, s);
  return r;
}
// double-word times float (the float exact as a double-word with lo = 0)
__device__ __forceinline__ DW dw_mul_f(DW a, float b) {
  const float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  DW r;
  r.hi = p + e;
  r.lo = e - (r.hi - p);
  return r;
}
// g t for a double-word complex g and an FP32 complex t
__device__ __forceinline__ DWC dwc_mul_f(const DWC& g, float tx, float ty) {
  DWC r;
  r.re = dw_sum(dw_mul_f(g.re, tx), dw_neg(dw_mul_f(g.im, ty)));
  r.im = dw_sum(dw_mul_f(g.re, ty), dw_mul_f(g.im, tx));
  return r;
}

// Reduce-scatter of NV = 2^p partial sums over a warp (recursive halving): at
// offset o each lane keeps the half of its values named by bit o of its lane
// and adds the partner's copy; offsets left once a single value remains add
// across the rest of the warp. Lane L ends with the total of value
// L >> (5 - p) in v[0] (p <= 5), or of values 2L and 2L + 1 in v[0], v[1]
// (p = 6). The order of the additions is fixed.
template <int NV, typename V>
__device__ __forceinline__ void warp_reduce_scatter(V (&v)[NV], int lane) {
#pragma unroll
  for (int lev = 0; lev < 5; ++lev) {
    const int o = 16 >> lev;
    constexpr int n0 = NV;
    const int n = n0 >> lev;
    if (n >= 2) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < n / 2; ++k) {
        const V keep = up ? v[k + n / 2] : v[k];
        const V send = up ? v[k] : v[k + n / 2];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    }
  }
}

// ----------------------------------------------------------------- the kernel

// Vector load of 4 consecutive complex values (16-byte loads when the row
// stride keeps them aligned: the L2-resident layout).
template <int ZSM, typename T2>
__device__ __forceinline__ void load4(const T2* p, T2 (&v)[4]) {
  if constexpr (ZSM == 0 && sizeof(T2) == 8) {
    // FP32 stage state in global memory: one 32-byte access (rows of Mp = 4j
    // complex64 entries from a 256-byte aligned region, column quads m0 = 4i)
    float x[8];
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7])
                 : "l"(p)
                 : "memory");
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = cm<T2>(x[2 * u], x[2 * u + 1]);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = p[u];
  }
}
template <int ZSM, typename T2>
__device__ __forceinline__ void store4(T2* p, const T2 (&v)[4]) {
  if constexpr (ZSM == 0 && sizeof(T2) == 8) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0].x), "f"(v[0].y),
                 "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y), "f"(v[3].x), "f"(v[3].y)
                 : "memory");
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) p[u] = v[u];
  }
}

// ----------------------------------------------------------------- tcgen05 helpers
// Operand tiles are K-major without swizzle: 8-row x 16-byte core matrices,
// rows of a core 16 bytes apart, cores of consecutive 8-row groups 128 bytes
// apart (stride offset) and cores consecutive in K rows*16 bytes apart
// (leading offset).
constexpr int TC_ROWS = 128;   // MMA M (rows of Z_s per tile), one TMEM lane per row
constexpr int TC_ACC = 64;     // TMEM columns per accumulator (N = 2 Mp padded to 16 <= 64)
constexpr int TC_KSPLIT = 2;   // independent accumulators per pass (halves of K)
constexpr int TC_COLS = 512;   // TMEM columns allocated: up to 3 passes x TC_KSPLIT accumulators

constexpr int GS_W = 10;                             // slicing warps (warp GS_W issues the MMAs)

__device__ __forceinline__ int kmaj_off(int row, int k, int rows) {
  return (k >> 2) * (rows * 16) + (row >> 3) * 128 + (row & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

template <typename T2, int GRAM_DW, int ZSM, int TC, int FRAME, int NTH = threads_for(TC)>
__global__ void __launch_bounds__(NTH, 1) fused_kernel(const Args a) {
  constexpr int NT = NTH, NWARP = NTH / 32;
  static_assert(TC == 0 || (ZSM == 0 && sizeof(T2) == 8), "tensor-core projection: FP32 state in L2 only");
  using T = typename Real<T2>::t;
  constexpr int TP = sizeof(T) == 4 ? 4 : 2;     // phase-P tile edge
  constexpr int TR = sizeof(T) == 4 ? 5 : 2;     // phase-F rows per thread tile
  // first step of this launch: the device step counter (so that a replayed
  // capture of the launch continues the pulse run), else the argument
  const long step0 = a.p.dstep ? (long)*a.p.dstep : a.step0;
  if (step0 < 0 || step0 + a.n_steps > a.rp.max_steps) {
    // every thread of every CTA reads the same value: the whole grid leaves
    // here, before any barrier, tensor-memory allocation or write
    if (blockIdx.x == 0 && threadIdx.x == 0) set_error(a.p.err, DEV_CAPACITY);
    return;
  }
  if (GRAM_DW == 2 && (a.Mp != 20 || a.R > GS_MAXR)) {
    // the tensor-core Gram is laid out for 20 complex columns and exact for at
    // most GS_MAXR rows per CTA; the whole grid leaves before any barrier
    if (blockIdx.x == 0 && threadIdx.x == 0) set_error(a.p.err, DEV_CAPACITY);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = a.C;
  const int q = (int)cluster.block_rank();
  const int cid = blockIdx.x / C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Mp = a.Mp;
  // row stride of Z_s: odd in complex elements in shared memory, so lanes that
  // read consecutive rows hit distinct banks; 32-byte aligned rows in L2 for
  // 16-byte vector loads
  const int lds = ZSM ? Mp + 1 : Mp;
  const long long zs_buf = (long long)a.R * lds;  // elements per smem Z_s buffer

  double2* Gd = reinterpret_cast<double2*>(smem + a.o_gd);     // [Mp][Mp+1]  G -> L -> G^-1
  double2* W = reinterpret_cast<double2*>(smem + a.o_w);       // [Mp][Mp+1]  L^-1
  T2* Tred = reinterpret_cast<T2*>(smem + a.o_tred);           // [2][Mp*Mp]
  double* trd = reinterpret_cast<double*>(smem + a.o_trd);     // [Mp] diag of T_r (FP64)
  T2* XT = reinterpret_cast<T2*>(smem + a.o_xs);               // [2][Mp][Mp] (l, m)
  // misc (FP64 scalars): [0] pulse coefficient, [1] not-PD flag, [8..24) photon
  // partials per level, [32..64) Im diag T_r, [64..81) reduced populations and
  // photons, [96..128) 1/L[k][k], [128..131) bulk-precision coefficient and
  // steps, [136..140) mbarriers of the tensor-core Gram, [140] phase-P task
  // counter, [141] tensor-core timeout flag, [142] tensor-core mbarrier, [143]
  // TMEM base address, [144..164) column maxima of the tensor-core Gram
  double* misc = reinterpret_cast<double*>(smem + a.o_misc);
  if (a.debug_wait > 0) {
    // Test hook for the timeout path: thread 0 waits on an mbarrier that
    // nothing arrives on, with a budget of debug_wait cycles. The wait runs
    // out, the error word gets DEV_TIMEOUT, and the launch then carries on
    // as usual (nothing asynchronous is in flight), so the context stays usable.
    __shared__ __align__(8) unsigned long long dbg_bar;
    if (tid == 0) {
      const uint32_t mb = smem_u32(&dbg_bar);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1) : "memory");
      if (!mbar_wait(mb, 0u, a.debug_wait)) set_error(a.p.err, DEV_TIMEOUT);
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mb) : "memory");
    }
    __syncthreads();
  }
  // row-ordered lower-triangle index table: entry e = i(i+1)/2 + j -> (i, j)
  __shared__ short2 tri[LR_MAX_RANK * (LR_MAX_RANK + 1) / 2];
  for (int i = tid; i < LR_MAX_RANK; i += NT)
    for (int j = 0; j <= i; ++j) tri[i * (i + 1) / 2 + j] = make_short2((short)i, (short)j);
  T* sq = reinterpret_cast<T*>(smem + a.o_tab);                 // sqrt(k), k < TAB
  T* dtab = sq + TAB;                                           // [3][TAB][2]: diagonal energies (hi, lo)
  const int ldg = Mp + 1;

  // Stage buffers: in shared memory, or (when they do not fit) in a global
  // scratch region with the same per-CTA layout [C][2][R][lds] that stays L2
  // resident; both are addressed by local row.
  T2* zs_local = a.zs_smem ? reinterpret_cast<T2*>(smem + a.o_zs)
                           : reinterpret_cast<T2*>(a.zs_glob) + ((size_t)cid * C + q) * 2 * zs_buf;
  T2* accg = reinterpret_cast<T2*>(a.acc_glob) + (size_t)cid * a.Nmax * Mp;

  const double dt = a.rp.dt;
  const int pe = a.rp.pop_every;

  // ---- tensor-core projection: operand tiles, D staging, TMEM and its mbarrier
  float* ta_big = reinterpret_cast<float*>(smem + a.o_ta);
  float* ta_small = ta_big + TC_ROWS * 4 * Mp;
  float* tb_big = reinterpret_cast<float*>(smem + a.o_tb);
  float* tb_small = tb_big + a.npad * 4 * Mp;
  const uint32_t mbar = smem_u32(misc + 142);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 143);
  uint32_t tmem = 0, tc_phase = 0;
  // Gram on the tensor cores: one mbarrier per slice buffer, and the number
  // of completed phases of each
  const uint32_t gs_bar[2] = {smem_u32(misc + 138), smem_u32(misc + 139)};
  uint32_t gs_ph[2] = {0u, 0u};
  // ... and one per buffer on which the slicing warps arrive when a chunk is in
  // place (the issuing warp's phase counts)
  const uint32_t gs_fill[2] = {smem_u32(misc + 136), smem_u32(misc + 137)};
  uint32_t gs_fph[2] = {0u, 0u};
  // column maxima max(|Re|, |Im|) of the own rows of the stage input, as float
  // bits: [2][20] at misc[144..164), by stage parity; phase F of a stage forms
  // the next one's from the rows it writes
  uint32_t* gs_cmax = reinterpret_cast<uint32_t*>(misc + 144);
  int gs_par = 0;
  if constexpr (TC > 0 || GRAM_DW == 2) {
    // B rows beyond 2 Mp stay zero for the whole launch
    if constexpr (TC > 0)
      for (int e = tid; e < (a.npad - 2 * Mp) * 4 * Mp; e += NT) {
        const int n = 2 * Mp + e / (4 * Mp), k = e % (4 * Mp);
        tb_big[kmaj_off(n, k, a.npad) / 4] = 0.0f;
        if (TC == 3) tb_small[kmaj_off(n, k, a.npad) / 4] = 0.0f;
      }
    if (tid == 0) {
      *reinterpret_cast<int*>(misc + 141) = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1));
      if (GRAM_DW == 2) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gs_bar[0]), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gs_bar[1]), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gs_fill[0]), "r"(GS_W * 32));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gs_fill[1]), "r"(GS_W * 32));
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                   "r"(TC_COLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    async_proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem = *tslot;
  }

  for (int it_idx = cid; it_idx < a.rp.n_traj; it_idx += a.n_clusters) {
    const int tj = a.order[it_idx];
    const TrajDev d = a.p.traj[tj];
    const int M = d.M;
    // this trajectory's rank padded to 4: the extent of its tile grids and
    // column quads (storage keeps the batch-wide stride Mp; the tensor-core
    // GEMM spans all of Mp)
    const int Mq = TC > 0 ? Mp : (M + 3) / 4 * 4;
    const Part P = part_of(d, C, q);
    const Part Pm = part_of(d, C, q > 0 ? q - 1 : q);
    const Part Pp = part_of(d, C, q < C - 1 ? q + 1 : q);
    const int Nf = d.Nf, Nr = d.Nr, Nt = d.Nt;
    const bool three = d.n_modes == 3;
    const int dro = three ? Nf : Nr;
    T2* Zn = reinterpret_cast<T2*>(a.p.Zn) + d.z_off;
    const PulseDev pulse = a.p.pulse[d.cand];
    // Z_s bases of the neighbouring ranks (DSMEM or the neighbours' global regions)
    T2* zs_m = zs_local;
    T2* zs_p = zs_local;
    if (a.zs_smem) {
      zs_m = cluster.map_shared_rank(zs_local, q > 0 ? q - 1 : q);
      zs_p = cluster.map_shared_rank(zs_local, q < C - 1 ? q + 1 : q);
    } else {
      zs_m = zs_local - (q > 0 ? 2 * zs_buf : 0);
      zs_p = zs_local + (q < C - 1 ? 2 * zs_buf : 0);
    }

    // pointer to the start of row (it, ir, iff) of Z_s buffer b (any owner)
    auto zrow = [&](int b, int it2, int ir2, int iff2) -> const T2* {
      if (ir2 < P.r_lo) {
        const int l = (it2 * Pm.nr + (ir2 - Pm.r_lo)) * Nf + iff2;
        return zs_m + (size_t)b * zs_buf + (size_t)l * lds;
      }
      if (ir2 >= P.r_lo + P.nr) {
        const int l = (it2 * Pp.nr + (ir2 - Pp.r_lo)) * Nf + iff2;
        return zs_p + (size_t)b * zs_buf + (size_t)l * lds;
      }
      const int l = (it2 * P.nr + (ir2 - P.r_lo)) * Nf + iff2;
      return zs_local + (size_t)b * zs_buf + (size_t)l * lds;
    };
    // own row l of buffer b (writable)
    auto own = [&](int b, int l) -> T2* { return zs_local + (size_t)b * zs_buf + (size_t)l * lds; };
    // global row of local row l
    auto grow = [&](int l) {
      const int it = l / P.st, rem = l - it * P.st, irl = rem / Nf, iff = rem - irl * Nf;
      return (it * Nr + P.r_lo + irl) * Nf + iff;
    };

    // ---- per-trajectory tables: sqrt(k) and the separable diagonal of H,
    //      wq i_t + alpha/2 i_t(i_t-1) | wr i_r | wf i_f, each as hi + lo so that
    //      the bulk precision does not round the mode frequencies
    for (int k = tid; k < TAB; k += NT) {
      sq[k] = (T)sqrt((double)k);
      // in the rotating frame every mode frequency becomes a detuning w - w_d
      const double wfr = FRAME ? pulse_drive_frequency(pulse) : 0.0;
      const double v[3] = {(d.wq - wfr) * k + 0.5 * d.alpha * k * (k - 1.0), (d.wr - wfr) * k,
                           three ? (d.wf - wfr) * k : 0.0};
      for (int c3 = 0; c3 < 3; ++c3) {
        const T hi = (T)v[c3];
        dtab[(c3 * TAB + k) * 2] = hi;
        dtab[(c3 * TAB + k) * 2 + 1] = (T)(v[c3] - (double)hi);
      }
    }
    if (tid == 0) *reinterpret_cast<int*>(misc + 140) = 0;
    // ---- load Z_n into Z_s buffer 0 (own rows), zero the rank padding
    for (int e = tid; e < P.R * Mp; e += NT) {
      const int l = e / Mp, m = e - l * Mp;
      own(0, l)[m] = m < M ? Zn[(size_t)grow(l) * M + m] : cm<T2>(0, 0);
    }
    if constexpr (GRAM_DW == 2) {   // column maxima of the loaded rows
      if (tid < 20) gs_cmax[gs_par * 20 + tid] = 0u;
      __syncthreads();
      if (tid < 500) {
        const int j = tid % 20;
        float mx = 0.f;
        for (int l = tid / 20; l < P.R; l += 25) {
          const T2 v = own(0, l)[j];
          mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        atomicMax(gs_cmax + gs_par * 20 + j, __float_as_uint(mx));
      }
    }
    __syncthreads();

    int cur = 0;
    const long s_end = step0 + a.n_steps;
    for (long step = step0;; ++step) {
      const bool last = step == s_end;
      for (int stage = 0; stage < 4; ++stage) {
        const int par = stage & 1;
        const bool record = stage == 0 && (step % pe) == 0;
        unsigned char* slot = smem + a.o_slot + par * a.slot_bytes;
        double2* gp = reinterpret_cast<double2*>(slot + a.s_gp);
        T2* tp = reinterpret_cast<T2*>(slot + a.s_tp);
        double* popp = reinterpret_cast<double*>(slot + a.s_pop);

        // ================= P: partial sums over own rows of Z_s[cur]
        {
          const int nt_ = Mq / TP;
          const int n_g = GRAM_DW == 2 ? 0 : nt_ * (nt_ + 1) / 2, n_t = nt_ * nt_;
          // warps take tasks dynamically (heavier Gram tiles first); every task's
          // arithmetic is independent of which warp runs it, so results stay bitwise
          // reproducible
          int* task_ctr = reinterpret_cast<int*>(misc + 140);
          if (tid == NT - 1) {
            // drive coefficient of this stage (FP64 pulse shape), off the serial
            // M x M phase: read by phase F after the barriers that follow
            const double ts = (double)step * dt + (stage == 0 ? 0.0 : (stage == 3 ? dt : 0.5 * dt));
            if (FRAME) {
              // RWA drive w r + conj(w) r^dag, w = (Omega/2) e^{i phi}
              const double2 w = pulse_rwa_drive(pulse, a.rp.tau, ts);
              misc[0] = w.x;
              misc[2] = w.y;
            } else {
              misc[0] = pulse_coefficient(pulse, a.rp.tau, ts);
              misc[2] = 0.0;
            }
            T* tb = reinterpret_cast<T*>(misc + 128);
            tb[0] = (T)misc[0];
            tb[5] = (T)misc[2];
          }
          if constexpr (GRAM_DW == 2) {
            // ---- Gram on the tensor cores. GS_W warps slice the chunks of GS_CH
            // rows into the two buffers and arrive on the buffer's fill mbarrier;
            // warp GS_W waits on it and one of its threads issues the chunk's MMAs,
            // committed to the buffer's MMA mbarrier, on which the slicing warps
            // wait before they refill it. The other warps start on the T tiles
            // below, and the slicing and issuing warps join them when done.
            if (tid < 20) gs_cmax[(gs_par ^ 1) * 20 + tid] = 0u;   // phase F fills it for the next stage
            if (warp < GS_W) {
              const uint32_t* cmax = gs_cmax + gs_par * 20;
              volatile int* tc_abort = reinterpret_cast<volatile int*>(misc + 141);
              const int n_ch = (P.R + GS_CH - 1) / GS_CH;
              // warp task: rows rg*8 .. +7 of a chunk x real columns ag*8 .. +7,
              // task = warp + GS_W t; lane = (column ag*8 + lane/4, rows 2 (lane%4)
              // and +1), so that each slice is one 128-byte core-matrix store per
              // warp. The values of the next chunk are loaded while this one is
              // sliced.
              constexpr int GTASK = (GS_CH / 8) * 5;   // warp tasks per chunk
              constexpr int GT = GTASK / GS_W;         // per slicing warp
              static_assert(GTASK % GS_W == 0, "slicing tasks per warp");
              float gsc[GT];
              int gcol[GT];
#pragma unroll
              for (int t = 0; t < GT; ++t) {
                const int task = warp + GS_W * t, ag = task % 5, ar = ag * 8 + (lane >> 2);
                gcol[t] = ar;
                int ex = 0;
                frexpf(__uint_as_float(cmax[ar < 20 ? ar : ar - 20]), &ex);
                gsc[t] = ldexpf(1.0f, -ex);   // |value| scale < 1, exact
              }
              auto gload = [&](int ch, float (&v)[GT][2]) {
#pragma unroll
                for (int t = 0; t < GT; ++t) {
                  const int task = warp + GS_W * t, rg = task / 5, ar = gcol[t];
                  const int j = ar < 20 ? ar : ar - 20, r0 = ch * GS_CH + rg * 8 + 2 * (lane & 3);
                  const float* z0 =
                      reinterpret_cast<const float*>(own(cur, r0 < P.R ? r0 : 0) + j) + (ar < 20 ? 0 : 1);
                  const float* z1 =
                      reinterpret_cast<const float*>(own(cur, r0 + 1 < P.R ? r0 + 1 : 0) + j) + (ar < 20 ? 0 : 1);
                  v[t][0] = r0 < P.R ? *z0 : 0.f;
                  v[t][1] = r0 + 1 < P.R ? *z1 : 0.f;
                }
              };
              float gnext[GT][2];
              gload(0, gnext);
              for (int ch = 0; ch < n_ch; ++ch) {
                const int b = ch & 1;
                float gv[GT][2];
#pragma unroll
                for (int t = 0; t < GT; ++t) {
                  gv[t][0] = gnext[t][0] * gsc[t];
                  gv[t][1] = gnext[t][1] * gsc[t];
                }
                if (ch + 1 < n_ch) gload(ch + 1, gnext);
                if (ch >= 2) {   // the MMAs of chunk ch - 2 are done with buffer b
                  if (*tc_abort == 0 && !mbar_wait(gs_bar[b], gs_ph[b] & 1u)) {
                    *tc_abort = 1;
                    set_error(a.p.err, DEV_TIMEOUT);
                  }
                  ++gs_ph[b];
                  tc_fence_after();
                }
                unsigned char* buf = smem + a.o_gs + b * GS_BUF;
#pragma unroll
                for (int sl = 0; sl < GS_N; ++sl)
#pragma unroll
                  for (int t = 0; t < GT; ++t) {
                    const int task = warp + GS_W * t, rg = task / 5, ag = task % 5;
                    const float y0 = gv[t][0] * 128.f, y1 = gv[t][1] * 128.f;
                    // round to the nearest integer by adding and subtracting 1.5 2^23
                    // (exact for |y| < 2^22; ties to even, as rintf)
                    const float k0 = __fsub_rn(__fadd_rn(y0, 12582912.f), 12582912.f);
                    const float k1 = __fsub_rn(__fadd_rn(y1, 12582912.f), 12582912.f);
                    gv[t][0] = y0 - k0;
                    gv[t][1] = y1 - k1;
                    // the integers are exact in bf16: the upper halves of their floats
                    reinterpret_cast<uint32_t*>(buf + rg * GS_LBO + (sl * 5 + ag) * 128)[lane] =
                        __byte_perm(__float_as_uint(k0), __float_as_uint(k1), 0x7632);
                  }
                // the chunk is in place: visible to the tensor cores, then announced
                async_proxy_fence();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(gs_fill[b]) : "memory");
              }
            } else {
              const int n_ch = (P.R + GS_CH - 1) / GS_CH;
              if (warp == GS_W) {
                // the issuing warp: per chunk, wait until it is sliced, then one
                // thread issues its MMAs and commits them to the buffer's mbarrier
                volatile int* tc_abort = reinterpret_cast<volatile int*>(misc + 141);
                for (int ch = 0; ch < n_ch; ++ch) {
                  const int b = ch & 1;
                  if (*tc_abort == 0 && !mbar_wait(gs_fill[b], gs_fph[b] & 1u)) {
                    *tc_abort = 1;
                    set_error(a.p.err, DEV_TIMEOUT);
                  }
                  ++gs_fph[b];
                  if (lane == 0 && *tc_abort == 0) {
                    tc_fence_after();
                    const uint32_t bb = smem_u32(smem + a.o_gs + b * GS_BUF);
                    for (int ks = 0; ks < GS_CH / 16; ++ks) {
                      const uint32_t ko = bb + (uint32_t)(ks * 2 * GS_LBO);
                      const uint32_t acc = (ch > 0 || ks > 0) ? 1u : 0u;
                      const uint64_t d0 = tc_desc(ko, GS_LBO, 128);              // m-rows 0..127
                      const uint64_t d2 = tc_desc(ko + 15 * 128, GS_LBO, 128);   // m-rows 120..247
                      gs_mma(tmem + GS_D0, d0, d0, gs_idesc(240), acc);
                      gs_mma(tmem + GS_D1, d0, tc_desc(ko + 30 * 128, GS_LBO, 128), gs_idesc(80), acc);
                      gs_mma(tmem + GS_D2, d2, d2, gs_idesc(128), acc);
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(gs_bar[b])
                        : "memory");
                  }
                  __syncwarp();
                }
              }
              // the slicing warps waited on every commit of buffer b but its last
              // (chunks b, b + 2, ...): the other warps count those phases too, so
              // that every thread waits on the same phase in the readout
#pragma unroll
              for (int b = 0; b < 2; ++b) {
                const int cb = (n_ch + 1 - b) / 2;
                if (cb > 1) gs_ph[b] += (uint32_t)(cb - 1);
              }
            }
          }
          for (;;) {
            int task = 0;
            if (lane == 0) task = atomicAdd(task_ctr, 1);
            task = __shfl_sync(0xffffffffu, task, 0);
            if (task >= n_g + n_t) break;
            if (task < n_g) {
              // upper tile (ti <= tj) of G
              int ti = 0, rem = task;
              while (rem >= nt_ - ti) { rem -= nt_ - ti; ++ti; }
              const int tj2 = ti + rem;
              const int i0 = ti * TP, j0 = tj2 * TP;
              if constexpr (GRAM_DW != 0) {
                DW acc[TP][TP][2];
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                  for (int j = 0; j < TP; ++j) acc[i][j][0] = acc[i][j][1] = DW{0.f, 0.f};
                for (int l = lane; l < P.R; l += 32) {
                  const T2* z = own(cur, l);
                  T2 zi[TP], zj[TP];
                  if constexpr (TP == 4) {
                    load4<ZSM>(z + i0, zi);
                    load4<ZSM>(z + j0, zj);
                  } else {
#pragma unroll
                    for (int i = 0; i < TP; ++i) zi[i] = z[i0 + i];
#pragma unroll
                    for (int j = 0; j < TP; ++j) zj[j] = z[j0 + j];
                  }
                  if (ti == tj2) {
                    // diagonal tile: only the upper triangle is needed
#pragma unroll
                    for (int i = 0; i < TP; ++i)
#pragma unroll
                      for (int j = i; j < TP; ++j) {   // conj(zi) * zj
                        dw_add_prod(acc[i][j][0], zi[i].x, zj[j].x);
                        dw_add_prod(acc[i][j][0], zi[i].y, zj[j].y);
                        dw_add_prod(acc[i][j][1], zi[i].x, zj[j].y);
                        dw_add_prod(acc[i][j][1], -zi[i].y, zj[j].x);
                      }
                  } else {
#pragma unroll
                    for (int i = 0; i < TP; ++i)
#pragma unroll
                      for (int j = 0; j < TP; ++j) {   // conj(zi) * zj
                        dw_add_prod(acc[i][j][0], zi[i].x, zj[j].x);
                        dw_add_prod(acc[i][j][0], zi[i].y, zj[j].y);
                        dw_add_prod(acc[i][j][1], zi[i].x, zj[j].y);
                        dw_add_prod(acc[i][j][1], -zi[i].y, zj[j].x);
                      }
                  }
                }
                // reduce-scatter over the warp (recursive halving): at offset o
                // every lane keeps the half of its values named by bit o of
                // its lane and adds the partner's copy; lane L ends with the
                // sum of value L = (i, j, re/im) of the 4 x 4 tile
                DW v[32];
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                  for (int j = 0; j < TP; ++j)
#pragma unroll
                    for (int c = 0; c < 2; ++c) v[(i * 4 + j) * 2 + c] = acc[i][j][c];
#pragma unroll
                for (int lev = 0; lev < 5; ++lev) {
                  const int o = 16 >> lev;
                  const bool up = (lane & o) != 0;
#pragma unroll
                  for (int k = 0; k < (16 >> lev); ++k) {
                    DW keep = up ? v[k + (16 >> lev)] : v[k];
                    const DW send = up ? v[k] : v[k + (16 >> lev)];
                    DW t;
                    t.hi = __shfl_xor_sync(0xffffffffu, send.hi, o);
                    t.lo = __shfl_xor_sync(0xffffffffu, send.lo, o);
                    dw_add(keep, t);
                    v[k] = keep;
                  }
                }
                reinterpret_cast<double*>(gp)[2 * ((i0 + (lane >> 3)) * Mp + j0 + ((lane >> 1) & 3)) + (lane & 1)] =
                    dw_value(v[0]);
              } else {
                T gr[TP][TP], gi[TP][TP];
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                  for (int j = 0; j < TP; ++j) gr[i][j] = gi[i][j] = 0;
                for (int l = lane; l < P.R; l += 32) {
                  const T2* z = own(cur, l);
                  T2 zi[TP], zj[TP];
#pragma unroll
                  for (int i = 0; i < TP; ++i) zi[i] = z[i0 + i];
#pragma unroll
                  for (int j = 0; j < TP; ++j) zj[j] = z[j0 + j];
#pragma unroll
                  for (int i = 0; i < TP; ++i)
#pragma unroll
                    for (int j = 0; j < TP; ++j) {
                      gr[i][j] = fma(zi[i].x, zj[j].x, fma(zi[i].y, zj[j].y, gr[i][j]));
                      gi[i][j] = fma(zi[i].x, zj[j].y, fma(-zi[i].y, zj[j].x, gi[i][j]));
                    }
                }
                // reduce-scatter: value (i TP + j) 2 + c, c = re / im
                constexpr int NVg = 2 * TP * TP, SH = TP == 4 ? 0 : 2;   // 2^p values, lane L holds L >> (5 - p)
                T v[NVg];
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                  for (int j = 0; j < TP; ++j) {
                    v[(i * TP + j) * 2] = gr[i][j];
                    v[(i * TP + j) * 2 + 1] = gi[i][j];
                  }
                warp_reduce_scatter(v, lane);
                if ((lane & ((1 << SH) - 1)) == 0) {
                  const int idx = lane >> SH, e2 = idx >> 1;
                  reinterpret_cast<double*>(gp)[2 * ((i0 + e2 / TP) * Mp + j0 + e2 % TP) + (idx & 1)] = (double)v[0];
                }
              }
            } else {
              // tile of T_r and T_b
              const int t2 = task - n_g, ti = t2 / nt_, tj2 = t2 - ti * nt_;
              const int i0 = ti * TP, j0 = tj2 * TP;
              T rr[TP][TP], ri[TP][TP], br[TP][TP], bi[TP][TP];
#pragma unroll
              for (int i = 0; i < TP; ++i)
#pragma unroll
                for (int j = 0; j < TP; ++j) rr[i][j] = ri[i][j] = br[i][j] = bi[i][j] = 0;
              // mode indices of row l, advanced by 32 rows per iteration without divisions
              int it = lane / P.st, irl = (lane - it * P.st) / Nf, iff = lane - it * P.st - irl * Nf;
              const int dq = 32 / Nf, dr = 32 - dq * Nf;
              for (int l = lane; l < P.R; l += 32) {
                const int iro = three ? iff : irl;     // with two modes C == 1 and r_lo == 0
                const T sr = iro + 1 < dro ? sq[iro + 1] : (T)0;
                const T sb = it + 1 < Nt ? sq[it + 1] : (T)0;
                const T2* z = own(cur, l);
                const T2* zr = own(cur, iro + 1 < dro ? l + 1 : l);
                const T2* zb = own(cur, it + 1 < Nt ? l + P.st : l);
                T2 wr[TP], wb[TP], yr[TP], yb[TP], zz[TP];
                if constexpr (TP == 4) {
                  load4<ZSM>(z + i0, zz);
                  load4<ZSM>(zr + j0, yr);
                  load4<ZSM>(zb + j0, yb);
                } else {
#pragma unroll
                  for (int i = 0; i < TP; ++i) zz[i] = z[i0 + i];
#pragma unroll
                  for (int j = 0; j < TP; ++j) {
                    yr[j] = zr[j0 + j];
                    yb[j] = zb[j0 + j];
                  }
                }
#pragma unroll
                for (int i = 0; i < TP; ++i) {
                  wr[i] = cm<T2>(sr * zz[i].x, -sr * zz[i].y);   // sr conj(z_i)
                  wb[i] = cm<T2>(sb * zz[i].x, -sb * zz[i].y);
                }
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                  for (int j = 0; j < TP; ++j) {
                    rr[i][j] = fma(wr[i].x, yr[j].x, fma(-wr[i].y, yr[j].y, rr[i][j]));
                    ri[i][j] = fma(wr[i].x, yr[j].y, fma(wr[i].y, yr[j].x, ri[i][j]));
                    br[i][j] = fma(wb[i].x, yb[j].x, fma(-wb[i].y, yb[j].y, br[i][j]));
                    bi[i][j] = fma(wb[i].x, yb[j].y, fma(wb[i].y, yb[j].x, bi[i][j]));
                  }
                iff += dr;
                irl += dq;
                if (iff >= Nf) {
                  iff -= Nf;
                  ++irl;
                }
                while (irl >= P.nr) {
                  irl -= P.nr;
                  ++it;
                }
              }
              if constexpr (TP == 4) {
                // reduce-scatter of the 64 partial sums (recursive halving, as
                // for the Gram tiles): lane L ends with the (re, im) pair of
                // entry L = (jump, i, j)
                T v[64];
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                  for (int j = 0; j < TP; ++j) {
                    v[(i * 4 + j) * 2] = rr[i][j];
                    v[(i * 4 + j) * 2 + 1] = ri[i][j];
                    v[(16 + i * 4 + j) * 2] = br[i][j];
                    v[(16 + i * 4 + j) * 2 + 1] = bi[i][j];
                  }
#pragma unroll
                for (int lev = 0; lev < 5; ++lev) {
                  const int o = 16 >> lev;
                  const bool up = (lane & o) != 0;
#pragma unroll
                  for (int k = 0; k < (32 >> lev); ++k) {
                    const T keep = up ? v[k + (32 >> lev)] : v[k];
                    const T send = up ? v[k] : v[k + (32 >> lev)];
                    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                  }
                }
                const int jb = lane >> 4, ii = (lane >> 2) & 3, jj = lane & 3;
                tp[jb * Mp * Mp + (i0 + ii) * Mp + j0 + jj] = cm<T2>(v[0], v[1]);
              } else {
                // TP = 2: 16 values ((jump 4 + i 2 + j) 2 + c), lane L holds L >> 1
                T v[16];
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                  for (int j = 0; j < TP; ++j) {
                    v[(i * 2 + j) * 2] = rr[i][j];
                    v[(i * 2 + j) * 2 + 1] = ri[i][j];
                    v[(4 + i * 2 + j) * 2] = br[i][j];
                    v[(4 + i * 2 + j) * 2 + 1] = bi[i][j];
                  }
                warp_reduce_scatter(v, lane);
                if ((lane & 1) == 0) {
                  const int idx = lane >> 1, e = idx >> 1, jb = e >> 2, ii = (e >> 1) & 1, jj = e & 1;
                  reinterpret_cast<T*>(tp)[2 * (jb * Mp * Mp + (i0 + ii) * Mp + j0 + jj) + (idx & 1)] = v[0];
                }
              }
            }
          }
          if (record) {
            // level populations and readout photons of own rows (FP64)
            for (int lv = warp; lv < Nt; lv += NWARP) {
              double s = 0.0, ph = 0.0;
              for (int r = lane; r < P.st; r += 32) {
                const int l = lv * P.st + r;
                const int irl = r / Nf, iff = r - irl * Nf;
                const int iro = three ? iff : irl;
                const T2* z = own(cur, l);
                double w = 0.0;
                for (int m = 0; m < M; ++m) w += (double)z[m].x * z[m].x + (double)z[m].y * z[m].y;
                s += w;
                ph += iro * w;
              }
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) {
                s += __shfl_xor_sync(0xffffffffu, s, o);
                ph += __shfl_xor_sync(0xffffffffu, ph, o);
              }
              if (lane == 0) {
                popp[lv] = s;
                misc[8 + lv] = ph;
              }
            }
            __syncthreads();
            if (tid == 0) {
              double ph = 0.0;
              for (int lv = 0; lv < Nt; ++lv) ph += misc[8 + lv];
              popp[LR_MAX_NT] = ph;
            }
          }
          if constexpr (GRAM_DW == 2) {
            // every chunk is sliced and issued before any thread waits here: a
            // parity wait tells a phase from the next one only, and the warps that
            // do not slice would otherwise arrive several commits early
            __syncthreads();
          }
          if constexpr (GRAM_DW == 2) {
            // ---- Gram on the tensor cores: wait for the last MMAs, stage the
            // slice-pair sums D(s,t) (s <= t, s + t <= 8) in the slice buffers,
            // then add them in double-word with their weights
            volatile int* tc_abort = reinterpret_cast<volatile int*>(misc + 141);
            const int n_ch = (P.R + GS_CH - 1) / GS_CH;
            for (int q2 = 0; q2 < (n_ch >= 2 ? 2 : 1); ++q2) {   // one commit pending per used buffer
              if (*tc_abort == 0 && !mbar_wait(gs_bar[q2], gs_ph[q2] & 1u)) {
                *tc_abort = 1;
                set_error(a.p.err, DEV_TIMEOUT);
              }
              ++gs_ph[q2];
            }
            tc_fence_after();
            // V[a][b] = sum over pairs s <= t, s + t <= 8 of c_st 2^-7(s+t) D_st[a][b]
            // with c_st = 1/2 for s = t, else 1, so that S = A^T A = V + V^T (D_ss is
            // symmetric). TMEM lane m holds row a = m % 40 of slice s = m / 40 (D0,
            // D1) and of slice 3 + m / 40 (D2); each warp of a lane quarter takes
            // blocks of 8 columns b and sums its slices' pairs over t in double-word
            // into V (double-word, in the slice buffers).
            DW* V = reinterpret_cast<DW*>(smem + a.o_gs);   // [40][40]
            const int qd = warp & 3, part = warp >> 2, m = qd * 32 + lane;
            const int sA = m / 40, aa = m % 40, sB = 3 + m / 40;
            static_assert(NWARP == 16, "four warps per TMEM lane quarter");
            for (int it2 = 0; it2 < 2; ++it2) {   // b-blocks part and part + 4 (< 5)
              const int bk = part + 4 * it2, b0 = bk * 8;
              const bool has = bk < 5;   // uniform within the warp
              DW cA[8], cB[8];           // slice sA (D0, D1) and slice sB (D2)
#pragma unroll
              for (int u = 0; u < 8; ++u) cA[u] = cB[u] = DW{0.f, 0.f};
              if (has) {
                // columns t = 0..10: D0 t = 0..5 and D1 t = 6, 7 (slice sA), D2 t = 3..5
                // (slice sB); loaded four blocks of 8 at a time, one wait per group
                auto tcol = [&](int t) {
                  return t < 6 ? GS_D0 + t * 40 + b0 : (t < 8 ? GS_D1 + (t - 6) * 40 + b0 : GS_D2 + (t - 8) * 40 + b0);
                };
                const uint32_t lane_base = tmem + ((uint32_t)(qd * 32) << 16);
#pragma unroll
                for (int g = 0; g < 3; ++g) {
                  uint32_t v[4][8];
#pragma unroll
                  for (int q = 0; q < 4; ++q) {
                    const int t = 4 * g + q;
                    if (t < 11)
                      asm volatile(
                          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                          : "=r"(v[q][0]), "=r"(v[q][1]), "=r"(v[q][2]), "=r"(v[q][3]), "=r"(v[q][4]), "=r"(v[q][5]),
                            "=r"(v[q][6]), "=r"(v[q][7])
                          : "r"(lane_base + (uint32_t)tcol(t)));
                  }
                  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                  for (int q = 0; q < 4; ++q) {
                    const int t = 4 * g + q;
                    if (t >= 11) continue;
                    const int s0 = t < 8 ? sA : sB, tt = t < 8 ? t : t - 5;
                    if (m < 120 && tt >= s0 && s0 + tt <= 8) {
                      // 2^-7(s+t), halved on the diagonal pairs: an exact power of two
                      const float w = __int_as_float((127 - 7 * (s0 + tt) - (s0 == tt ? 1 : 0)) << 23);
#pragma unroll
                      for (int u = 0; u < 8; ++u) {
                        if (t < 8)
                          dw_add_f(cA[u], w * __uint_as_float(v[q][u]));
                        else
                          dw_add_f(cB[u], w * __uint_as_float(v[q][u]));
                      }
                    }
                  }
                }
              }
              // every thread has seen the last MMA complete: the slice buffers are free.
              // Lane m < 40 holds slices 0 and 3 of row a, 40 <= m < 80 slices 1 and 4,
              // 80 <= m < 120 slice 2: each adds its two, and the three lane groups add
              // their rows into V in that order, one barrier apart.
              if (has && m < 120)
#pragma unroll
                for (int u = 0; u < 8; ++u) dw_add(cA[u], cB[u]);
              for (int round = 0; round < 3; ++round) {
                if (has && m < 120 && sA == round)
#pragma unroll
                  for (int u = 0; u < 8; ++u) {
                    DW& dst = V[aa * 40 + b0 + u];
                    if (round == 0) {
                      dst = cA[u];
                    } else {
                      DW x = dst;
                      dw_add(x, cA[u]);
                      dst = x;
                    }
                  }
                __syncthreads();
              }
            }
            tc_fence_before();
            __syncthreads();
            // S entries for G: S[a][b] = V[a][b] + V[b][a]
            DW* Sb = reinterpret_cast<DW*>(W);
            for (int e = tid; e < 820; e += NT) {
              int ia, ib;
              if (e < 420) {
                const int e2 = e < 210 ? e : e - 210, off = e < 210 ? 0 : 20;
                ia = tri[e2].y + off;
                ib = tri[e2].x + off;
              } else {
                ia = (e - 420) / 20;
                ib = 20 + (e - 420) % 20;
              }
              DW acc = V[ia * 40 + ib];
              dw_add(acc, V[ib * 40 + ia]);
              Sb[e] = acc;
            }
            __syncthreads();
            for (int e = tid; e < 210; e += NT) {
              const int i = tri[e].y, j = tri[e].x;   // i <= j
              int ei = 0, ej = 0;
              frexpf(__uint_as_float(gs_cmax[gs_par * 20 + i]), &ei);
              frexpf(__uint_as_float(gs_cmax[gs_par * 20 + j]), &ej);
              const double sc = ldexp(1.0, ei + ej - 14);
              DW re = Sb[e], im = Sb[420 + i * 20 + j];
              dw_add(re, Sb[210 + e]);
              const DW n2 = Sb[420 + j * 20 + i];
              dw_add(im, DW{-n2.hi, -n2.lo});
              gp[i * Mp + j] = mk(dw_value(re) * sc, dw_value(im) * sc);
            }
          }
        }
        // ================= B1
        cluster.sync();

        // ================= R: reduce in rank order, FP64 Cholesky and inverse
        {
          const int MM = Mp * Mp, MMq = Mq * Mq;
          for (int e = tid; e < 3 * MMq; e += NT) {
            const int mat = e / MMq, iq = e - mat * MMq, i = iq / Mq, j = iq - i * Mq, ij = i * Mp + j;
            if (mat == 0) {
              if (i > j || j >= M) continue;
              // issue the remote loads four at a time, then sum in rank order
              double re = 0.0, im = 0.0;
              for (int r0 = 0; r0 < C; r0 += 4) {
                double2 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                  v[u] = r0 + u < C ? cluster.map_shared_rank(gp, r0 + u)[i * Mp + j] : mk(0.0, 0.0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  re += v[u].x;
                  im += v[u].y;
                }
              }
              if (i == j) {
                Gd[i * ldg + i] = mk(re, 0.0);
              } else {
                Gd[i * ldg + j] = mk(re, im);
                Gd[j * ldg + i] = mk(re, -im);
              }
            } else {
              T re = 0, im = 0;
              for (int r0 = 0; r0 < C; r0 += 4) {
                T2 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                  v[u] = r0 + u < C ? cluster.map_shared_rank(tp, r0 + u)[(mat - 1) * MM + ij] : cm<T2>(0, 0);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  re += v[u].x;
                  im += v[u].y;
                }
              }
              Tred[(mat - 1) * MM + ij] = cm<T2>(re, im);
              if (mat == 1 && i == j) {
                trd[i] = (double)re;
                misc[32 + i] = (double)im;
              }
            }
          }
          if (record && tid < LR_MAX_NT + 1) {
            double s = 0.0;
            const bool use = tid < Nt || tid == LR_MAX_NT;
            if (use)
              for (int r = 0; r < C; ++r) s += cluster.map_shared_rank(popp, r)[tid];
            misc[64 + tid] = s;
          }
          if (tid == 0) {
            misc[1] = 0.0;   // not-PD flag
            *reinterpret_cast<int*>(misc + 140) = 0;   // phase-P task counter of the next stage
            // bulk-precision copies: coefficient, step sizes split as hi + lo
            T* tb = reinterpret_cast<T*>(misc + 128);
            const double hs = stage == 2 ? dt : 0.5 * dt, h6 = dt / 6.0;
            tb[1] = (T)hs;
            tb[2] = (T)(hs - (double)tb[1]);
            tb[3] = (T)h6;
            tb[4] = (T)(h6 - (double)tb[3]);
          }
          __syncthreads();
          if (record && q == 0 && a.p.gsnap) {
            // FP64 Gram matrix of this record step, for the diagnostics
            double2* gs = a.p.gsnap + ((size_t)tj * a.rp.n_rec + step / pe) * a.rp.snap_m * a.rp.snap_m;
            for (int e = tid; e < M * M; e += NT) gs[(e / M) * a.rp.snap_m + e % M] = Gd[(e / M) * ldg + e % M];
            __syncthreads();   // the M x M phase below overwrites G in place
          }
          if (stage == 0 && q == 0 && tid == 0) {
            double br = 0.0, bi = 0.0;
            for (int i = 0; i < M; ++i) {
              br += trd[i];
              bi += misc[32 + i];
            }
            a.p.beta[(size_t)tj * (a.rp.max_steps + 1) + step] = mk(br, bi);
            if (!isfinite(br) || !isfinite(bi)) set_error(a.p.err, DEV_NONFINITE);
            if (record) {
              const long rec = step / pe;
              double trace = 0.0;
              for (int lv = 0; lv < a.rp.nt_max; ++lv) {
                const double v = lv < Nt ? misc[64 + lv] : 0.0;
                a.p.pops[((size_t)tj * a.rp.n_rec + rec) * a.rp.nt_max + lv] = v;
                trace += v;
              }
              a.p.nphot[(size_t)tj * a.rp.n_rec + rec] = misc[64 + LR_MAX_NT];
              a.p.trace[(size_t)tj * a.rp.n_rec + rec] = trace;
            }
          }
          if (last) break;
          T2* Gi = reinterpret_cast<T2*>(Gd);   // G^-1 reuses the storage of L once L is no longer needed
          if constexpr (sizeof(T) == 4) {
            // FP32 state: the same factorisation and inverse in double-word FP32
            // (~2^-48 relative, FP64-class like the Gram matrix), on the FP32 pipes:
            // on this GPU an FP64 warp instruction holds its SMSP's FP64 pipe for
            // ~60 cycles, and G^-1 is rounded to FP32 at the end anyway. G, L and W
            // use the storage of their FP64 counterparts (16 bytes per entry).
            DWC* Gw = reinterpret_cast<DWC*>(Gd);
            DWC* Ww = reinterpret_cast<DWC*>(W);
            DW* dinv = reinterpret_cast<DW*>(misc + 96);   // [M] 1 / D[k]
            float* diag0 = reinterpret_cast<float*>(W);    // W[k][0] slot: the diagonal of G
            for (int e = tid; e < M * (M + 1) / 2; e += NT) {
              const int i = tri[e].x, j = tri[e].y;
              const double2 v = Gd[i * ldg + j];
              DWC g;
              g.re = dw_make(v.x);
              g.im = dw_make(v.y);
              if (i == j) diag0[i * ldg * 4] = (float)v.x;
              Gw[i * ldg + j] = g;
            }
            // pivot k: breakdown check against the original diagonal, then 1 / D[k]
            auto pivot = [&](int k) {
              const DW piv = Gw[k * ldg + k].re;
              if (!(piv.hi > 1e-13f * diag0[k * ldg * 4]) || !isfinite(piv.hi) || piv.hi < 1e-30f) {
                misc[1] = 1.0;
                dinv[k].hi = 1.0f;
                dinv[k].lo = 0.0f;
              } else {
                dinv[k] = dw_recip(piv);
              }
            };
            __syncthreads();
            if (tid == 0) pivot(0);
            __syncthreads();
            for (int k = 0; k < M; ++k) {
              const DW rk = dinv[k];
              const int w = M - k - 1;
              // trailing update G[i][j] -= G[i][k] conj(G[j][k]) / D[k], i >= j > k;
              // entry 0 (the next pivot) belongs to thread 0, which then forms
              // 1 / D[k+1] before the barrier: one barrier per elimination step
              for (int e = tid; e < w * (w + 1) / 2; e += NT) {
                const int i = k + 1 + tri[e].x, j = k + 1 + tri[e].y;
                const DWC t = dwc_scale(dwc_mul_conj(Gw[i * ldg + k], Gw[j * ldg + k]), rk);
                Gw[i * ldg + j] = dwc_sub(Gw[i * ldg + j], t);
              }
              if (tid == 0 && k + 1 < M) pivot(k + 1);
              __syncthreads();
            }
            if (tid == 0 && misc[1] != 0.0) set_error(a.p.err, DEV_NOT_PD);
            // W = L^-1 (unit lower, L[i][k] = G[i][k] / D[k]) by columns: column j
            // by warp j mod NWARP, lane i = row i, forward substitution
            // W[i][j] = delta_ij - sum_{j <= k < i} L[i][k] W[k][j] with W[k][j]
            // broadcast from lane k (no block barrier)
            for (int j = warp; j < M; j += NWARP) {
              DWC wv;
              wv.re.hi = lane == j ? 1.0f : 0.0f;
              wv.re.lo = wv.im.hi = wv.im.lo = 0.0f;
              for (int k = j; k < M - 1; ++k) {
                DWC wk;
                wk.re.hi = __shfl_sync(0xffffffffu, wv.re.hi, k);
                wk.re.lo = __shfl_sync(0xffffffffu, wv.re.lo, k);
                wk.im.hi = __shfl_sync(0xffffffffu, wv.im.hi, k);
                wk.im.lo = __shfl_sync(0xffffffffu, wv.im.lo, k);
                if (lane > k && lane < M) wv = dwc_sub(wv, dwc_mul(dwc_scale(Gw[lane * ldg + k], dinv[k]), wk));
              }
              if (lane < M) Ww[lane * ldg + j] = wv;
            }
            __syncthreads();
            // G^-1 = W^dag D^-1 W (Hermitian): entry (i, j), i <= j, is
            // sum_{k >= j} conj(W[k][i]) W[k][j] / D[k], kept in double-word (in the
            // storage of G, no longer needed): X_k = G^-1 T_k is formed from it in
            // double-word below, because G^-1 has entries up to 1 / p_M and a product
            // rounded to FP32 first would lose the small columns to cancellation
            for (int e = tid; e < M * M; e += NT) {
              const int i = e / M, j = e - i * M;
              if (i > j) continue;
              DWC acc;
              acc.re.hi = acc.re.lo = acc.im.hi = acc.im.lo = 0.0f;
              for (int k = j; k < M; ++k)   // W[k][j] conj(W[k][i]) = conj of the term
                acc = dwc_add(acc, dwc_scale(dwc_mul_conj(Ww[k * ldg + j], Ww[k * ldg + i]), dinv[k]));
              Gw[i * ldg + j] = acc;
              if (i != j) {
                acc.im = dw_neg(acc.im);
                Gw[j * ldg + i] = acc;
              }
            }
            __syncthreads();
          } else {
            // FP64 G = L D L^dag (unit lower L, right-looking, in place in Gd), then
            // W = L^-1 (unit lower) and G^-1 = W^dag D^-1 W. One FP64 reciprocal per
            // pivot (formed once and shared: FP64 runs at 2 FMA/clk/SM here) and two
            // block barriers per elimination step.
            double* dinv = misc + 96;     // [M] 1 / D[k]
            // keep the diagonal of G: a pivot below 1e-13 of it is a numerical breakdown
            for (int k = tid; k < M; k += NT) W[k * ldg] = Gd[k * ldg + k];
            __syncthreads();
            for (int k = 0; k < M; ++k) {
              if (tid == 0) {
                const double piv = Gd[k * ldg + k].x;
                if (!(piv > 1e-13 * W[k * ldg].x) || !isfinite(piv) || piv < 1e-30) {
                  misc[1] = 1.0;
                  dinv[k] = 1.0;
                } else {
                  // reciprocal by Newton-Raphson, r <- r (2 - piv r), from the FP32
                  // estimate: 24 -> 48 -> 96 correct bits, two FP64 FMA pairs on the
                  // serial path instead of a full FP64 division
                  double r = (double)(1.0f / (float)piv);
                  r = r * fma(-piv, r, 2.0);
                  r = r * fma(-piv, r, 2.0);
                  dinv[k] = r;
                }
              }
              __syncthreads();
              const double rk = dinv[k];
              const int w = M - k - 1;
              // trailing update G[i][j] -= G[i][k] conj(G[j][k]) / D[k], i >= j > k
              for (int e = tid; e < w * (w + 1) / 2; e += NT) {
                const int i = k + 1 + tri[e].x, j = k + 1 + tri[e].y;
                const double2 x = Gd[i * ldg + k], y = Gd[j * ldg + k], g = Gd[i * ldg + j];
                Gd[i * ldg + j] = mk(g.x - rk * (x.x * y.x + x.y * y.y), g.y - rk * (x.y * y.x - x.x * y.y));
              }
              __syncthreads();
            }
            if (tid == 0 && misc[1] != 0.0) set_error(a.p.err, DEV_NOT_PD);
            // unit lower L[i][k] = G[i][k] / D[k]; W = L^-1 row by row (unit diagonal)
            for (int e = tid; e < M * M; e += NT) {
              const int i = e / M, j = e - i * M;
              W[i * ldg + j] = mk(i == j ? 1.0 : 0.0, 0.0);
              if (i > j) {
                const double2 v = Gd[i * ldg + j];
                Gd[i * ldg + j] = mk(v.x * dinv[j], v.y * dinv[j]);
              }
            }
            __syncthreads();
            for (int k = 0; k < M - 1; ++k) {
              // rows i > k: W[i][j] -= L[i][k] W[k][j], j <= k (W[k] is final)
              const int rows = M - k - 1;
              for (int e = tid; e < rows * (k + 1); e += NT) {
                const int i = k + 1 + e / (k + 1), j = e % (k + 1);
                const double2 l = Gd[i * ldg + k], wv = W[k * ldg + j], o = W[i * ldg + j];
                W[i * ldg + j] = mk(o.x - (l.x * wv.x - l.y * wv.y), o.y - (l.x * wv.y + l.y * wv.x));
              }
              __syncthreads();
            }
            // G^-1 = W^dag D^-1 W (Hermitian), rounded once to the bulk precision
            for (int e = tid; e < M * M; e += NT) {
              const int i = e / M, j = e - i * M;
              if (i > j) continue;
              double re = 0.0, im = 0.0;
              for (int k = j; k < M; ++k) {          // W[k][i], W[k][j] nonzero for k >= max(i, j) = j
                const double2 x = W[k * ldg + i], y = W[k * ldg + j];   // conj(x) y / D[k]
                re += dinv[k] * (x.x * y.x + x.y * y.y);
                im += dinv[k] * (x.x * y.y - x.y * y.x);
              }
              Gi[i * Mp + j] = cm<T2>((T)re, (T)im);
              if (i != j) Gi[j * Mp + i] = cm<T2>((T)re, (T)-im);
            }
            __syncthreads();
          }
          // XT_k[l][m] = s_k conj(X_k[m][l]), X_k = G^-1 T_k
          const double sk[2] = {0.5 * d.kappa, 0.5 * d.gamma};
          for (int e = tid; e < 2 * Mq * Mq; e += NT) {
            const int k = e / (Mq * Mq), lq = e - k * (Mq * Mq), l = lq / Mq, m = lq - l * Mq, lm = l * Mp + m;
            T xr = 0, xi = 0;
            if (l < M && m < M) {
              const T2* Tk = Tred + k * MM;
              if constexpr (sizeof(T) == 4) {
                // FP32 state: double-word sums of G^-1 (double-word) times T_k (exact)
                const DWC* Giw = reinterpret_cast<const DWC*>(Gd);
                DWC acc;
                acc.re.hi = acc.re.lo = acc.im.hi = acc.im.lo = 0.0f;
                for (int j = 0; j < M; ++j) {
                  const T2 t = Tk[j * Mp + l];
                  acc = dwc_add(acc, dwc_mul_f(Giw[m * ldg + j], t.x, t.y));
                }
                xr = acc.re.hi + acc.re.lo;
                xi = acc.im.hi + acc.im.lo;
              } else {
                for (int j = 0; j < M; ++j) {
                  const T2 gv = Gi[m * Mp + j];
                  const T gr = gv.x, gi = gv.y;
                  const T2 t = Tk[j * Mp + l];
                  xr = fma(gr, t.x, fma(-gi, t.y, xr));
                  xi = fma(gr, t.y, fma(gi, t.x, xi));
                }
              }
            }
            const T s = (T)sk[k];
            XT[k * MM + lm] = cm<T2>(s * xr, -s * xi);
            if constexpr (TC > 0) {
              // real 2x2 block of X = (xr', xi') at B rows (2m, 2m+1), K columns
              // (k 2Mp + 2l, +1): [xr', -xi'; xi', xr'] maps (re, im) of A to D
              const float Xr = (float)(s * xr), Xi = (float)(-s * xi);
              const int kk = k * 2 * Mp + 2 * l;
              const float vals[4] = {Xr, -Xi, Xi, Xr};
              for (int u = 0; u < 4; ++u) {
                const int o = kmaj_off(2 * m + (u >> 1), kk + (u & 1), a.npad) / 4;
                const float big = tf32_rna(vals[u]);
                tb_big[o] = big;
                if (TC == 3) tb_small[o] = tf32_rna(vals[u] - big);
              }
            }
          }
          if constexpr (TC > 0) async_proxy_fence();
          __syncthreads();
        }

        // ================= F: right-hand side and RK4 stage update
        // Thread tile: TR consecutive rows x 4 columns. Pass 1 forms -i H_eff Z_s
        // per row, pass 2 adds the projection terms with every XT load shared by
        // the TR rows, pass 3 applies the RK4 stage update.
        {
          // coefficient and split step sizes h = hi + lo (no systematic FP32 step error)
          const T* tb = reinterpret_cast<const T*>(misc + 128);
          const T c = tb[0], hs_hi = tb[1], hs_lo = tb[2], h6_hi = tb[3], h6_lo = tb[4], ci = tb[5];
          constexpr bool rwa = FRAME != 0;
          // Z_n rows start on 16-byte boundaries for the paired FP32 accesses
          const bool zn_vec = sizeof(T2) == 8 && (M % 2) == 0 && (d.z_off % 2) == 0;
          const int nxt = cur ^ 1;
          const int mq = Mq / 4;
          const int nrt_all = (P.R + TR - 1) / TR;
          const T g = (T)d.g, J = (T)d.J, ka = (T)d.kappa, ga = (T)d.gamma;
          const int MM = Mp * Mp;
          if constexpr (TC > 0) {
            // ---- projection term on the tensor cores, in tiles of TC_ROWS rows.
            // Thread (warp w, lane) owns tile row 32 (w % 4) + lane, the TMEM lane
            // it may read, and column quads w / 4, w / 4 + 3, ... The MMAs of a
            // tile run while the threads form -i H_eff Z_s for it; the next tile's
            // operand staging and MMAs overlap the RK4 update of this one.
            const int qd = warp & 3, grp = warp >> 2;
            constexpr int QMAX = 3;   // column quads per thread (Mp <= 36)
            const int n_sub = (P.R + TC_ROWS - 1) / TC_ROWS;
            const uint32_t lboA = TC_ROWS * 16, lboB = (uint32_t)a.npad * 16;
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(a.npad >> 3) << 17) |
                                   ((uint32_t)(TC_ROWS >> 4) << 24);
            // operand A of the tile starting at row_lo: row tid % TC_ROWS, float4
            // chunks c4 = tid / TC_ROWS + 3 j; chunk c4 holds complex columns 2cj,
            // 2cj+1 of s_r rZ_s (c4 < Mp/2) or s_b bZ_s (c4 >= Mp/2)
            auto build_a = [&](int row_lo) {
              const int r = tid % TC_ROWS, l = row_lo + r;
              const T2* srcr = nullptr;
              const T2* srcb = nullptr;
              float scr = 0.f, scb = 0.f;
              if (l < P.R) {
                const int it = l / P.st, rem = l - it * P.st, irl = rem / Nf, iff = rem - irl * Nf;
                const int iro = three ? iff : P.r_lo + irl;
                if (iro + 1 < dro) {
                  srcr = own(cur, l + 1);
                  scr = sq[iro + 1];
                }
                if (it + 1 < Nt) {
                  srcb = own(cur, l + P.st);
                  scb = sq[it + 1];
                }
              }
              for (int c4 = tid / TC_ROWS; c4 < Mp; c4 += NT / TC_ROWS) {
                const int jump = c4 >= Mp / 2 ? 1 : 0;
                const int cj = c4 - jump * (Mp / 2);
                const T2* src = jump ? srcb : srcr;
                const float sc = jump ? scb : scr;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (src) {
                  v = reinterpret_cast<const float4*>(src)[cj];
                  v.x *= sc;
                  v.y *= sc;
                  v.z *= sc;
                  v.w *= sc;
                }
                const int o = kmaj_off(r, 4 * c4, TC_ROWS) / 4;
                const float4 big = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
                *reinterpret_cast<float4*>(ta_big + o) = big;
                if (TC == 3)
                  *reinterpret_cast<float4*>(ta_small + o) = make_float4(
                      tf32_rna(v.x - big.x), tf32_rna(v.y - big.y), tf32_rna(v.z - big.z), tf32_rna(v.w - big.w));
              }
              async_proxy_fence();
            };
            auto issue = [&]() {
              if (tid == 0) {
                tc_fence_after();
                // K = 4 Mp in steps of 8; each pass and half of K accumulates in
                // its own TMEM columns so that the MMA chains run side by side
                const int nks = Mp / 2, half = (nks + 1) / 2;
                for (int ks = 0; ks < nks; ++ks)
                  for (int pass = 0; pass < TC; ++pass) {
                    const uint32_t A0 = smem_u32(pass == 2 ? ta_small : ta_big);
                    const uint32_t B0 = smem_u32(pass == 1 ? tb_small : tb_big);
                    const int acc = pass * TC_KSPLIT + (ks >= half ? 1 : 0);
                    tc_mma(tmem + (uint32_t)(acc * TC_ACC), tc_desc(A0 + ks * 2 * lboA, lboA, 128),
                           tc_desc(B0 + ks * 2 * lboB, lboB, 128), idesc, ks != 0 && ks != half);
                  }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                             : "memory");
              }
            };
            build_a(0);
            __syncthreads();
            issue();
            for (int sub = 0; sub < n_sub; ++sub) {
              const int l = sub * TC_ROWS + qd * 32 + lane;
              const bool in = l < P.R;
              int it = 0, irl = 0, iff = 0;
              if (in) {
                it = l / P.st;
                const int rem = l - it * P.st;
                irl = rem / Nf;
                iff = rem - irl * Nf;
              }
              const int ir = P.r_lo + irl, iro = three ? iff : ir;
              T fr[QMAX][4], fi[QMAX][4];
              // -i H_eff Z_s for the thread's row and column quads
              T dh = 0, dl = 0, dim_ = 0;
              if (in) {
                const T a0 = dtab[(0 * TAB + it) * 2], a1 = dtab[(1 * TAB + ir) * 2], a2 = dtab[(2 * TAB + iff) * 2];
                T s1 = a0 + a1;
                T bp = s1 - a0;
                T er = (a0 - (s1 - bp)) + (a1 - bp);
                T s2 = s1 + a2;
                bp = s2 - s1;
                er += (s1 - (s2 - bp)) + (a2 - bp);
                dh = s2;
                dl = er + dtab[(0 * TAB + it) * 2 + 1] + dtab[(1 * TAB + ir) * 2 + 1] + dtab[(2 * TAB + iff) * 2 + 1];
                dim_ = (T)(-0.5) * (ka * (T)iro + ga * (T)it);
              }
#pragma unroll
              for (int qq = 0; qq < QMAX; ++qq) {
                const int m0 = (grp + 3 * qq) * 4;
#pragma unroll
                for (int u = 0; u < 4; ++u) fr[qq][u] = fi[qq][u] = 0;
                if (m0 >= Mp || !in) continue;
                T2 z[4];
                load4<ZSM>(own(cur, l) + m0, z);
                T hr[4], hi[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  hr[u] = fma(dh, z[u].x, fma(dl, z[u].x, -dim_ * z[u].y));
                  hi[u] = fma(dh, z[u].y, fma(dl, z[u].y, dim_ * z[u].x));
                }
                auto add_row = [&](const T2* vp, T w) {
                  T2 v[4];
                  load4<ZSM>(vp, v);
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    hr[u] = fma(w, v[u].x, hr[u]);
                    hi[u] = fma(w, v[u].y, hi[u]);
                  }
                };
                // complex weight wr + i wi (the rotating-frame drive)
                auto add_row_c = [&](const T2* vp, T wr, T wi) {
                  T2 v[4];
                  load4<ZSM>(vp, v);
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    hr[u] = fma(wr, v[u].x, fma(-wi, v[u].y, hr[u]));
                    hi[u] = fma(wr, v[u].y, fma(wi, v[u].x, hi[u]));
                  }
                };
                // g (b + b^dag)(a + a^dag)
#pragma unroll
                for (int sa = -1; sa <= 1; sa += 2) {
                  const int it2 = it + sa;
                  if (it2 < 0 || it2 >= Nt) continue;
                  const T ct = g * sq[max(it, it2)];
#pragma unroll
                  for (int sb2 = -1; sb2 <= 1; sb2 += 2) {
                    const int ir2 = ir + sb2;
                    if (ir2 < 0 || ir2 >= Nr) continue;
                    if (rwa && sa == sb2) continue;   // RWA: g (b^dag a + b a^dag) only
                    add_row(zrow(cur, it2, ir2, iff) + m0, ct * sq[max(ir, ir2)]);
                  }
                }
                if (three) {
                  // J (a + a^dag)(f + f^dag)
#pragma unroll
                  for (int sa = -1; sa <= 1; sa += 2) {
                    const int ir2 = ir + sa;
                    if (ir2 < 0 || ir2 >= Nr) continue;
                    const T cr = J * sq[max(ir, ir2)];
#pragma unroll
                    for (int sb2 = -1; sb2 <= 1; sb2 += 2) {
                      const int if2 = iff + sb2;
                      if (if2 < 0 || if2 >= Nf) continue;
                      if (rwa && sa == sb2) continue;   // RWA: J (a^dag f + a f^dag) only
                      add_row(zrow(cur, it, ir2, if2) + m0, cr * sq[max(iff, if2)]);
                    }
                  }
                  // drive on the filter
#pragma unroll
                  for (int sa = -1; sa <= 1; sa += 2) {
                    const int if2 = iff + sa;
                    if (if2 < 0 || if2 >= Nf) continue;
                    if (rwa)
                      add_row_c(own(cur, l + sa) + m0, c * sq[max(iff, if2)], (sa > 0 ? ci : -ci) * sq[max(iff, if2)]);
                    else
                      add_row(own(cur, l + sa) + m0, c * sq[max(iff, if2)]);
                  }
                } else {
                  // drive on the resonator (two modes, C == 1)
#pragma unroll
                  for (int sa = -1; sa <= 1; sa += 2) {
                    const int ir2 = ir + sa;
                    if (ir2 < 0 || ir2 >= Nr) continue;
                    if (rwa)
                      add_row_c(own(cur, l + sa) + m0, c * sq[max(ir, ir2)], (sa > 0 ? ci : -ci) * sq[max(ir, ir2)]);
                    else
                      add_row(own(cur, l + sa) + m0, c * sq[max(ir, ir2)]);
                  }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  fr[qq][u] = hi[u];
                  fi[qq][u] = -hr[u];
                }
              }
              // + projection term D from tensor memory (lane = tile row)
              volatile int* tc_abort = reinterpret_cast<volatile int*>(misc + 141);
              if (*tc_abort == 0 && !mbar_wait(mbar, tc_phase)) {
                *tc_abort = 1;
                set_error(a.p.err, DEV_TIMEOUT);
              }
              tc_phase ^= 1u;
              tc_fence_after();
#pragma unroll
              for (int qq = 0; qq < QMAX; ++qq) {
                const int quad = grp + 3 * qq;
                if (quad * 4 >= Mp) continue;   // uniform across the warp
                const int n_acc = Mp / 2 > 1 ? TC * TC_KSPLIT : TC;
                float dsum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int acc = 0; acc < n_acc; ++acc) {
                  uint32_t v[8];
                  asm volatile(
                      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                      : "r"(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(acc * TC_ACC + quad * 8)));
                  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                  for (int u = 0; u < 8; ++u) dsum[u] += __uint_as_float(v[u]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  fr[qq][u] += dsum[2 * u];
                  fi[qq][u] += dsum[2 * u + 1];
                }
              }
              tc_fence_before();
              __syncthreads();   // TMEM and operand A of this tile are free
              if (sub + 1 < n_sub) {
                build_a((sub + 1) * TC_ROWS);
                __syncthreads();
                issue();
              }
              // RK4 update (weights 1/6, 1/3, 1/3, 1/6)
              if (in) {
                const int n = (it * Nr + ir) * Nf + iff;
#pragma unroll
                for (int qq = 0; qq < QMAX; ++qq) {
                  const int m0 = (grp + 3 * qq) * 4;
                  if (m0 >= Mp) continue;
                  T2 zo[4];
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    const int m = m0 + u;
                    if (m >= M) {
                      zo[u] = cm<T2>(0, 0);
                      continue;
                    }
                    const size_t oz = (size_t)n * M + m, oa = (size_t)n * Mp + m;
                    const T2 zn = Zn[oz];
                    if (stage == 0) {
                      accg[oa] = cm<T2>(fr[qq][u], fi[qq][u]);
                    } else if (stage < 3) {
                      const T2 ac = accg[oa];
                      accg[oa] = cm<T2>(fma((T)2, fr[qq][u], ac.x), fma((T)2, fi[qq][u], ac.y));
                    }
                    if (stage < 3) {
                      zo[u] = cm<T2>(zn.x + fma(hs_lo, fr[qq][u], hs_hi * fr[qq][u]),
                                     zn.y + fma(hs_lo, fi[qq][u], hs_hi * fi[qq][u]));
                    } else {
                      const T2 ac = accg[oa];
                      const T s_r = ac.x + fr[qq][u], s_i = ac.y + fi[qq][u];
                      const T2 z1 =
                          cm<T2>(zn.x + fma(h6_lo, s_r, h6_hi * s_r), zn.y + fma(h6_lo, s_i, h6_hi * s_i));
                      Zn[oz] = z1;
                      zo[u] = z1;
                    }
                  }
                  store4<ZSM>(own(nxt, l) + m0, zo);
                }
              }
            }
          } else {
          const int nrt = nrt_all;
          const int row_lo = 0;
          for (int tile = tid; tile < nrt * mq; tile += NT) {
            const int rt = tile / mq, m0 = (tile - rt * mq) * 4;
            float cmx[4] = {0.f, 0.f, 0.f, 0.f};   // column maxima of the rows written (tensor-core Gram)
            T fr[TR][4], fi[TR][4];
            T sr[TR], sb[TR];
            const T2* yrp[TR];
            const T2* ybp[TR];
            int nrow[TR];
            const int l0 = row_lo + rt * TR;
            int it = l0 / P.st, irl = (l0 - it * P.st) / Nf, iff = l0 - it * P.st - irl * Nf;
#pragma unroll
            for (int r = 0; r < TR; ++r) {
              const int l = l0 + r;
              sr[r] = 0;
              sb[r] = 0;
              yrp[r] = own(cur, 0);
              ybp[r] = own(cur, 0);
              nrow[r] = -1;
#pragma unroll
              for (int u = 0; u < 4; ++u) fr[r][u] = fi[r][u] = 0;
              if (l < P.R) {
                const int ir = P.r_lo + irl;
                const int iro = three ? iff : ir;
                nrow[r] = (it * Nr + ir) * Nf + iff;
                // H_eff diagonal: real part as an unevaluated sum dh + dl
                T dh, dl;
                {
                  const T a0 = dtab[(0 * TAB + it) * 2], a1 = dtab[(1 * TAB + ir) * 2], a2 = dtab[(2 * TAB + iff) * 2];
                  T s1 = a0 + a1;
                  T bp = s1 - a0;
                  T er = (a0 - (s1 - bp)) + (a1 - bp);
                  T s2 = s1 + a2;
                  bp = s2 - s1;
                  er += (s1 - (s2 - bp)) + (a2 - bp);
                  dh = s2;
                  dl = er + dtab[(0 * TAB + it) * 2 + 1] + dtab[(1 * TAB + ir) * 2 + 1] + dtab[(2 * TAB + iff) * 2 + 1];
                }
                const T dim_ = (T)(-0.5) * (ka * (T)iro + ga * (T)it);
                T2 z[4];
                load4<ZSM>(own(cur, l) + m0, z);
                T hr[4], hi[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  hr[u] = fma(dh, z[u].x, fma(dl, z[u].x, -dim_ * z[u].y));
                  hi[u] = fma(dh, z[u].y, fma(dl, z[u].y, dim_ * z[u].x));
                }
                auto add_row = [&](const T2* vp, T w) {
                  T2 v[4];
                  load4<ZSM>(vp, v);
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    hr[u] = fma(w, v[u].x, hr[u]);
                    hi[u] = fma(w, v[u].y, hi[u]);
                  }
                };
                // complex weight wr + i wi (the rotating-frame drive)
                auto add_row_c = [&](const T2* vp, T wr, T wi) {
                  T2 v[4];
                  load4<ZSM>(vp, v);
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    hr[u] = fma(wr, v[u].x, fma(-wi, v[u].y, hr[u]));
                    hi[u] = fma(wr, v[u].y, fma(wi, v[u].x, hi[u]));
                  }
                };
                // Rows (it, ir -+ 1, iff), wherever their owner keeps them; the
                // other resonator neighbours are constant offsets from these two:
                // one transmon slab (the owner's P.st rows) or one row away.
                const T2* pl[2] = {nullptr, nullptr};
                size_t sl[2] = {0, 0};
                if (ir > 0) {
                  pl[0] = zrow(cur, it, ir - 1, iff);
                  sl[0] = (size_t)(ir - 1 < P.r_lo ? Pm.st : P.st) * lds;
                }
                if (ir + 1 < Nr) {
                  pl[1] = zrow(cur, it, ir + 1, iff);
                  sl[1] = (size_t)(ir + 1 >= P.r_lo + P.nr ? Pp.st : P.st) * lds;
                }
                // g (b + b^dag)(a + a^dag)
#pragma unroll
                for (int sa = -1; sa <= 1; sa += 2) {
                  const int it2 = it + sa;
                  if (it2 < 0 || it2 >= Nt) continue;
                  const T ct = g * sq[max(it, it2)];
#pragma unroll
                  for (int sb2 = -1; sb2 <= 1; sb2 += 2) {
                    const int ir2 = ir + sb2;
                    if (ir2 < 0 || ir2 >= Nr) continue;
                    if (rwa && sa == sb2) continue;   // RWA: g (b^dag a + b a^dag) only
                    const int h = sb2 > 0;
                    add_row((sa > 0 ? pl[h] + sl[h] : pl[h] - sl[h]) + m0, ct * sq[max(ir, ir2)]);
                  }
                }
                if (three) {
                  // J (a + a^dag)(f + f^dag)
#pragma unroll
                  for (int sa = -1; sa <= 1; sa += 2) {
                    const int ir2 = ir + sa;
                    if (ir2 < 0 || ir2 >= Nr) continue;
                    const T cr = J * sq[max(ir, ir2)];
                    const int h = sa > 0;
#pragma unroll
                    for (int sb2 = -1; sb2 <= 1; sb2 += 2) {
                      const int if2 = iff + sb2;
                      if (if2 < 0 || if2 >= Nf) continue;
                      if (rwa && sa == sb2) continue;   // RWA: J (a^dag f + a f^dag) only
                      add_row((sb2 > 0 ? pl[h] + lds : pl[h] - lds) + m0, cr * sq[max(iff, if2)]);
                    }
                  }
                  // drive on the filter
#pragma unroll
                  for (int sa = -1; sa <= 1; sa += 2) {
                    const int if2 = iff + sa;
                    if (if2 < 0 || if2 >= Nf) continue;
                    if (rwa)
                      add_row_c(own(cur, l + sa) + m0, c * sq[max(iff, if2)], (sa > 0 ? ci : -ci) * sq[max(iff, if2)]);
                    else
                      add_row(own(cur, l + sa) + m0, c * sq[max(iff, if2)]);
                  }
                } else {
                  // drive on the resonator (two modes, C == 1)
#pragma unroll
                  for (int sa = -1; sa <= 1; sa += 2) {
                    const int ir2 = ir + sa;
                    if (ir2 < 0 || ir2 >= Nr) continue;
                    if (rwa)
                      add_row_c(own(cur, l + sa) + m0, c * sq[max(ir, ir2)], (sa > 0 ? ci : -ci) * sq[max(ir, ir2)]);
                    else
                      add_row(own(cur, l + sa) + m0, c * sq[max(ir, ir2)]);
                  }
                }
                // F = -i H_eff z
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  fr[r][u] = hi[u];
                  fi[r][u] = -hr[u];
                }
                if (iro + 1 < dro) {
                  sr[r] = sq[iro + 1];
                  yrp[r] = own(cur, l + 1);
                }
                if (it + 1 < Nt) {
                  sb[r] = sq[it + 1];
                  ybp[r] = own(cur, l + P.st);
                }
              }
              // next local row
              if (++iff == Nf) {
                iff = 0;
                if (++irl == P.nr) {
                  irl = 0;
                  ++it;
                }
              }
            }
            // projection terms: + sr (rZ_s) XT_r + sb (bZ_s) XT_b
            if constexpr (TC == 0 && ZSM == 0 && sizeof(T2) == 8) {
              // FP32 state in L2: k in pairs with 16-byte loads of the Y rows
              // (Mp-wide, 32-byte aligned) and of XT; the padding columns and rows
              // up to Mp are zero, and every accumulator sees the same k order
              for (int k = 0; k < Mq; k += 2) {
                float4 yr2[TR], yb2[TR];
#pragma unroll
                for (int r = 0; r < TR; ++r) {
                  yr2[r] = *reinterpret_cast<const float4*>(yrp[r] + k);
                  yb2[r] = *reinterpret_cast<const float4*>(ybp[r] + k);
                }
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                  const float4* xrp = reinterpret_cast<const float4*>(XT + (k + kk) * Mp + m0);
                  const float4* xbp = reinterpret_cast<const float4*>(XT + MM + (k + kk) * Mp + m0);
                  const float4 xa0 = xrp[0], xa1 = xrp[1], xb0 = xbp[0], xb1 = xbp[1];
                  const T2 xr[4] = {cm<T2>(xa0.x, xa0.y), cm<T2>(xa0.z, xa0.w), cm<T2>(xa1.x, xa1.y),
                                    cm<T2>(xa1.z, xa1.w)};
                  const T2 xb[4] = {cm<T2>(xb0.x, xb0.y), cm<T2>(xb0.z, xb0.w), cm<T2>(xb1.x, xb1.y),
                                    cm<T2>(xb1.z, xb1.w)};
#pragma unroll
                  for (int r = 0; r < TR; ++r) {
                    const T y0x = kk ? yr2[r].z : yr2[r].x, y0y = kk ? yr2[r].w : yr2[r].y;
                    const T y1x = kk ? yb2[r].z : yb2[r].x, y1y = kk ? yb2[r].w : yb2[r].y;
                    const T ar = sr[r] * y0x, ai = sr[r] * y0y, br = sb[r] * y1x, bi = sb[r] * y1y;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                      fr[r][u] = fma(ar, xr[u].x, fma(-ai, xr[u].y, fma(br, xb[u].x, fma(-bi, xb[u].y, fr[r][u]))));
                      fi[r][u] = fma(ar, xr[u].y, fma(ai, xr[u].x, fma(br, xb[u].y, fma(bi, xb[u].x, fi[r][u]))));
                    }
                  }
                }
              }
            } else if constexpr (TC == 0) {
            for (int k = 0; k < M; ++k) {
              T2 xr[4], xb[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                xr[u] = XT[k * Mp + m0 + u];
                xb[u] = XT[MM + k * Mp + m0 + u];
              }
#pragma unroll
              for (int r = 0; r < TR; ++r) {
                const T2 y0 = yrp[r][k], y1 = ybp[r][k];
                const T ar = sr[r] * y0.x, ai = sr[r] * y0.y, br = sb[r] * y1.x, bi = sb[r] * y1.y;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  fr[r][u] = fma(ar, xr[u].x, fma(-ai, xr[u].y, fma(br, xb[u].x, fma(-bi, xb[u].y, fr[r][u]))));
                  fi[r][u] = fma(ar, xr[u].y, fma(ai, xr[u].x, fma(br, xb[u].y, fma(bi, xb[u].x, fi[r][u]))));
                }
              }
            }
            }
            // RK4 update (weights 1/6, 1/3, 1/3, 1/6)
#pragma unroll
            for (int r = 0; r < TR; ++r) {
              const int n = nrow[r];
              if (n < 0) continue;
              T2 zo[4];
              if constexpr (sizeof(T2) == 8) {
                // FP32 state: columns in pairs, 16-byte loads and stores (Z_n rows
                // are 16-byte aligned when M and the trajectory offset are even;
                // accumulator rows, of Mp = 4k columns, always are)
#pragma unroll
                for (int pr = 0; pr < 2; ++pr) {
                  const int u0 = 2 * pr, m = m0 + u0;
                  if (m >= M) {
                    zo[u0] = zo[u0 + 1] = cm<T2>(0, 0);
                    continue;
                  }
                  const bool two = m + 1 < M;
                  const size_t oz = (size_t)n * M + m, oa = (size_t)n * Mp + m;
                  T2 zn0, zn1 = cm<T2>(0, 0);
                  if (zn_vec) {
                    const float4 v = *reinterpret_cast<const float4*>(Zn + oz);
                    zn0 = cm<T2>(v.x, v.y);
                    zn1 = cm<T2>(v.z, v.w);
                  } else {
                    zn0 = Zn[oz];
                    if (two) zn1 = Zn[oz + 1];
                  }
                  float4* ap = reinterpret_cast<float4*>(accg + oa);
                  const T f0r = fr[r][u0], f0i = fi[r][u0], f1r = fr[r][u0 + 1], f1i = fi[r][u0 + 1];
                  if (stage < 3) {
                    if (stage == 0) {
                      *ap = make_float4(f0r, f0i, f1r, f1i);
                    } else {
                      const float4 ac = *ap;
                      *ap = make_float4(fma((T)2, f0r, ac.x), fma((T)2, f0i, ac.y), fma((T)2, f1r, ac.z),
                                        fma((T)2, f1i, ac.w));
                    }
                    zo[u0] = cm<T2>(zn0.x + fma(hs_lo, f0r, hs_hi * f0r), zn0.y + fma(hs_lo, f0i, hs_hi * f0i));
                    zo[u0 + 1] = two ? cm<T2>(zn1.x + fma(hs_lo, f1r, hs_hi * f1r), zn1.y + fma(hs_lo, f1i, hs_hi * f1i))
                                     : cm<T2>(0, 0);
                  } else {
                    const float4 ac = *ap;
                    const T s0r = ac.x + f0r, s0i = ac.y + f0i, s1r = ac.z + f1r, s1i = ac.w + f1i;
                    zo[u0] = cm<T2>(zn0.x + fma(h6_lo, s0r, h6_hi * s0r), zn0.y + fma(h6_lo, s0i, h6_hi * s0i));
                    zo[u0 + 1] = two ? cm<T2>(zn1.x + fma(h6_lo, s1r, h6_hi * s1r), zn1.y + fma(h6_lo, s1i, h6_hi * s1i))
                                     : cm<T2>(0, 0);
                    if (zn_vec) {
                      *reinterpret_cast<float4*>(Zn + oz) = make_float4(zo[u0].x, zo[u0].y, zo[u0 + 1].x, zo[u0 + 1].y);
                    } else {
                      Zn[oz] = zo[u0];
                      if (two) Zn[oz + 1] = zo[u0 + 1];
                    }
                  }
                }
                store4<ZSM>(own(nxt, l0 + r) + m0, zo);
                if constexpr (GRAM_DW == 2)   // column maxima of the next stage input
#pragma unroll
                  for (int u = 0; u < 4; ++u) cmx[u] = fmaxf(cmx[u], fmaxf(fabsf(zo[u].x), fabsf(zo[u].y)));
                continue;
              }
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int m = m0 + u;
                if (m >= M) {
                  zo[u] = cm<T2>(0, 0);
                  continue;
                }
                const size_t oz = (size_t)n * M + m, oa = (size_t)n * Mp + m;
                const T2 zn = Zn[oz];
                if (stage == 0) {
                  accg[oa] = cm<T2>(fr[r][u], fi[r][u]);
                } else if (stage < 3) {
                  const T2 ac = accg[oa];
                  accg[oa] = cm<T2>(fma((T)2, fr[r][u], ac.x), fma((T)2, fi[r][u], ac.y));
                }
                if (stage < 3) {
                  zo[u] = cm<T2>(zn.x + fma(hs_lo, fr[r][u], hs_hi * fr[r][u]),
                                 zn.y + fma(hs_lo, fi[r][u], hs_hi * fi[r][u]));
                } else {
                  const T2 ac = accg[oa];
                  const T s_r = ac.x + fr[r][u], s_i = ac.y + fi[r][u];
                  const T2 z1 = cm<T2>(zn.x + fma(h6_lo, s_r, h6_hi * s_r), zn.y + fma(h6_lo, s_i, h6_hi * s_i));
                  Zn[oz] = z1;
                  zo[u] = z1;
                }
              }
              store4<ZSM>(own(nxt, l0 + r) + m0, zo);
            }
            if constexpr (GRAM_DW == 2)
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (m0 + u < 20) atomicMax(gs_cmax + (gs_par ^ 1) * 20 + m0 + u, __float_as_uint(cmx[u]));
          }
          }
          cur = nxt;
          gs_par ^= 1;
          __syncthreads();
        }
      }
      if (last) break;
    }
    // every CTA is done reading its peers' shared memory before it is reused
    cluster.sync();
  }
  if constexpr (TC > 0 || GRAM_DW == 2) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
  }
}

// Rotating-frame instantiations (lr_fused_rwa.cu).
const void* rwa_kernel_ptr(lr_precision prec, int zs_smem);
cudaError_t rwa_launch(const cudaLaunchConfig_t& cfg, lr_precision prec, int zs_smem, const Args& a);

}  // namespace fz
}  // namespace lr
