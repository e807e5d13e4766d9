#pragma once
// Fused persistent kernel of the sparse-operator engine (FP32 state with the
// FP64-class Gram matrix): the paper's normal-mode model of Sec. S2, or any
// operator set given as CSR rows with time channels, integrated by one launch
// per lr_sparse_integrate call.
//
// A team of C CTAs (a thread-block cluster, C = 1 .. 16) integrates one
// trajectory at a time (persistent over the batch); CTA q of the team owns the
// rows [N q / C, N (q + 1) / C). When the batch has more trajectories than the
// grid has CTAs, teams are single CTAs and each takes an equal span of the
// batch's trajectory-steps instead: a trajectory cut between two CTAs passes
// its state Z_n from one to the other through global memory (release /
// acquire on a per-trajectory flag).
// The stage input Z_s, the operator images Y_k = L_k(t) Z_s and the RK4
// accumulator live in a per-team global region ((3 + K) N Mp complex64) that
// stays L2-resident when the batch in flight is small; r(t) Z_s, needed only
// for the signal, is summed where it is formed. Per stage, each CTA works on its own
// rows (the operator gathers read any row), with two team barriers: B1 after
// the partial sums of G, T_k and the signal over its rows (every CTA then adds
// the team's partials in rank order from distributed shared memory and runs
// the M x M phase itself), B2 after the RK4 update (the new Z_s is visible).
// The phases:
//   C  channel factors Omega(t)^a e^{i q w_d t} of the stage time in FP32
//      (the stage time and the phase reduced to one cycle in FP64);
//   Y  Y_k = L_k(t) Z_s by CSR gathers; at the first stage of every step also
//      r(t) Z_s, the readout signal beta = tr(Z_s^dag r Z_s) and, at recording
//      steps, the photon number |r Z_s|^2 (FP64 sums in a fixed order);
//   P  warp tasks over 4 x 4 tiles: G = Z_s^dag Z_s (upper tiles, exact FP32
//      products in double-word sums) and T_k = Z_s^dag Y_k (FP32), each tile
//      summed over all rows and reduced over the warp by recursive halving;
//   R  G = L D L^dag, L^-1, G^-1 and X_k = G^-1 T_k in double-word FP32
//      (~2^-48 relative), XT_k[l][m] = 1/2 conj(X_k[m][l]) rounded to FP32;
//   F  F = A(t) Z_s (A = -i H_eff: its static diagonal as hi + lo floats, the
//      other entries by CSR gathers) + sum_k Y_k XT_k and the classical RK4
//      stage update; the next stage input goes to the other
//      Z_s buffer, the accumulator and Z_n are updated in place.
#include <cooperative_groups.h>

#include "lr_internal.cuh"
#include "lr_tc.cuh"

namespace lr {
namespace sfz {

namespace cg = cooperative_groups;

constexpr int NT = 512;       // 16 warps at <= 128 registers
constexpr int NWARP = NT / 32;
constexpr int NCH = 10;   // time channels
constexpr int TP = 4;     // phase-P tile edge
constexpr int TR = 4;     // phase-F rows per thread tile
constexpr int PB = 4;     // phase-P row blocks (at most)
// bound of the wait for a head piece (~10 s at 2 GHz); the wait normally ends
// at once, since the previous CTA runs that head first
constexpr long long SPLIT_WAIT_BUDGET = 20000000000LL;

constexpr double INV_2PI = 0.15915494309189533577;
// logistic((t - t0) / s) with t - t0 formed in FP64 and the rest in FP32
__device__ __forceinline__ float logistic_f(double t, double t0, float s) {
  return 1.0f / (1.0f + __expf(-(float)(t - t0) / s));
}
// The envelope Omega(t) of Sec. S2.C in FP32 (the channel factors it enters are
// rounded to FP32)
__device__ __forceinline__ float envelope_f(const PulseDev& P, double tau, double t) {
  if (P.kind == 0) {
    const double s = 0.2 * P.p[2], t0 = 6.0 * s;
    return (float)P.p[0] * logistic_f(t, t0, (float)s) * (1.0f - logistic_f(t, tau - t0, (float)s));
  }
  const double sr = 0.2 * P.p[3], sf = 0.2 * P.p[4], sm = 0.2 * P.p[5];
  return (float)P.p[0] * logistic_f(t, 6.0 * sr, (float)sr) +
         (float)(P.p[1] - P.p[0]) * logistic_f(t, P.p[2], (float)sm) -
         (float)P.p[1] * logistic_f(t, tau - 6.0 * sf, (float)sf);
}

struct Args {
  const int* rowptr;   // [(K + 2) (N + 1)]
  const int* col;
  const float2* valf;
  const float2* valf_a;    // valf with the static diagonal of A (operator 0) set to zero
  const float4* diag_a;    // that diagonal per row as hi + lo floats (re_hi, im_hi, re_lo, im_lo)
  const unsigned char* chan;
  const int* level;
  const PulseDev* pulse;   // per trajectory
  unsigned* err;
  float2* Z;               // state [T][N][M]
  int* flag;               // [T] split schedule: 1 once the head of trajectory t is written
  int split;               // 1: equal spans of trajectory-steps per CTA (cooperative launch)
  float2* scratch;         // per team: Z_s [2][N][Mp], Y [K][N][Mp], accumulator [N][Mp]
  double2* beta;           // [T][max_steps + 1]
  double *pops, *nphot, *trace;
  int N, M, Mp, K, T, n_levels;
  int C;                   // CTAs per team (cluster size; 1 with the split schedule)
  double wd, tau, dt;
  long max_steps, n_rec;
  int pop_every;
  long step0, n_steps;
  // byte offsets in dynamic shared memory
  int o_gd, o_w, o_tred, o_xt, o_misc, o_gpart, o_tsum;
  int o_gs, o_gv;   // Gram on the tensor cores: two slice buffers, V [40][40] double-word
};

constexpr int SG_W = 10;   // slicing warps of the tensor-core Gram (warp SG_W issues the MMAs)

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
__device__ __forceinline__ void dw_add_f(DW& s, float x) {   // s += x (Knuth's two-sum into hi)
  const float t = s.hi + x;
  const float bp = t - s.hi;
  s.lo += (s.hi - (t - bp)) + (x - bp);
  s.hi = t;
}
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
// 1/p for p > 0: one Newton step r + r (1 - p r) in double-word from the FP32 quotient
__device__ __forceinline__ DW dw_recip(DW p) {
  DW r0{1.0f / p.hi, 0.0f};
  const DW one{1.0f, 0.0f};
  const DW e = dw_sum(one, dw_neg(dw_mul(p, r0)));
  return dw_sum(r0, dw_mul(r0, e));
}
struct DWC {
  DW re, im;
};
__device__ __forceinline__ DWC dwc_mul_conj(const DWC& x, const DWC& y) {   // x conj(y)
  DWC r;
  r.re = dw_sum(dw_mul(x.re, y.re), dw_mul(x.im, y.im));
  r.im = dw_sum(dw_mul(x.im, y.re), dw_neg(dw_mul(x.re, y.im)));
  return r;
}
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
__device__ __forceinline__ DW dw_mul_f(DW a, float b) {   // b exact as a double-word
  const float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  DW r;
  r.hi = p + e;
  r.lo = e - (r.hi - p);
  return r;
}
__device__ __forceinline__ DWC dwc_mul_f(const DWC& g, float tx, float ty) {
  DWC r;
  r.re = dw_sum(dw_mul_f(g.re, tx), dw_neg(dw_mul_f(g.im, ty)));
  r.im = dw_sum(dw_mul_f(g.re, ty), dw_mul_f(g.im, tx));
  return r;
}

__device__ __forceinline__ void load4(const float2* p, float2 (&v)[4]) {
  const float4 x = reinterpret_cast<const float4*>(p)[0], y = reinterpret_cast<const float4*>(p)[1];
  v[0] = make_float2(x.x, x.y);
  v[1] = make_float2(x.z, x.w);
  v[2] = make_float2(y.x, y.y);
  v[3] = make_float2(y.z, y.w);
}
__device__ __forceinline__ void store4(float2* p, const float2 (&v)[4]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}

// The same as one 32-byte access per thread (global memory only; p 32-byte
// aligned: rows of Mp = 4j complex64 entries, or column quads of Y_k, in a
// 256-byte aligned region, at column quads m0 = 4i). Half the load and store
// instructions, and half the cache-line lookups, of the 16-byte pairs.
__device__ __forceinline__ void load4w(const float2* p, float2 (&v)[4]) {
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x), "=f"(v[2].y), "=f"(v[3].x),
                 "=f"(v[3].y)
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void store4w(float2* p, const float2 (&v)[4]) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0].x), "f"(v[0].y),
               "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y), "f"(v[3].x), "f"(v[3].y)
               : "memory");
}

// Reduce-scatter of 32 values over the warp (recursive halving, fixed order):
// lane L ends with the total of value L in v[0].
template <typename V, typename Add>
__device__ __forceinline__ void reduce_scatter32(V (&v)[32], int lane, Add add) {
#pragma unroll
  for (int lev = 0; lev < 5; ++lev) {
    const int o = 16 >> lev;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < (16 >> lev); ++k) {
      V keep = up ? v[k + (16 >> lev)] : v[k];
      const V send = up ? v[k] : v[k + (16 >> lev)];
      add(keep, send, o);
      v[k] = keep;
    }
  }
}

// acc[u] += sum over the entries [e, e1) of one CSR row of chi[ch] val * Z[col][m0 + u]
// (vals: the operator's values). Entries go in groups of four: their indices and
// weights first, then the four row loads, then the products, so that four
// gathers are in flight at once (the order of the additions is the entry order
// either way). The caller loads the row extents, several rows' at once. zs:
// Z_s in global memory (32-byte row quads).
__device__ __forceinline__ void row_gather4(const Args& a, const float2* __restrict__ vals, int e, const int e1,
                                            int m0, const float2* __restrict__ zs, const float2* chi,
                                            float2 (&acc)[4]) {
  for (; e + 4 <= e1; e += 4) {
    int c[4];
    float2 w[4], z[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      c[q] = a.col[e + q];
      const float2 ch = chi[a.chan[e + q]], v = vals[e + q];
      w[q] = make_float2(ch.x * v.x - ch.y * v.y, ch.x * v.y + ch.y * v.x);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) load4w(zs + (size_t)c[q] * a.Mp + m0, z[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc[u].x = fmaf(w[q].x, z[q][u].x, fmaf(-w[q].y, z[q][u].y, acc[u].x));
        acc[u].y = fmaf(w[q].x, z[q][u].y, fmaf(w[q].y, z[q][u].x, acc[u].y));
      }
  }
  for (; e < e1; ++e) {
    const float2 ch = chi[a.chan[e]], v = vals[e];
    const float wr = ch.x * v.x - ch.y * v.y, wi = ch.x * v.y + ch.y * v.x;
    float2 z[4];
    load4w(zs + (size_t)a.col[e] * a.Mp + m0, z);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc[u].x = fmaf(wr, z[u].x, fmaf(-wi, z[u].y, acc[u].x));
      acc[u].y = fmaf(wr, z[u].y, fmaf(wi, z[u].x, acc[u].y));
    }
  }
}

// y[k][u] = sum over the row n of operator 1 + k0 + k (k < nk <= KM; operators
// 1 .. K are the jumps, K + 1 the readout) of chi[ch] val * Z[col][m0 + u].
// The operators' rows go in lockstep (entry j
// of every operator, then entry j + 1), so that their extents, indices,
// weights and row loads are in flight together; within an operator the
// additions keep the entry order.
template <int KM>
__device__ __forceinline__ void gather_ops(const Args& a, int k0, int nk, int n, int m0,
                                           const float2* __restrict__ zs, const float2* chi, float2 (&y)[KM][4]) {
  int e[KM], e1[KM];
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    e[k] = e1[k] = 0;
    if (k < nk) {
      const int* rp = a.rowptr + (size_t)(1 + k0 + k) * (a.N + 1);
      e[k] = rp[n];
      e1[k] = rp[n + 1];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) y[k][u] = make_float2(0.f, 0.f);
  }
  int len = 0;
#pragma unroll
  for (int k = 0; k < KM; ++k) len = max(len, e1[k] - e[k]);
  for (int j = 0; j < len; ++j) {
    int c[KM];
    float2 w[KM], z[KM][4];
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      c[k] = -1;
      if (e[k] + j < e1[k]) {
        const int ei = e[k] + j;
        c[k] = a.col[ei];
        const float2 ch = chi[a.chan[ei]], v = a.valf[ei];
        w[k] = make_float2(ch.x * v.x - ch.y * v.y, ch.x * v.y + ch.y * v.x);
      }
    }
#pragma unroll
    for (int k = 0; k < KM; ++k)
      if (c[k] >= 0) load4(zs + (size_t)c[k] * a.Mp + m0, z[k]);
#pragma unroll
    for (int k = 0; k < KM; ++k)
      if (c[k] >= 0)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          y[k][u].x = fmaf(w[k].x, z[k][u].x, fmaf(-w[k].y, z[k][u].y, y[k][u].x));
          y[k][u].y = fmaf(w[k].x, z[k][u].y, fmaf(w[k].y, z[k][u].x, y[k][u].y));
        }
  }
}

// Fixed-order block sum of NV double-word values (warp shuffles, then the warp
// partials in warp order); thread 0 returns the totals as doubles. red: NWARP
// * NV float2 of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum_dw(DW (&v)[NV], float2* red, int tid, double (&out)[NV]) {
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c)
    for (int o = 16; o > 0; o >>= 1) {
      DW t;
      t.hi = __shfl_down_sync(0xffffffffu, v[c].hi, o);
      t.lo = __shfl_down_sync(0xffffffffu, v[c].lo, o);
      dw_add(v[c], t);
    }
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) red[warp * NV + c] = make_float2(v[c].hi, v[c].lo);
  __syncthreads();
  if (tid == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      DW s{0.f, 0.f};
      for (int w = 0; w < NWARP; ++w) {
        const float2 p = red[w * NV + c];
        dw_add(s, DW{p.x, p.y});
      }
      out[c] = (double)s.hi + (double)s.lo;
    }
}

// TEAM = false: teams of one CTA (C = 1 known at compile time; the equal-span
// schedule); TEAM = true: clusters of a.C CTAs.
template <bool TEAM, bool GTC>
__global__ void __launch_bounds__(NT, 1) sf_kernel(const Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  // tensor-core Gram (GTC): TMEM base, mbarriers (MMA commits and chunk fills per
  // buffer, TMEM free after a readout) and column maxima [2][20] by stage parity
  __shared__ __align__(8) unsigned long long gbar_s[5];
  __shared__ uint32_t gslot;
  __shared__ uint32_t gcmax[2][20];
  __shared__ short2 tri[LR_MAX_RANK * (LR_MAX_RANK + 1) / 2];
  __shared__ float2 chi[NCH];
  __shared__ double red[NWARP * 4];
  __shared__ int task_ctr[2];   // phase-P task counters of alternate row blocks
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = a.N, M = a.M, Mp = a.Mp, K = a.K, MM = Mp * Mp;
  const int Mq = (M + 3) / 4 * 4;
  const int ldg = Mp + 1;
  for (int i = tid; i < LR_MAX_RANK; i += NT)
    for (int j = 0; j <= i; ++j) tri[i * (i + 1) / 2 + j] = make_short2((short)i, (short)j);
  const uint32_t gbar[2] = {smem_u32(&gbar_s[0]), smem_u32(&gbar_s[1])};
  const uint32_t gfill[2] = {smem_u32(&gbar_s[2]), smem_u32(&gbar_s[3])};
  const uint32_t gfree = smem_u32(&gbar_s[4]);
  uint32_t tmem = 0;
  // phases waited: commits (slicing warps), fills (issuing warp), TMEM frees (issuing warp)
  uint32_t gph[2] = {0u, 0u}, gfph[2] = {0u, 0u}, gtf = 0u;
  bool gused = false;   // the issuing warp: TMEM held a readout before
  int gpar = 0;         // stage parity of the column maxima
  if constexpr (GTC) {
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gbar[0]), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gbar[1]), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gfill[0]), "r"(SG_W * 32));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gfill[1]), "r"(SG_W * 32));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gfree), "r"(SG_W * 32));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&gslot)),
                   "r"(512));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem = gslot;
  }
  double2* Gd = reinterpret_cast<double2*>(smem + a.o_gd);   // [Mp][Mp+1]  G -> L -> G^-1
  double2* W = reinterpret_cast<double2*>(smem + a.o_w);     // [Mp][Mp+1]  L^-1
  float2* Tred = reinterpret_cast<float2*>(smem + a.o_tred);  // [K][Mp*Mp]  T_k over this CTA's rows
  float2* XT = reinterpret_cast<float2*>(smem + a.o_xt);      // [K][Mp][Mp] (l, m)
  // [0] not-PD flag, [8..11) signal partials (Re, Im beta, photons), [32..64) 1/D,
  // [64..96) population partials
  double* misc = reinterpret_cast<double*>(smem + a.o_misc);
  double2* gpart = reinterpret_cast<double2*>(smem + a.o_gpart);   // [Mp][Mp]  G over this CTA's rows
  float2* tsum = reinterpret_cast<float2*>(smem + a.o_tsum);       // [K][Mp*Mp]  T_k of the team
  cg::cluster_group cluster = cg::this_cluster();
  const int C = TEAM ? a.C : 1;
  const int q = C > 1 ? (int)cluster.block_rank() : 0;
  const int team = blockIdx.x / C, n_teams = gridDim.x / C;
  const int r_lo = (int)((long long)N * q / C), r_hi = (int)((long long)N * (q + 1) / C), NR = r_hi - r_lo;
  auto team_sync = [&]() {
    if (C > 1)
      cluster.sync();
    else
      __syncthreads();
  };
  // rank r's copy of a shared-memory object of this CTA
  auto at_rank = [&](auto* p, int r) { return r == q ? p : cluster.map_shared_rank(p, r); };
  const size_t zsb = (size_t)N * Mp;
  float2* zs0 = a.scratch + (size_t)team * (size_t)(3 + K) * zsb;
  // Y_1 .. Y_K (r Z_s is only summed, never stored), each in column quads: entry
  // (n, m) at yq(n, m), so that a warp's loads of one quad over 32 consecutive
  // rows (phase P) cover 1 KB of contiguous memory instead of 32 cache lines
  float2* ybuf = zs0 + 2 * zsb;
  auto yq = [N](int n, int m) { return (size_t)(m >> 2) * N * 4 + (size_t)n * 4 + (m & 3); };
  float2* accg = zs0 + (2 + K) * zsb;
  const double dt = a.dt;
  const int pe = a.pop_every;

  // ---- Gram matrix of the own rows on the tensor cores (GTC; Mp = 20): exact
  // bf16 slices of the scaled columns (see lr_tc.cuh), chunks of GS_CH rows,
  // accumulation windows of GS_MAXR rows (the FP32 sums stay exact). Warps
  // 0 .. SG_W-1 slice into the two buffers, arrive on the buffer's fill
  // mbarrier and, at the end of each window, read the window's slice-pair sums
  // out of tensor memory into V (double-word) and free it; warp SG_W waits on
  // the fills (and, before a window, on the free) and issues the MMAs; the
  // other warps go on to the T tiles. The slicing warps then form G over the
  // own rows into gpart.
  auto gram_tc = [&](int cur_buf) {
    if (tid < 20) gcmax[gpar ^ 1][tid] = 0u;   // phase F fills it for the next stage
    const int n_ch = (NR + GS_CH - 1) / GS_CH;
    const int chw = GS_MAXR / GS_CH;            // chunks per window
    const float2* zc = zs0 + (size_t)cur_buf * zsb;
    if (warp < SG_W) {
      constexpr int GTASK = (GS_CH / 8) * 5;
      constexpr int GT = (GTASK + SG_W - 1) / SG_W;
      float gsc[GT];
      int gcol[GT];
#pragma unroll
      for (int t = 0; t < GT; ++t) {
        const int task = (warp + SG_W * t) % GTASK, ag = task % 5, ar = ag * 8 + (lane >> 2);
        gcol[t] = ar;
        int ex = 0;
        frexpf(__uint_as_float(gcmax[gpar][ar < 20 ? ar : ar - 20]), &ex);
        gsc[t] = ldexpf(1.0f, -ex);   // |value| scale < 1, exact
      }
      auto gload = [&](int ch, float (&v)[GT][2]) {
#pragma unroll
        for (int t = 0; t < GT; ++t) {
          const int task = (warp + SG_W * t) % GTASK, rg = task / 5, ar = gcol[t];
          const int j = ar < 20 ? ar : ar - 20, r0 = ch * GS_CH + rg * 8 + 2 * (lane & 3);
          const float* z0 = reinterpret_cast<const float*>(zc + (size_t)(r_lo + (r0 < NR ? r0 : 0)) * Mp + j) +
                            (ar < 20 ? 0 : 1);
          const float* z1 = reinterpret_cast<const float*>(zc + (size_t)(r_lo + (r0 + 1 < NR ? r0 + 1 : 0)) * Mp + j) +
                            (ar < 20 ? 0 : 1);
          v[t][0] = r0 < NR ? *z0 : 0.f;
          v[t][1] = r0 + 1 < NR ? *z1 : 0.f;
        }
      };
      // every commit is waited on once, in chunk order (a parity wait tells
      // adjacent phases apart only)
      int waited = -1;
      auto wait_chunk = [&](int c) {
        while (waited < c) {
          ++waited;
          const int b = waited & 1;
          if (!mbar_wait(gbar[b], gph[b] & 1u)) set_error(a.err, DEV_TIMEOUT);
          ++gph[b];
        }
      };
      DW* V = reinterpret_cast<DW*>(smem + a.o_gv);   // [40][40]
      const int qd = warp & 3, nq = (SG_W - qd + 3) / 4, rw = warp >> 2, m = qd * 32 + lane;
      const int sA = m / 40, aa = m % 40, sB = 3 + m / 40;
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
        if (ch >= 2) wait_chunk(ch - 2);   // the MMAs of chunk ch - 2 are done with buffer b
        tc_fence_after();
        unsigned char* buf = smem + a.o_gs + b * GS_BUF;
#pragma unroll
        for (int sl = 0; sl < GS_N; ++sl)
#pragma unroll
          for (int t = 0; t < GT; ++t) {
            if (warp + SG_W * t >= GTASK) continue;   // uniform across the warp
            const int task = warp + SG_W * t, rg = task / 5, ag = task % 5;
            const float y0 = gv[t][0] * 128.f, y1 = gv[t][1] * 128.f;
            // round to the nearest integer by adding and subtracting 1.5 2^23
            const float k0 = __fsub_rn(__fadd_rn(y0, 12582912.f), 12582912.f);
            const float k1 = __fsub_rn(__fadd_rn(y1, 12582912.f), 12582912.f);
            gv[t][0] = y0 - k0;
            gv[t][1] = y1 - k1;
            reinterpret_cast<uint32_t*>(buf + rg * GS_LBO + (sl * 5 + ag) * 128)[lane] =
                __byte_perm(__float_as_uint(k0), __float_as_uint(k1), 0x7632);
          }
        async_proxy_fence();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(gfill[b]) : "memory");
        if ((ch + 1) % chw == 0 || ch + 1 == n_ch) {
          // end of a window: its slice-pair sums D_st, s <= t, s + t <= 8, from TMEM
          // lane m (row a = m % 40 of slices s = m / 40 and s + 3) into V, V[a][b]
          // += sum c_st 2^-7(s+t) D_st[a][b] (c_st = 1/2 for s = t, else 1), so that
          // G's real form is V + V^T; lanes m < 40, < 80, < 120 add in that order
          const int win = ch / chw;
          wait_chunk(ch);
          tc_fence_after();
          for (int it2 = 0; it2 < 3; ++it2) {
            const int bk = rw + nq * it2, b0 = bk * 8;
            const bool has = bk < 5;   // uniform within the warp
            DW cA[8], cB[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) cA[u] = cB[u] = DW{0.f, 0.f};
            if (has) {
              const uint32_t lane_base = tmem + ((uint32_t)(qd * 32) << 16);
#pragma unroll
              for (int g = 0; g < 3; ++g) {
                uint32_t v[4][8];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                  const int t = 4 * g + qq;
                  const int col = t < 6 ? GS_D0 + t * 40 + b0
                                        : (t < 8 ? GS_D1 + (t - 6) * 40 + b0 : GS_D2 + (t - 8) * 40 + b0);
                  if (t < 11)
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                        : "=r"(v[qq][0]), "=r"(v[qq][1]), "=r"(v[qq][2]), "=r"(v[qq][3]), "=r"(v[qq][4]),
                          "=r"(v[qq][5]), "=r"(v[qq][6]), "=r"(v[qq][7])
                        : "r"(lane_base + (uint32_t)col));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                  const int t = 4 * g + qq;
                  if (t >= 11) continue;
                  const int s0 = t < 8 ? sA : sB, tt = t < 8 ? t : t - 5;
                  if (m < 120 && tt >= s0 && s0 + tt <= 8) {
                    const float w = __int_as_float((127 - 7 * (s0 + tt) - (s0 == tt ? 1 : 0)) << 23);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                      if (t < 8)
                        dw_add_f(cA[u], w * __uint_as_float(v[qq][u]));
                      else
                        dw_add_f(cB[u], w * __uint_as_float(v[qq][u]));
                    }
                  }
                }
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) dw_add(cA[u], cB[u]);
            }
            for (int round = 0; round < 3; ++round) {
              if (has && m < 120 && sA == round)
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  DW& dst = V[aa * 40 + b0 + u];
                  if (win == 0 && round == 0) {
                    dst = cA[u];
                  } else {
                    DW x = dst;
                    dw_add(x, cA[u]);
                    dst = x;
                  }
                }
              asm volatile("bar.sync 1, %0;" ::"r"(SG_W * 32) : "memory");
            }
          }
          tc_fence_before();
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(gfree) : "memory");
        }
      }
      // G over the own rows from V: S[a][b] = V[a][b] + V[b][a] for the 820
      // entries G needs ([0, 210) (i, j), [210, 420) (20+i, 20+j), i <= j;
      // [420, 820) (i, 20+j)), then G_ij = 2^(e_i + e_j - 14) (S[i][j] +
      // S[20+i][20+j] + i (S[i][20+j] - S[j][20+i])) into gpart, both triangles
      DW* Sb = reinterpret_cast<DW*>(W);
      const int gt = tid;   // 0 .. SG_W * 32 - 1
      for (int e = gt; e < 820; e += SG_W * 32) {
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
      asm volatile("bar.sync 1, %0;" ::"r"(SG_W * 32) : "memory");
      for (int e = gt; e < 210; e += SG_W * 32) {
        const int i = tri[e].y, j = tri[e].x;   // i <= j
        int ei = 0, ej = 0;
        frexpf(__uint_as_float(gcmax[gpar][i]), &ei);
        frexpf(__uint_as_float(gcmax[gpar][j]), &ej);
        const double sc = ldexp(1.0, ei + ej - 14);
        DW re = Sb[e], im = Sb[420 + i * 20 + j];
        dw_add(re, Sb[210 + e]);
        const DW n2 = Sb[420 + j * 20 + i];
        dw_add(im, DW{-n2.hi, -n2.lo});
        const double gr = ((double)re.hi + (double)re.lo) * sc, gi = ((double)im.hi + (double)im.lo) * sc;
        gpart[i * Mp + j] = make_double2(gr, gi);
        gpart[j * Mp + i] = make_double2(gr, -gi);
      }
    } else if (warp == SG_W) {
      // the issuing warp
      for (int ch = 0; ch < n_ch; ++ch) {
        const int b = ch & 1;
        if (ch % chw == 0) {   // a window starts: the previous readout has left TMEM
          if (gused) {
            if (!mbar_wait(gfree, gtf & 1u)) set_error(a.err, DEV_TIMEOUT);
            ++gtf;
          }
          gused = true;
        }
        if (!mbar_wait(gfill[b], gfph[b] & 1u)) set_error(a.err, DEV_TIMEOUT);
        ++gfph[b];
        if (lane == 0) {
          tc_fence_after();
          const uint32_t bb = smem_u32(smem + a.o_gs + b * GS_BUF);
          for (int ks = 0; ks < GS_CH / 16; ++ks) {
            const uint32_t ko = bb + (uint32_t)(ks * 2 * GS_LBO);
            const uint32_t acc = (ch % chw != 0 || ks > 0) ? 1u : 0u;
            const uint64_t d0 = tc_desc(ko, GS_LBO, 128);              // m-rows 0..127
            const uint64_t d2 = tc_desc(ko + 15 * 128, GS_LBO, 128);   // m-rows 120..247
            gs_mma(tmem + GS_D0, d0, d0, gs_idesc(240), acc);
            gs_mma(tmem + GS_D1, d0, tc_desc(ko + 30 * 128, GS_LBO, 128), gs_idesc(80), acc);
            gs_mma(tmem + GS_D2, d2, d2, gs_idesc(128), acc);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(gbar[b])
                       : "memory");
        }
        __syncwarp();
      }
    }
  };
  // Steps [s_a, s_b) (relative to step0) of trajectory tj, and the signal at
  // s_b unless the piece is a head (its continuation evaluates it). A tail
  // piece first waits for the head's state; a head piece publishes it.
  auto piece = [&](int tj, long s_a, long s_b, bool head, bool tail) {
    const PulseDev pulse = a.pulse[tj];
    float2* Zn = a.Z + (size_t)tj * N * M;
    if (tail) {
      if (tid == 0) {
        const long long t0 = clock64();
        volatile int* f = a.flag + tj;
        while (*f == 0) {
          if (clock64() - t0 > SPLIT_WAIT_BUDGET) {
            set_error(a.err, DEV_TIMEOUT);
            break;
          }
        }
        __threadfence();
        *f = 0;   // consumed: ready for the next launch
      }
      __syncthreads();
    }
    if (C > 1) cluster.sync();   // the team is done with the previous trajectory's rows
    for (long long e = (long long)r_lo * Mp + tid; e < (long long)r_hi * Mp; e += NT) {
      const int n = (int)(e / Mp), m = (int)(e - (long long)n * Mp);
      zs0[e] = m < M ? __ldcg(Zn + (size_t)n * M + m) : make_float2(0.f, 0.f);
    }
    if constexpr (GTC) {   // column maxima of the own rows just loaded
      if (tid < 20) gcmax[gpar][tid] = 0u;
      __syncthreads();
      if (tid < 500) {
        const int j = tid % 20;
        float mx = 0.f;
        for (int n = r_lo + tid / 20; n < r_hi; n += 25) {
          const float2 v = zs0[(size_t)n * Mp + j];
          mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        atomicMax(&gcmax[gpar][j], __float_as_uint(mx));
      }
    }
    team_sync();
    int cur = 0;
    // rank 0 adds the team's signal and population partials (after a team
    // barrier) and writes the step's records
    auto publish = [&](long step, bool record) {
      if (q != 0 || tid != 0) return;
      double sg[3] = {0.0, 0.0, 0.0};
      for (int r = 0; r < C; ++r) {
        const double* mr = at_rank(misc, r);
        for (int c = 0; c < 3; ++c) sg[c] += mr[8 + c];
      }
      a.beta[(size_t)tj * (a.max_steps + 1) + step] = mk(sg[0], sg[1]);
      if (!isfinite(sg[0]) || !isfinite(sg[1])) set_error(a.err, DEV_NONFINITE);
      if (!record) return;
      const long rec = step / pe;
      a.nphot[(size_t)tj * a.n_rec + rec] = sg[2];
      double tr = 0.0;
      for (int lv = 0; lv < a.n_levels; ++lv) {
        double v = 0.0;
        for (int r = 0; r < C; ++r) v += at_rank(misc, r)[64 + lv];
        a.pops[((size_t)tj * a.n_rec + rec) * a.n_levels + lv] = v;
        tr += v;
      }
      a.trace[(size_t)tj * a.n_rec + rec] = tr;
    };
    const long s_end = a.step0 + s_b;
    for (long step = a.step0 + s_a;; ++step) {
      const bool last = step == s_end;
      if (last && head) break;
      for (int stage = 0; stage < 4; ++stage) {
        const bool record = stage == 0 && (step % pe) == 0;
        const float2* zc = zs0 + (size_t)cur * zsb;
        // ================= C: channel factors of the stage time
        if (tid < NCH) {
          const double ts = (double)step * dt + (stage == 0 ? 0.0 : (stage == 3 ? dt : 0.5 * dt));
          const int ach = tid / 5, q = tid % 5 - 2;
          const float om = ach ? envelope_f(pulse, a.tau, ts) : 1.0f;
          // e^{i q w_d t}: the phase in cycles, reduced to [-1/2, 1/2] in FP64, then
          // sine and cosine of the reduced phase in FP32 (FP64 transcendentals hold
          // the FP64 pipe for tens of cycles per warp instruction on this GPU)
          const double cyc = (double)q * a.wd * ts * INV_2PI;
          const float x = (float)(cyc - rint(cyc));
          float sn, cs;
          sincospif(2.0f * x, &sn, &cs);
          chi[tid] = make_float2(om * cs, om * sn);
        }
        if (tid == 0) task_ctr[0] = task_ctr[1] = 0;
        __syncthreads();
        // ================= Y: operator images, readout signal
        {
          const int nk = stage == 0 ? K + 1 : K;
          const int mq = Mq / 4;
          // Re, Im tr(Z^dag r Z), |r Z|^2: exact FP32 products in double-word sums
          DW s3[3] = {DW{0.f, 0.f}, DW{0.f, 0.f}, DW{0.f, 0.f}};
          for (int t = tid; t < NR * mq * nk; t += NT) {
            const int k = t / (NR * mq);
            const int rem = t - k * NR * mq, nl = rem / mq, m0 = (rem - nl * mq) * 4, n = r_lo + nl;
            float2 y[1][4];
            gather_ops<1>(a, k, 1, n, m0, zc, chi, y);
            if (k < K) store4(ybuf + (size_t)k * zsb + yq(n, m0), y[0]);
            if (k == K) {
              float2 z[4];
              load4(zc + (size_t)n * Mp + m0, z);
#pragma unroll
              for (int u = 0; u < 4; ++u) {   // padding columns are zero
                dw_add_prod(s3[0], z[u].x, y[0][u].x);
                dw_add_prod(s3[0], z[u].y, y[0][u].y);
                dw_add_prod(s3[1], z[u].x, y[0][u].y);
                dw_add_prod(s3[1], -z[u].y, y[0][u].x);
                dw_add_prod(s3[2], y[0][u].x, y[0][u].x);
                dw_add_prod(s3[2], y[0][u].y, y[0][u].y);
              }
            }
          }
          if (stage == 0) {
            double tot[3];
            block_sum_dw<3>(s3, reinterpret_cast<float2*>(red), tid, tot);
            if (tid == 0)
              for (int c = 0; c < 3; ++c) misc[8 + c] = tot[c];
          }
          if (record) {
            // level populations: warp per level, fixed order over the rows
            for (int lv = warp; lv < a.n_levels; lv += NWARP) {
              double s = 0.0;
              for (int n = r_lo + lane; n < r_hi; n += 32) {
                if (a.level[n] != lv) continue;
                const float2* z = zc + (size_t)n * Mp;
                for (int m = 0; m < M; ++m) s += (double)z[m].x * z[m].x + (double)z[m].y * z[m].y;
              }
              for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
              if (lane == 0) misc[64 + lv] = s;
            }
          }
          __syncthreads();
        }
        if (last) {
          team_sync();
          publish(step, record);
          break;
        }
        // ================= P: Gram and T_k tiles over all rows
        {
          const int nt_ = Mq / TP;
          const int n_g = GTC ? 0 : nt_ * (nt_ + 1) / 2, n_t = K * nt_ * nt_;
          if constexpr (GTC) gram_tc(cur);
          // The rows go in PB blocks, each swept by all tasks before the next, so
          // that a block's columns of Z_s and Y_k stay in L2 while the tasks re-read
          // them (the whole of a trajectory's Z_s and Y_k, 0.96 MB at N = 2000, M =
          // 20, times the CTAs in flight exceeds L2); the blocks' sums are added in
          // block order, a barrier apart. (The tensor-core Gram's slicing warps keep
          // to their own schedule: one block.)
          const int nb = GTC ? 1 : max(1, min(PB, NR / 256));   // blocks of at least 256 rows
          for (int blk = 0; blk < nb; ++blk) {
          const int b_lo = r_lo + (int)((long long)NR * blk / nb), b_hi = r_lo + (int)((long long)NR * (blk + 1) / nb);
          for (;;) {
            int task = 0;
            if (lane == 0) task = atomicAdd(&task_ctr[blk & 1], 1);
            task = __shfl_sync(0xffffffffu, task, 0);
            if (task >= n_g + n_t) break;
            if (task < n_g) {
              int ti = 0, rem = task;
              while (rem >= nt_ - ti) {
                rem -= nt_ - ti;
                ++ti;
              }
              const int tj2 = ti + rem, i0 = ti * TP, j0 = tj2 * TP;
              DW acc[TP][TP][2];
#pragma unroll
              for (int i = 0; i < TP; ++i)
#pragma unroll
                for (int j = 0; j < TP; ++j) acc[i][j][0] = acc[i][j][1] = DW{0.f, 0.f};
              for (int n = b_lo + lane; n < b_hi; n += 32) {
                float2 zi[4], zj[4];
                load4w(zc + (size_t)n * Mp + i0, zi);
                load4w(zc + (size_t)n * Mp + j0, zj);
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                  for (int j = 0; j < TP; ++j) {   // conj(zi) zj
                    if (ti == tj2 && j < i) continue;
                    dw_add_prod(acc[i][j][0], zi[i].x, zj[j].x);
                    dw_add_prod(acc[i][j][0], zi[i].y, zj[j].y);
                    dw_add_prod(acc[i][j][1], zi[i].x, zj[j].y);
                    dw_add_prod(acc[i][j][1], -zi[i].y, zj[j].x);
                  }
              }
              DW v[32];
#pragma unroll
              for (int i = 0; i < TP; ++i)
#pragma unroll
                for (int j = 0; j < TP; ++j)
#pragma unroll
                  for (int c = 0; c < 2; ++c) v[(i * 4 + j) * 2 + c] = acc[i][j][c];
              reduce_scatter32(v, lane, [](DW& keep, const DW& send, int o) {
                DW t;
                t.hi = __shfl_xor_sync(0xffffffffu, send.hi, o);
                t.lo = __shfl_xor_sync(0xffffffffu, send.lo, o);
                dw_add(keep, t);
              });
              const int i = i0 + (lane >> 3), j = j0 + ((lane >> 1) & 3), c = lane & 1;
              const double val = (double)v[0].hi + (double)v[0].lo;
              // G[i][j] and its conjugate G[j][i] over this CTA's rows (the diagonal's
              // imaginary part is zero), summed over the row blocks in order
              double* gp = reinterpret_cast<double*>(gpart);
              if (i < j) {
                const double lower = c ? -val : val;
                gp[2 * (i * Mp + j) + c] = blk ? gp[2 * (i * Mp + j) + c] + val : val;
                gp[2 * (j * Mp + i) + c] = blk ? gp[2 * (j * Mp + i) + c] + lower : lower;
              } else if (i == j) {
                const double d = c ? 0.0 : val;
                gp[2 * (i * Mp + i) + c] = blk ? gp[2 * (i * Mp + i) + c] + d : d;
              }
            } else {
              const int t2 = task - n_g, k = t2 / (nt_ * nt_), r2 = t2 - k * nt_ * nt_, ti = r2 / nt_,
                        tj2 = r2 - ti * nt_;
              const int i0 = ti * TP, j0 = tj2 * TP;
              const float2* yk = ybuf + (size_t)k * zsb;
              float tr_[TP][TP], ti_[TP][TP];
#pragma unroll
              for (int i = 0; i < TP; ++i)
#pragma unroll
                for (int j = 0; j < TP; ++j) tr_[i][j] = ti_[i][j] = 0.f;
              for (int n = b_lo + lane; n < b_hi; n += 32) {
                float2 z[4], y[4];
                load4w(zc + (size_t)n * Mp + i0, z);
                load4w(yk + yq(n, j0), y);
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                  for (int j = 0; j < TP; ++j) {   // conj(z_i) y_j
                    tr_[i][j] = fmaf(z[i].x, y[j].x, fmaf(z[i].y, y[j].y, tr_[i][j]));
                    ti_[i][j] = fmaf(z[i].x, y[j].y, fmaf(-z[i].y, y[j].x, ti_[i][j]));
                  }
              }
              float v[32];
#pragma unroll
              for (int i = 0; i < TP; ++i)
#pragma unroll
                for (int j = 0; j < TP; ++j) {
                  v[(i * 4 + j) * 2] = tr_[i][j];
                  v[(i * 4 + j) * 2 + 1] = ti_[i][j];
                }
              reduce_scatter32(v, lane, [](float& keep, const float& send, int o) {
                keep += __shfl_xor_sync(0xffffffffu, send, o);
              });
              const int i = i0 + (lane >> 3), j = j0 + ((lane >> 1) & 3), c = lane & 1;
              float* tp = reinterpret_cast<float*>(Tred) + 2 * (k * MM + i * Mp + j) + c;
              *tp = blk ? *tp + v[0] : v[0];
            }
          }
          if (blk + 1 < nb) {
            __syncthreads();   // block blk's sums are in place; its counter is free
            if (tid == 0) task_ctr[blk & 1] = 0;   // next used by block blk + 2, a barrier later
          }
          }
        }
        // ================= B1: the team's partials are visible
        team_sync();
        if (stage == 0) publish(step, record);
        // ================= R: G = L D L^dag, L^-1, G^-1 (double-word FP32), XT_k
        {
          DWC* Gw = reinterpret_cast<DWC*>(Gd);
          DWC* Ww = reinterpret_cast<DWC*>(W);
          DW* dinv = reinterpret_cast<DW*>(misc + 32);   // [M] 1 / D[k]
          float* diag0 = reinterpret_cast<float*>(W);    // W[k][0] slot: the diagonal of G
          if (tid == 0) misc[0] = 0.0;
          // T_k of the team: the partials added in rank order (the same in every CTA)
          for (int e = tid; e < K * MM; e += NT) {
            float2 v = at_rank(Tred, 0)[e];
            for (int r = 1; r < C; ++r) {
              const float2 u = at_rank(Tred, r)[e];
              v.x += u.x;
              v.y += u.y;
            }
            tsum[e] = v;
          }
          for (int e = tid; e < M * (M + 1) / 2; e += NT) {
            const int i = tri[e].x, j = tri[e].y;
            double2 v = at_rank(gpart, 0)[i * Mp + j];
            for (int r = 1; r < C; ++r) {
              const double2 u = at_rank(gpart, r)[i * Mp + j];
              v.x += u.x;
              v.y += u.y;
            }
            DWC g;
            g.re = dw_make(v.x);
            g.im = dw_make(v.y);
            if (i == j) diag0[i * ldg * 4] = (float)v.x;
            Gw[i * ldg + j] = g;
          }
          auto pivot = [&](int k) {
            const DW piv = Gw[k * ldg + k].re;
            if (!(piv.hi > 1e-13f * diag0[k * ldg * 4]) || !isfinite(piv.hi) || piv.hi < 1e-30f) {
              misc[0] = 1.0;
              dinv[k] = DW{1.0f, 0.0f};
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
            for (int e = tid; e < w * (w + 1) / 2; e += NT) {
              const int i = k + 1 + tri[e].x, j = k + 1 + tri[e].y;
              const DWC t = dwc_scale(dwc_mul_conj(Gw[i * ldg + k], Gw[j * ldg + k]), rk);
              Gw[i * ldg + j] = dwc_sub(Gw[i * ldg + j], t);
            }
            if (tid == 0 && k + 1 < M) pivot(k + 1);
            __syncthreads();
          }
          if (tid == 0 && misc[0] != 0.0) set_error(a.err, DEV_NOT_PD);
          // W = L^-1 by columns (warp j mod NWARP, lane i = row i)
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
          // G^-1 = W^dag D^-1 W in double-word, into the storage of L (no longer needed)
          for (int e = tid; e < M * M; e += NT) {
            const int i = e / M, j = e - i * M;
            if (i > j) continue;
            DWC acc;
            acc.re.hi = acc.re.lo = acc.im.hi = acc.im.lo = 0.0f;
            for (int k = j; k < M; ++k)
              acc = dwc_add(acc, dwc_scale(dwc_mul_conj(Ww[k * ldg + j], Ww[k * ldg + i]), dinv[k]));
            Gw[i * ldg + j] = acc;
            if (i != j) {
              acc.im = dw_neg(acc.im);
              Gw[j * ldg + i] = acc;
            }
          }
          __syncthreads();
          // XT_k[l][m] = 1/2 conj(X_k[m][l]), X_k = G^-1 T_k (the 1/2 of Eq. S5), in
          // double-word sums: G^-1 has entries up to 1 / p_M, and a product rounded
          // to FP32 first would lose the small columns to cancellation
          for (int e = tid; e < K * Mq * Mq; e += NT) {
            const int k = e / (Mq * Mq), lq = e - k * (Mq * Mq), l = lq / Mq, m = lq - l * Mq;
            float xr = 0.f, xi = 0.f;
            if (l < M && m < M) {
              const float2* Tk = tsum + k * MM;
              DWC acc;
              acc.re.hi = acc.re.lo = acc.im.hi = acc.im.lo = 0.0f;
              for (int j = 0; j < M; ++j) {
                const float2 t = Tk[j * Mp + l];
                acc = dwc_add(acc, dwc_mul_f(Gw[m * ldg + j], t.x, t.y));
              }
              xr = acc.re.hi + acc.re.lo;
              xi = acc.im.hi + acc.im.lo;
            }
            XT[k * MM + l * Mp + m] = make_float2(0.5f * xr, -0.5f * xi);
          }
          __syncthreads();
        }
        // ================= F: A Z_s + projection, RK4 stage update
        {
          const double hsd = stage == 2 ? dt : 0.5 * dt, h6d = dt / 6.0;
          const float hs_hi = (float)hsd, hs_lo = (float)(hsd - (double)hs_hi);
          const float h6_hi = (float)h6d, h6_lo = (float)(h6d - (double)h6_hi);
          const bool zn_vec = (M % 2) == 0;
          float2* zo_buf = zs0 + (size_t)(cur ^ 1) * zsb;
          const int mq = Mq / 4, nrt = (NR + TR - 1) / TR;
          const float2* zg = zc;
          for (int tile = tid; tile < nrt * mq; tile += NT) {
            const int rt = tile / mq, m0 = (tile - rt * mq) * 4, l0 = r_lo + rt * TR;
            float cmx[4] = {0.f, 0.f, 0.f, 0.f};   // column maxima of the rows written (tensor-core Gram)
            float2 f[TR][4];
            int ext[TR + 1];   // CSR extents of the tile's rows of A, loaded together
#pragma unroll
            for (int r = 0; r <= TR; ++r) ext[r] = a.rowptr[min(l0 + r, r_hi)];
#pragma unroll
            for (int r = 0; r < TR; ++r) {
#pragma unroll
              for (int u = 0; u < 4; ++u) f[r][u] = make_float2(0.f, 0.f);
              if (l0 + r < r_hi) {
                // the static diagonal of A as hi + lo floats (FP32 does not round the
                // detunings), then the other entries of the row
                const float4 dg = a.diag_a[l0 + r];
                float2 z[4];
                load4w(zg + (size_t)(l0 + r) * Mp + m0, z);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  f[r][u].x = fmaf(dg.x, z[u].x, fmaf(-dg.y, z[u].y, fmaf(dg.z, z[u].x, -dg.w * z[u].y)));
                  f[r][u].y = fmaf(dg.x, z[u].y, fmaf(dg.y, z[u].x, fmaf(dg.z, z[u].y, dg.w * z[u].x)));
                }
                row_gather4(a, a.valf_a, ext[r], ext[r + 1], m0, zg, chi, f[r]);
              }
            }
            // + sum_k Y_k XT_k: l in pairs, 16-byte loads of the Y entries
            for (int k = 0; k < K; ++k) {
              const float2* yk = ybuf + (size_t)k * zsb;
              const float2* xk = XT + k * MM;
              for (int l = 0; l < Mq; l += 2) {
                float4 y2[TR];
#pragma unroll
                for (int r = 0; r < TR; ++r)
                  y2[r] = l0 + r < r_hi ? *reinterpret_cast<const float4*>(yk + yq(l0 + r, l))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int ll = 0; ll < 2; ++ll) {
                  const float4 xa = reinterpret_cast<const float4*>(xk + (l + ll) * Mp + m0)[0];
                  const float4 xb = reinterpret_cast<const float4*>(xk + (l + ll) * Mp + m0)[1];
                  const float2 x[4] = {make_float2(xa.x, xa.y), make_float2(xa.z, xa.w), make_float2(xb.x, xb.y),
                                       make_float2(xb.z, xb.w)};
#pragma unroll
                  for (int r = 0; r < TR; ++r) {
                    const float yx = ll ? y2[r].z : y2[r].x, yy = ll ? y2[r].w : y2[r].y;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                      f[r][u].x = fmaf(yx, x[u].x, fmaf(-yy, x[u].y, f[r][u].x));
                      f[r][u].y = fmaf(yx, x[u].y, fmaf(yy, x[u].x, f[r][u].y));
                    }
                  }
                }
              }
            }
            // RK4 (weights 1/6, 1/3, 1/3, 1/6), step sizes as hi + lo floats
#pragma unroll
            for (int r = 0; r < TR; ++r) {
              const int n = l0 + r;
              if (n >= r_hi) continue;
              float2 zo[4];
#pragma unroll
              for (int pr = 0; pr < 2; ++pr) {
                const int u0 = 2 * pr, m = m0 + u0;
                if (m >= M) {
                  zo[u0] = zo[u0 + 1] = make_float2(0.f, 0.f);
                  continue;
                }
                const bool two = m + 1 < M;
                const size_t oz = (size_t)n * M + m, oa = (size_t)n * Mp + m;
                float2 zn0, zn1 = make_float2(0.f, 0.f);
                if (zn_vec) {
                  const float4 v = *reinterpret_cast<const float4*>(Zn + oz);
                  zn0 = make_float2(v.x, v.y);
                  zn1 = make_float2(v.z, v.w);
                } else {
                  zn0 = Zn[oz];
                  if (two) zn1 = Zn[oz + 1];
                }
                float4* ap = reinterpret_cast<float4*>(accg + oa);
                const float f0r = f[r][u0].x, f0i = f[r][u0].y, f1r = f[r][u0 + 1].x, f1i = f[r][u0 + 1].y;
                if (stage < 3) {
                  if (stage == 0) {
                    *ap = make_float4(f0r, f0i, f1r, f1i);
                  } else {
                    const float4 ac = *ap;
                    *ap = make_float4(fmaf(2.f, f0r, ac.x), fmaf(2.f, f0i, ac.y), fmaf(2.f, f1r, ac.z),
                                      fmaf(2.f, f1i, ac.w));
                  }
                  zo[u0] = make_float2(zn0.x + fmaf(hs_lo, f0r, hs_hi * f0r), zn0.y + fmaf(hs_lo, f0i, hs_hi * f0i));
                  zo[u0 + 1] = two ? make_float2(zn1.x + fmaf(hs_lo, f1r, hs_hi * f1r),
                                                 zn1.y + fmaf(hs_lo, f1i, hs_hi * f1i))
                                   : make_float2(0.f, 0.f);
                } else {
                  const float4 ac = *ap;
                  const float s0r = ac.x + f0r, s0i = ac.y + f0i, s1r = ac.z + f1r, s1i = ac.w + f1i;
                  zo[u0] = make_float2(zn0.x + fmaf(h6_lo, s0r, h6_hi * s0r), zn0.y + fmaf(h6_lo, s0i, h6_hi * s0i));
                  zo[u0 + 1] = two ? make_float2(zn1.x + fmaf(h6_lo, s1r, h6_hi * s1r),
                                                 zn1.y + fmaf(h6_lo, s1i, h6_hi * s1i))
                                   : make_float2(0.f, 0.f);
                  if (zn_vec) {
                    *reinterpret_cast<float4*>(Zn + oz) = make_float4(zo[u0].x, zo[u0].y, zo[u0 + 1].x, zo[u0 + 1].y);
                  } else {
                    Zn[oz] = zo[u0];
                    if (two) Zn[oz + 1] = zo[u0 + 1];
                  }
                }
              }
              store4w(zo_buf + (size_t)n * Mp + m0, zo);
              if constexpr (GTC)
#pragma unroll
                for (int u = 0; u < 4; ++u) cmx[u] = fmaxf(cmx[u], fmaxf(fabsf(zo[u].x), fabsf(zo[u].y)));
            }
            if constexpr (GTC)
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (m0 + u < 20) atomicMax(&gcmax[gpar ^ 1][m0 + u], __float_as_uint(cmx[u]));
          }
          cur ^= 1;
          gpar ^= 1;
          team_sync();   // B2: the next stage input is visible to the team
        }
      }
      if (last) break;
    }
    if (head && tid == 0) {   // every thread's Z_n rows are written (barrier above)
      __threadfence();
      atomicExch(a.flag + tj, 1);
    }
  };

  auto release_tmem = [&]() {
    if constexpr (GTC) {
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
  };
  if (!a.split) {
    for (int tj = team; tj < a.T; tj += n_teams) piece(tj, 0, a.n_steps, false, false);
    if (C > 1) cluster.sync();   // no CTA leaves while the team may read its shared memory
    release_tmem();
    return;
  }
  // Equal spans of the T x n_steps trajectory-steps, in trajectory-major
  // order, one per CTA (T >= gridDim.x, so a span covers at least one whole
  // trajectory's steps and cuts at most two trajectories): the head of the
  // trajectory cut at the span's end runs first, then the whole trajectories,
  // then the tail of the trajectory cut at its start, whose head the previous
  // CTA ran first. (The launch is cooperative: every CTA is resident.)
  const long long nts = (long long)a.T * a.n_steps;
  const long long lo = nts * blockIdx.x / gridDim.x, hi = nts * (blockIdx.x + 1) / gridDim.x;
  const int ta = (int)(lo / a.n_steps), tb = (int)((hi - 1) / a.n_steps);
  const long sa = (long)(lo - (long long)ta * a.n_steps), sb = (long)(hi - (long long)tb * a.n_steps);
  if (sb < a.n_steps) piece(tb, 0, sb, true, false);
  for (int tj = sa > 0 ? ta + 1 : ta; tj <= (sb < a.n_steps ? tb - 1 : tb); ++tj) piece(tj, 0, a.n_steps, false, false);
  if (sa > 0) piece(ta, sa, a.n_steps, false, true);
  release_tmem();
}

}  // namespace sfz
}  // namespace lr
