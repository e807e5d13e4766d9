// Sparse-operator engine (FP64) for operator sets given as CSR rows with time
// channels: the paper's own model of Sec. S2 (built by lr_paper_model.cu) or
// any other H_eff(t), L_k(t), r with that structure.
//
// One RK4 stage of Eq. S5 is four launches:
//   sp_apply  - one thread per element (n, m) of the stage input Zs:
//               W = A(t) Zs with A = -i H_eff, Y_k = L_k(t) Zs, and at stage 1
//               of every step Yr = r Zs; the ten channel factors
//               Omega(t)^a e^{i q w_d t} of the step's four stage times come
//               from sp_chi, one small launch per step;
//   sp_gram   - per block, over row tiles of 16 (FP64) or 32 (FP32) rows held in
//               shared memory, register sums of G = Zs^dag Zs (upper
//               triangle), T_k = Zs^dag Y_k, and at stage 1 tr(Zs^dag Yr) =
//               tr(rho r), plus level populations, |Yr|^2 and |Zs|^2 at
//               recording steps;
//   sp_solve  - one block per trajectory: reduce the partials in block order,
//               record beta and the observables, Cholesky G = L L^dag and
//               X_k = G^-1 T_k (the Moore-Penrose projection Zs^+ L_k Zs) by
//               right-looking substitutions over all K M columns at once;
//   sp_update - whole rows per block (Y_k rows staged in shared memory):
//               F = W + 1/2 sum_k Y_k X_k^dag, then the classical RK4 stage.
// After the last step an observation pass (apply r, Gram, solve without
// Cholesky) records beta and the observables of the final state.
//
// FP32_G64 contexts run, by default, the fused persistent kernel of
// lr_sparse_fused.cuh instead: one launch per integrate call, one CTA per
// trajectory (or, for batches larger than the grid, an equal span of the
// batch's trajectory-steps per CTA), all phases of a stage inside the CTA
// (the four-launch path stays selectable with LR_SPARSE_FUSED=0 and is the
// FP64 path).
//
// Precisions: FP64 throughout, or FP32_G64 - the state, the operator apply,
// T_k, the projection term and the RK4 update in FP32, the Gram matrix
// summed in double-word FP32 (~2^-48) from the exact products of FP32
// entries (TwoProduct by one FMA), the M x M solves (FP64 here, double-word
// in the fused kernel) and the signal in FP64.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lr_internal.cuh"
#include "lr_sparse_fused.cuh"

namespace lr {
namespace {

constexpr int SP_T = 256;   // threads per block
// rows per Gram block: 16 complex128 or 32 complex64 rows of Z and of the K + 1
// operator images fit the 48 KB of static shared memory
template <typename T2> __host__ __device__ constexpr int rows_per_block();
template <> __host__ __device__ constexpr int rows_per_block<double2>() { return 16; }
template <> __host__ __device__ constexpr int rows_per_block<float2>() { return 32; }
constexpr int NCH = 10;     // time channels

struct SpDev {
  const int* rowptr;
  const int* col;
  const double2* val;
  const float2* valf;   // FP32 copy of val
  const unsigned char* chan;
  const int* level;
  const PulseDev* pulse;
  unsigned* err;
  void *Z, *Zs, *acc, *W, *Y, *Yr;   // state-type arrays (double2 or float2)
  double2* X;
  float2* Xf;     // FP32 copy of X for the FP32 update
  double2* chi;   // [T][4][NCH] channel factors at the four stage times of the current step
  double* part;
  double2* beta;
  double *pops, *nphot, *trace;
};

template <typename T2> struct Scalar;
template <> struct Scalar<double2> { using type = double; };
template <> struct Scalar<float2> { using type = float; };

__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(v.x, v.y); }
template <typename T2> __device__ __forceinline__ T2 from_d(double2 v);
template <> __device__ __forceinline__ double2 from_d<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <typename T2> __device__ __forceinline__ T2 mk2(typename Scalar<T2>::type r, typename Scalar<T2>::type i) {
  T2 v;
  v.x = r;
  v.y = i;
  return v;
}
__device__ __forceinline__ const double2& op_val(const SpDev& d, int e, double2) { return d.val[e]; }
__device__ __forceinline__ const float2& op_val(const SpDev& d, int e, float2) { return d.valf[e]; }

struct SpParams {
  int N, M, K, T, n_levels, nblk;   // nblk: Gram blocks (partial sums) per trajectory
  int ntile;                        // row tiles per trajectory (rows_per_block rows each)
  long long NM;      // N * M
  long long ps;      // doubles per partial block
  double wd, tau;
  long max_steps, n_rec;
  int pop_every;
};

enum : int { MODE_SOLVE = 1, MODE_OBS = 2, MODE_BETA = 4 };

template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  return mk2<T2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T2> __device__ __forceinline__ T2 cfma(T2 a, T2 b, T2 c) {
  return mk2<T2>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// conj(a) * b + c
template <typename T2> __device__ __forceinline__ T2 cfma_conj(T2 a, T2 b, T2 c) {
  return mk2<T2>(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}

// Double-word FP32 accumulator (hi + lo): s += a b with the product split
// exactly by one FMA (TwoProduct) and the sum by Knuth's TwoSum.
struct DWs {
  float hi, lo;
};
__device__ __forceinline__ void dw_acc(DWs& s, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}

// Channel factors Omega(t)^a e^{i q w_d t} of one trajectory at the four RK4
// stage times t, t + dt/2, t + dt/2, t + dt (one thread per factor).
__global__ void __launch_bounds__(64) sp_chi(SpDev d, SpParams p, double t, double dt) {
  const int tj = blockIdx.x, c = threadIdx.x;
  if (c >= 4 * NCH) return;
  const int stage = c / NCH, ch = c - stage * NCH;
  const double ts = t + (stage == 0 ? 0.0 : stage == 3 ? dt : 0.5 * dt);
  const int a = ch / 5, q = ch % 5 - 2;
  const double om = a ? pulse_envelope(d.pulse[tj], p.tau, ts) : 1.0;
  double sn, cs;
  sincos((double)q * p.wd * ts, &sn, &cs);
  d.chi[(size_t)tj * 4 * NCH + c] = mk(om * cs, om * sn);
}

// out[e] = sum over the row's entries of chi[ch] val Zs[col][m]
template <typename T2>
__device__ __forceinline__ T2 row_apply(const SpDev& d, const SpParams& p, int op, int n, int m,
                                        const T2* __restrict__ Zs, const T2* chi) {
  const int* rp = d.rowptr + (size_t)op * (p.N + 1);
  T2 acc = mk2<T2>(0, 0);
  for (int e = rp[n]; e < rp[n + 1]; ++e) {
    const T2 v = cmul(chi[d.chan[e]], op_val(d, e, T2()));
    acc = cfma(v, Zs[(size_t)d.col[e] * p.M + m], acc);
  }
  return acc;
}

template <typename T2>
__global__ void __launch_bounds__(SP_T) sp_apply(SpDev d, SpParams p, int stage, int with_r, int only_r) {
  __shared__ T2 chi[NCH];
  const int tj = blockIdx.y;
  if (threadIdx.x < NCH) chi[threadIdx.x] = from_d<T2>(d.chi[((size_t)tj * 4 + stage) * NCH + threadIdx.x]);
  __syncthreads();
  const long long e = (long long)blockIdx.x * SP_T + threadIdx.x;
  if (e >= p.NM) return;
  const int n = (int)(e / p.M), m = (int)(e - (long long)n * p.M);
  const size_t off = (size_t)tj * p.NM;
  const T2* Zs = static_cast<const T2*>(d.Zs) + off;
  if (!only_r) {
    static_cast<T2*>(d.W)[off + e] = row_apply(d, p, 0, n, m, Zs, chi);
    for (int k = 0; k < p.K; ++k)
      static_cast<T2*>(d.Y)[((size_t)k * p.T + tj) * p.NM + e] = row_apply(d, p, 1 + k, n, m, Zs, chi);
  }
  if (with_r) static_cast<T2*>(d.Yr)[off + e] = row_apply(d, p, 1 + p.K, n, m, Zs, chi);
}

// Register accumulator of one G or T_k entry: double-word FP32 (re.hi, re.lo,
// im.hi, im.lo) for G in the FP32 variant, plain sums otherwise.
template <typename T2> struct Acc;
template <> struct Acc<double2> {
  double2 v;
  __device__ void zero() { v = mk(0.0, 0.0); }
  __device__ void add_g(double2 a, double2 c) { v = cfma_conj(a, c, v); }
  __device__ void add_t(double2 a, double2 c) { v = cfma_conj(a, c, v); }
  __device__ double2 g() const { return v; }
  __device__ double2 t() const { return v; }
};
template <> struct Acc<float2> {
  DWs re, im;
  __device__ void zero() { re = im = DWs{0.f, 0.f}; }
  __device__ void add_g(float2 a, float2 c) {   // conj(a) c, exact products
    dw_acc(re, a.x, c.x);
    dw_acc(re, a.y, c.y);
    dw_acc(im, a.x, c.y);
    dw_acc(im, -a.y, c.x);
  }
  __device__ void add_t(float2 a, float2 c) {   // conj(a) c in FP32 (re.hi, im.hi)
    re.hi = fmaf(a.x, c.x, fmaf(a.y, c.y, re.hi));
    im.hi = fmaf(a.x, c.y, fmaf(-a.y, c.x, im.hi));
  }
  __device__ double2 g() const { return mk((double)re.hi + (double)re.lo, (double)im.hi + (double)im.lo); }
  __device__ double2 t() const { return mk((double)re.hi, (double)im.hi); }
};

// Entries per thread of the (1 + K) M^2 partial sums: up to (1 + 3) 32^2 / 256.
constexpr int ACC_MAX = (1 + LR_SPARSE_MAX_JUMPS) * LR_MAX_RANK * LR_MAX_RANK / SP_T;

// NACC: accumulators per thread, >= (1 + K) M^2 / SP_T (4, 8 or ACC_MAX)
template <typename T2, int NACC>
__global__ void __launch_bounds__(SP_T) sp_gram(SpDev d, SpParams p, int mode) {
  using T = typename Scalar<T2>::type;
  constexpr int R = rows_per_block<T2>();
  __shared__ T2 sZ[R][LR_MAX_RANK], sY[LR_SPARSE_MAX_JUMPS + 1][R][LR_MAX_RANK];
  __shared__ T rsum[R][4];
  __shared__ T stot[4 + LR_MAX_NT];   // signal, photons, trace, populations (written by thread 0)
  __shared__ int slev[R];
  const int tj = blockIdx.y, b = blockIdx.x, M = p.M, K = p.K, MM = M * M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t off = (size_t)tj * p.NM;
  const bool solve = mode & MODE_SOLVE, obs = mode & MODE_OBS, beta = mode & MODE_BETA;
  const T2* Zs = static_cast<const T2*>(d.Zs);
  const T2* Yk = static_cast<const T2*>(d.Y);
  const T2* Yr = static_cast<const T2*>(d.Yr);
  const int n_ent = (1 + K) * MM;
  Acc<T2> acc[NACC];
#pragma unroll
  for (int q = 0; q < NACC; ++q) acc[q].zero();
  if (tid < 4 + LR_MAX_NT) stot[tid] = 0;
  // row tiles b, b + nblk, b + 2 nblk, ... in increasing order
  for (int tile = b; tile < p.ntile; tile += p.nblk) {
    const int r0 = tile * R, rows = min(R, p.N - r0);
    __syncthreads();   // the previous tile is consumed
    for (int e = tid; e < R * M; e += SP_T) {
      const int i = e / M, m = e - (e / M) * M;
      T2 z = mk2<T2>(0, 0), yr = mk2<T2>(0, 0);
      if (i < rows) {
        const size_t idx = off + (size_t)(r0 + i) * M + m;
        z = Zs[idx];
        if (beta) yr = Yr[idx];
        if (solve)
          for (int k = 0; k < K; ++k) sY[k][i][m] = Yk[(size_t)k * p.T * p.NM + idx];
      } else if (solve) {
        for (int k = 0; k < K; ++k) sY[k][i][m] = mk2<T2>(0, 0);
      }
      sZ[i][m] = z;
      sY[LR_SPARSE_MAX_JUMPS][i][m] = yr;
      if (m == 0) slev[i] = i < rows ? d.level[r0 + i] : -1;
    }
    __syncthreads();
    if (solve) {
#pragma unroll
      for (int q = 0; q < NACC; ++q) {
        const int e = tid + q * SP_T;
        if (e < n_ent) {
          const int mat = e / MM, ij = e - mat * MM, i = ij / M, j = ij - (ij / M) * M;
          if (mat == 0) {
            if (i <= j)
              for (int r = 0; r < rows; ++r) acc[q].add_g(sZ[r][i], sZ[r][j]);
          } else {
            for (int r = 0; r < rows; ++r) acc[q].add_t(sZ[r][i], sY[mat - 1][r][j]);
          }
        }
      }
    }
    if (beta || obs) {
      // one warp per row, lanes over m: conj(z) r z, |r z|^2, |z|^2 in the
      // state's arithmetic; then one lane per row; fixed-order shuffle sums
      for (int r = warp; r < R; r += SP_T / 32) {
        T v[4] = {0, 0, 0, 0};
        if (r < rows && lane < M) {
          const T2 z = sZ[r][lane], y = sY[LR_SPARSE_MAX_JUMPS][r][lane];
          v[0] = fma(z.x, y.x, z.y * y.y);
          v[1] = fma(z.x, y.y, -z.y * y.x);
          v[2] = fma(y.x, y.x, y.y * y.y);
          v[3] = fma(z.x, z.x, z.y * z.y);
        }
        for (int o = 16; o > 0; o >>= 1)
          for (int c = 0; c < 4; ++c) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
        if (lane == 0)
          for (int c = 0; c < 4; ++c) rsum[r][c] = v[c];
      }
      __syncthreads();
      if (warp == 0) {
        T v[4];
        for (int c = 0; c < 4; ++c) v[c] = lane < rows ? rsum[lane][c] : (T)0;
        for (int o = 16; o > 0; o >>= 1)
          for (int c = 0; c < 4; ++c) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
        if (lane == 0)
          for (int c = 0; c < 4; ++c) stot[c] += v[c];
        if (obs)
          for (int l = 0; l < p.n_levels; ++l) {
            T w = (lane < rows && slev[lane] == l) ? rsum[lane][3] : (T)0;
            for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
            if (lane == 0) stot[4 + l] += w;
          }
      }
    }
  }
  double* out = d.part + ((size_t)tj * p.nblk + b) * p.ps;
  if (solve) {
#pragma unroll
    for (int q = 0; q < NACC; ++q) {
      const int e = tid + q * SP_T;
      if (e < n_ent) {
        const double2 v = e < MM ? acc[q].g() : acc[q].t();
        out[2 * e] = v.x;
        out[2 * e + 1] = v.y;
      }
    }
  }
  const size_t o2 = (size_t)2 * n_ent;   // beta re, im, nphot, trace, pops[n_levels]
  if ((beta || obs) && tid == 0) {   // stot was last written by this thread
    for (int c = 0; c < 4; ++c) out[o2 + c] = (double)stot[c];
    if (obs)
      for (int l = 0; l < p.n_levels; ++l) out[o2 + 4 + l] = (double)stot[4 + l];
  }
}

// Dynamic shared memory: L [M][M+1] then B [K M][M+1] (column c of the right-hand
// sides T_k, c = k M + j, stored as row B[c]), complex128.
__global__ void __launch_bounds__(SP_T) sp_solve(SpDev d, SpParams p, long step, int mode) {
  extern __shared__ double2 smem[];
  __shared__ int bad;
  const int tj = blockIdx.x, M = p.M, K = p.K, MM = M * M, tid = threadIdx.x, ld = M + 1;
  double2* L = smem;
  double2* B = smem + (size_t)M * ld;
  const double* P = d.part + (size_t)tj * p.nblk * p.ps;
  const size_t o2 = (size_t)2 * (1 + K) * MM;
  if (tid == 0) bad = 0;
  if (mode & (MODE_BETA | MODE_OBS)) {
    const int nv = 4 + p.n_levels;
    for (int v = tid; v < nv; v += SP_T) {
      double s = 0.0;
      for (int b = 0; b < p.nblk; ++b) s += P[b * p.ps + o2 + v];
      if (v < 2) {
        if (mode & MODE_BETA) {
          double* bt = reinterpret_cast<double*>(d.beta + (size_t)tj * (p.max_steps + 1) + step);
          bt[v] = s;
          if (!isfinite(s)) set_error(d.err, DEV_NONFINITE);
        }
      } else if (mode & MODE_OBS) {
        const long rec = step / p.pop_every;
        if (v == 2) d.nphot[(size_t)tj * p.n_rec + rec] = s;
        else if (v == 3) d.trace[(size_t)tj * p.n_rec + rec] = s;
        else d.pops[((size_t)tj * p.n_rec + rec) * p.n_levels + (v - 4)] = s;
      }
    }
  }
  if (!(mode & MODE_SOLVE)) return;
  for (int e = tid; e < (1 + K) * MM; e += SP_T) {   // block partials in block order
    const int mat = e / MM, ij = e - mat * MM, i = ij / M, j = ij - (ij / M) * M;
    if (mat == 0 && i > j) continue;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < p.nblk; ++b) {
      re += P[b * p.ps + 2 * e];
      im += P[b * p.ps + 2 * e + 1];
    }
    if (mat == 0) L[j * ld + i] = i == j ? mk(re, 0.0) : mk(re, -im);   // lower: G_ji = conj(G_ij)
    else B[((mat - 1) * M + j) * ld + i] = mk(re, im);                   // T_k (i, j)
  }
  __syncthreads();
  // right-looking Cholesky G = L L^dag on the lower triangle
  for (int k = 0; k < M; ++k) {
    if (tid == 0) {
      const double piv = L[k * ld + k].x;
      if (!(piv > 0.0) || !isfinite(piv)) {
        bad = 1;
        L[k * ld + k] = mk(1.0, 0.0);
      } else {
        L[k * ld + k] = mk(sqrt(piv), 0.0);
      }
    }
    __syncthreads();
    const double inv = 1.0 / L[k * ld + k].x;
    for (int i = k + 1 + tid; i < M; i += SP_T) L[i * ld + k] = mk(L[i * ld + k].x * inv, L[i * ld + k].y * inv);
    __syncthreads();
    const int rem = M - k - 1;
    for (int e = tid; e < rem * rem; e += SP_T) {
      const int i = k + 1 + e / rem, j = k + 1 + e % rem;
      if (j > i) continue;
      const double2 a = L[i * ld + k], c = L[j * ld + k];   // L_ij -= L_ik conj(L_jk)
      L[i * ld + j] = mk(L[i * ld + j].x - (a.x * c.x + a.y * c.y), L[i * ld + j].y - (a.y * c.x - a.x * c.y));
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) set_error(d.err, DEV_NOT_PD);
    return;
  }
  const int nc = K * M;
  // forward L y = t, right-looking: y_j = t_j / L_jj, then t_i -= L_ij y_j (i > j), all columns at once
  for (int j = 0; j < M; ++j) {
    const double dinv = 1.0 / L[j * ld + j].x;
    for (int c = tid; c < nc; c += SP_T) B[c * ld + j] = mk(B[c * ld + j].x * dinv, B[c * ld + j].y * dinv);
    __syncthreads();
    const int rem = M - j - 1;
    for (int e = tid; e < nc * rem; e += SP_T) {
      const int c = e / rem, i = j + 1 + e % rem;
      const double2 l = L[i * ld + j], y = B[c * ld + j];
      B[c * ld + i] = mk(B[c * ld + i].x - (l.x * y.x - l.y * y.y), B[c * ld + i].y - (l.x * y.y + l.y * y.x));
    }
    __syncthreads();
  }
  // back L^dag x = y: x_j = y_j / L_jj, then y_i -= conj(L_ji) x_j (i < j)
  for (int j = M - 1; j >= 0; --j) {
    const double dinv = 1.0 / L[j * ld + j].x;
    for (int c = tid; c < nc; c += SP_T) B[c * ld + j] = mk(B[c * ld + j].x * dinv, B[c * ld + j].y * dinv);
    __syncthreads();
    for (int e = tid; e < nc * j; e += SP_T) {
      const int c = e / j, i = e % j;
      const double2 l = L[j * ld + i], x = B[c * ld + j];
      B[c * ld + i] = mk(B[c * ld + i].x - (l.x * x.x + l.y * x.y), B[c * ld + i].y - (l.x * x.y - l.y * x.x));
    }
    __syncthreads();
  }
  double2* X = d.X + (size_t)tj * K * MM;
  float2* Xf = d.Xf + (size_t)tj * K * MM;
  for (int e = tid; e < K * MM; e += SP_T) {   // X[k][i][j] = (X_k)_ij = B[(k M + j)][i]
    const int k = e / MM, ij = e - k * MM, i = ij / M, j = ij - (ij / M) * M;
    const double2 v = B[(k * M + j) * ld + i];
    X[e] = v;
    Xf[e] = make_float2((float)v.x, (float)v.y);
  }
}

__device__ __forceinline__ double2 load_x(const SpDev& d, size_t i, double2) { return d.X[i]; }
__device__ __forceinline__ float2 load_x(const SpDev& d, size_t i, float2) { return d.Xf[i]; }

// Whole rows per block: rb = SP_T / M rows; thread e < rb M owns element
// (n0 + e / M, e % M). The block's rows of Y_k are contiguous in memory and are
// staged in shared memory with coalesced loads.
template <typename T2>
__global__ void __launch_bounds__(SP_T) sp_update(SpDev d, SpParams p, int stage, double dt_) {
  using T = typename Scalar<T2>::type;
  __shared__ T2 sX[LR_MAX_RANK * LR_MAX_RANK];
  __shared__ T2 sY[SP_T];
  const int tj = blockIdx.y, M = p.M, MM = M * M, e = threadIdx.x;
  const int rb = SP_T / M, n0 = blockIdx.x * rb;
  const int n = n0 + e / M, m = e - (e / M) * M;
  const bool live = e < rb * M && n < p.N;
  const size_t off = (size_t)tj * p.NM, idx = (size_t)n * M + m;
  T2* Z = static_cast<T2*>(d.Z);
  T2* Zs = static_cast<T2*>(d.Zs);
  T2* acc = static_cast<T2*>(d.acc);
  const T2* Yk = static_cast<const T2*>(d.Y);
  T2 F = live ? static_cast<const T2*>(d.W)[off + idx] : mk2<T2>(0, 0);
  const T half = (T)0.5;
  const int rbase = (e / M) * M;   // this row's first element in sY
  for (int k = 0; k < p.K; ++k) {
    __syncthreads();
    for (int i = threadIdx.x; i < MM; i += SP_T) sX[i] = load_x(d, ((size_t)tj * p.K + k) * MM + i, T2());
    if (live) sY[e] = Yk[((size_t)k * p.T + tj) * p.NM + idx];
    __syncthreads();
    if (live) {   // F += 1/2 sum_j Y_k[n][j] conj(X_k[m][j])
      T2 s = mk2<T2>(0, 0);
      for (int jj = 0; jj < M; ++jj) {
        const T2 a = sY[rbase + jj], x = sX[m * M + jj];
        s = mk2<T2>(fma(a.x, x.x, fma(a.y, x.y, s.x)), fma(a.y, x.x, fma(-a.x, x.y, s.y)));
      }
      F = mk2<T2>(fma(half, s.x, F.x), fma(half, s.y, F.y));
    }
  }
  if (!live) return;
  const T dt = (T)dt_;
  const T w = (stage == 0 || stage == 3) ? (T)1 : (T)2;
  const T2 a0 = stage == 0 ? mk2<T2>(0, 0) : acc[off + idx];
  const T2 a = mk2<T2>(fma(w, F.x, a0.x), fma(w, F.y, a0.y));
  const T2 z = Z[off + idx];
  if (stage < 3) {
    const T c = stage == 2 ? dt : (T)0.5 * dt;
    acc[off + idx] = a;
    Zs[off + idx] = mk2<T2>(fma(c, F.x, z.x), fma(c, F.y, z.y));
  } else {
    const T c = dt / (T)6;
    const T2 zn = mk2<T2>(fma(c, a.x, z.x), fma(c, a.y, z.y));
    if (!isfinite(zn.x) || !isfinite(zn.y)) set_error(d.err, DEV_NONFINITE);
    Z[off + idx] = zn;
    Zs[off + idx] = zn;
  }
}

// Sec. S3.A / S3.B for candidate c = trajectories (2c, 2c+1) = (g, e), over the
// steps [0, step]: S = trapezoid of |beta_e - beta_g|^2 (step dt),
// SNR = sqrt(2 eta kappa S), eps_a = erfc(SNR/2)/2 + tau gamma/2, tau = step dt;
// T = (1/tau) sum_{g,e} sum_{k>=2} trapezoid of P_k over the records
// [0, step / pop_every]; Lambda = log10(eps_a + T). out[c] = (eps_a, T, Lambda).
__global__ void __launch_bounds__(SP_T) sp_loss(SpDev d, SpParams p, long step, double dt, double eta, double kappa,
                                                double gamma, double* out) {
  __shared__ double red[SP_T / 32];
  const int c = blockIdx.x, tid = threadIdx.x;
  const double2* bg = d.beta + (size_t)(2 * c) * (p.max_steps + 1);
  const double2* be = d.beta + (size_t)(2 * c + 1) * (p.max_steps + 1);
  double acc = 0.0, ion = 0.0;
  for (long i = tid; i <= step; i += SP_T) {
    const double dx = be[i].x - bg[i].x, dy = be[i].y - bg[i].y;
    acc += (i == 0 || i == step ? 0.5 : 1.0) * (dx * dx + dy * dy);
  }
  const long last = step / p.pop_every;
  for (long r = tid; r <= last; r += SP_T) {
    double sum = 0.0;
    for (int tj = 2 * c; tj <= 2 * c + 1; ++tj)
      for (int k = 2; k < p.n_levels; ++k) sum += d.pops[((size_t)tj * p.n_rec + r) * p.n_levels + k];
    ion += (r == 0 || r == last ? 0.5 : 1.0) * sum;
  }
  double v[2] = {acc, ion};
  for (int q = 0; q < 2; ++q) {   // fixed-order block sum
    double x = v[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = x;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < SP_T / 32; ++w) t += red[w];
      v[q] = t;
    }
  }
  if (tid == 0) {
    const double tau = (double)step * dt;
    const double S = step > 0 ? dt * v[0] : 0.0;
    const double snr = sqrt(2.0 * eta * kappa * S);
    const double e = 0.5 * erfc(0.5 * snr) + 0.5 * tau * gamma;
    const double T = (step > 0 && last > 0) ? v[1] * p.pop_every * dt / tau : 0.0;
    out[3 * c] = e;
    out[3 * c + 1] = T;
    out[3 * c + 2] = log10(e + T);
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace lr

using namespace lr;

struct lr_sparse {
  int N, M, K, T, n_levels, nblk, ntile;
  int fp32;   // 1: FP32_G64 state arithmetic
  int fused;  // 1: the fused persistent kernel (FP32_G64), 0: four launches per RK4 stage
  int gram_tc;   // fused: 1 when the Gram matrix is formed on the tensor cores (rank padded to 20)
  int n_cta;   // fused: persistent CTAs (n_team teams of team_c)
  int n_team, team_c;   // fused: teams (one trajectory at a time each), CTAs per team
  size_t o_fsc;   // fused: per-CTA stage buffers
  size_t o_fvala, o_fdiag;   // fused: values of A without its static diagonal, and that diagonal (hi + lo)
  size_t o_fflag;   // fused: [T] hand-over flags of the split schedule
  long nnz, max_steps, n_rec, step;
  double dt;   // RK4 step of the run (0 before the first integrate)
  int pop_every;
  double wd, tau;
  std::vector<int> rowptr, col, level;
  std::vector<double> val;
  std::vector<unsigned char> chan;
  std::vector<PulseDev> pulses;
  char* ws;
  size_t ws_bytes;
  // offsets into the workspace
  size_t o_rowptr, o_col, o_val, o_valf, o_chan, o_level, o_pulse, o_traj, o_err, o_Z, o_Zs, o_acc, o_W, o_Y, o_Yr, o_X, o_chi, o_Xf, o_loss,
      o_part, o_beta, o_pops, o_nphot, o_trace, total;
  std::string msg;
};

namespace {

lr_status fail(lr_sparse* s, lr_status st, const char* m) {
  if (s) s->msg = m;
  return st;
}

lr_status cuda_fail(lr_sparse* s, cudaError_t e) {
  if (s) s->msg = cudaGetErrorString(e);
  return LR_ERR_CUDA;
}

void layout(lr_sparse* s) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o = align256(o + bytes);
    return r;
  };
  const size_t state = (size_t)s->T * s->N * s->M * (s->fp32 ? sizeof(float2) : sizeof(double2));
  const size_t state64 = (size_t)s->T * s->N * s->M * sizeof(double2);
  s->o_rowptr = take((size_t)(s->K + 2) * (s->N + 1) * sizeof(int));
  s->o_col = take((size_t)s->nnz * sizeof(int));
  s->o_val = take((size_t)s->nnz * sizeof(double2));
  s->o_valf = take((size_t)s->nnz * sizeof(float2));
  s->o_chan = take((size_t)s->nnz);
  s->o_level = take((size_t)s->N * sizeof(int));
  s->o_pulse = take((size_t)s->T * sizeof(PulseDev));
  s->o_traj = take((size_t)s->T * sizeof(TrajDev));
  s->o_err = take(sizeof(unsigned));
  s->o_Z = take(state);
  s->o_Zs = take(state);
  s->o_acc = take(state);
  s->o_W = take(state64);   // also the FP64 scratch of set_initial / set_state / get_state
  s->o_Y = take(state * s->K);
  s->o_Yr = take(state);
  s->o_X = take((size_t)s->T * s->K * s->M * s->M * sizeof(double2));
  s->o_chi = take((size_t)s->T * 4 * NCH * sizeof(double2));
  s->o_Xf = take((size_t)s->T * s->K * s->M * s->M * sizeof(float2));
  s->o_loss = take((size_t)(s->T / 2 + 1) * 3 * sizeof(double));
  const size_t ps = (size_t)2 * (1 + s->K) * s->M * s->M + 4 + s->n_levels;
  s->o_part = take((size_t)s->T * s->nblk * ps * sizeof(double));
  s->o_beta = take((size_t)s->T * (s->max_steps + 1) * sizeof(double2));
  s->o_pops = take((size_t)s->T * s->n_rec * s->n_levels * sizeof(double));
  s->o_nphot = take((size_t)s->T * s->n_rec * sizeof(double));
  s->o_trace = take((size_t)s->T * s->n_rec * sizeof(double));
  if (s->fused) {
    const size_t Mp = (size_t)(s->M + 3) / 4 * 4;
    s->o_fsc = take((size_t)s->n_team * (3 + s->K) * s->N * Mp * sizeof(float2));
    s->o_fvala = take((size_t)s->nnz * sizeof(float2));
    s->o_fdiag = take((size_t)s->N * sizeof(float4));
    s->o_fflag = take((size_t)s->T * sizeof(int));
  }
  s->total = o;
}

// Dynamic shared memory of the fused kernel: G and L^-1 (FP64-sized complex
// [Mp][Mp+1]), T_k and XT_k (FP32 complex [K][Mp][Mp]), scalars, and the
// partials of G (FP64 complex [Mp][Mp]) and the team's T_k ([K][Mp][Mp]).
struct SfSmem {
  int o_gd, o_w, o_tred, o_xt, o_misc, o_gpart, o_tsum, o_gs, o_gv, total;
};
// gtc: the slice buffers and V of the Gram matrix on the tensor cores
SfSmem sf_smem(int M, int K, int gtc) {
  const int Mp = (M + 3) / 4 * 4;
  SfSmem L;
  int o = 0;
  L.o_gd = o;
  o += Mp * (Mp + 1) * (int)sizeof(double2);
  L.o_w = o;
  o += Mp * (Mp + 1) * (int)sizeof(double2);
  L.o_tred = o;
  o += K * Mp * Mp * (int)sizeof(float2);
  L.o_xt = o;
  o += K * Mp * Mp * (int)sizeof(float2);
  L.o_misc = o;
  o += 96 * (int)sizeof(double);
  L.o_gpart = o;
  o += Mp * Mp * (int)sizeof(double2);
  L.o_tsum = o;
  o += K * Mp * Mp * (int)sizeof(float2);
  L.o_gs = L.o_gv = o;
  if (gtc) {
    o = (o + 127) / 128 * 128;
    L.o_gs = o;
    o += 2 * GS_BUF;
    L.o_gv = o;
    o += 40 * 40 * 8;
  }
  L.total = o;
  return L;
}

cudaError_t raise_fused_smem(int bytes) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  for (const void* k : {(const void*)sfz::sf_kernel<false, false>, (const void*)sfz::sf_kernel<true, false>,
                        (const void*)sfz::sf_kernel<false, true>, (const void*)sfz::sf_kernel<true, true>}) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    if (fa.maxDynamicSharedSizeBytes >= bytes && fa.nonPortableClusterSizeAllowed) continue;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < bytes)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Team size of the fused kernel for a batch of T trajectories on `sms` SMs:
// one CTA per trajectory when the batch fills the grid, else the largest team
// (<= 16 CTAs, >= 64 rows per CTA) that keeps the teams within the SMs and
// that the GPU can hold as resident clusters. LR_SPARSE_C forces a size.
void fused_teams(lr_sparse* s, int sms) {
  int C = 1;
  if (s->T < sms) C = std::max(1, std::min({16, sms / s->T, s->N / 64}));
  if (const char* e = getenv("LR_SPARSE_C")) C = std::max(1, std::min(16, atoi(e)));
  C = std::min(C, s->N);
  const SfSmem L = sf_smem(s->M, s->K, s->gram_tc);
  for (; C > 1; --C) {   // the largest team that fits as a cluster
    if (raise_fused_smem(L.total) != cudaSuccess) break;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C * std::max(1, std::min(s->T, sms / C)));
    cfg.blockDim = dim3(sfz::NT);
    cfg.dynamicSmemBytes = L.total;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    const void* kt = s->gram_tc ? (const void*)sfz::sf_kernel<true, true> : (const void*)sfz::sf_kernel<true, false>;
    if (cudaOccupancyMaxActiveClusters(&ncl, kt, &cfg) == cudaSuccess && ncl > 0) {
      s->team_c = C;
      s->n_team = std::min(s->T, ncl);
      s->n_cta = C * s->n_team;
      return;
    }
  }
  cudaGetLastError();
  s->team_c = 1;
  s->n_team = std::min(s->T, sms);
  s->n_cta = s->n_team;
}

SpDev dev(const lr_sparse* s) {
  char* w = s->ws;
  SpDev d;
  d.rowptr = reinterpret_cast<const int*>(w + s->o_rowptr);
  d.col = reinterpret_cast<const int*>(w + s->o_col);
  d.val = reinterpret_cast<const double2*>(w + s->o_val);
  d.valf = reinterpret_cast<const float2*>(w + s->o_valf);
  d.chan = reinterpret_cast<const unsigned char*>(w + s->o_chan);
  d.level = reinterpret_cast<const int*>(w + s->o_level);
  d.pulse = reinterpret_cast<const PulseDev*>(w + s->o_pulse);
  d.err = reinterpret_cast<unsigned*>(w + s->o_err);
  d.Z = w + s->o_Z;
  d.Zs = w + s->o_Zs;
  d.acc = w + s->o_acc;
  d.W = w + s->o_W;
  d.Y = w + s->o_Y;
  d.Yr = w + s->o_Yr;
  d.X = reinterpret_cast<double2*>(w + s->o_X);
  d.chi = reinterpret_cast<double2*>(w + s->o_chi);
  d.Xf = reinterpret_cast<float2*>(w + s->o_Xf);
  d.part = reinterpret_cast<double*>(w + s->o_part);
  d.beta = reinterpret_cast<double2*>(w + s->o_beta);
  d.pops = reinterpret_cast<double*>(w + s->o_pops);
  d.nphot = reinterpret_cast<double*>(w + s->o_nphot);
  d.trace = reinterpret_cast<double*>(w + s->o_trace);
  return d;
}

size_t state_bytes(const lr_sparse* s) {
  return (size_t)s->T * s->N * s->M * (s->fp32 ? sizeof(float2) : sizeof(double2));
}

size_t solve_smem(const lr_sparse* s) { return (size_t)(1 + s->K) * s->M * (s->M + 1) * sizeof(double2); }

// The dynamic shared-memory limit of sp_solve is a property of the function in
// the current device's context, not of a lr_sparse context: it only ever grows,
// so that a context bound later with a smaller rank does not lower it under one
// bound earlier. The current limit is read from the device each time (it is
// per device, and a device reset restores the default).
cudaError_t raise_solve_smem(int bytes) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, sp_solve);
  if (e != cudaSuccess) return e;
  if (fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(sp_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename T2>
void launch_gram(const lr_sparse* s, const SpDev& d, const SpParams& p, int mode, cudaStream_t st) {
  const dim3 gg((unsigned)s->nblk, (unsigned)s->T);
  const int per = ((1 + s->K) * s->M * s->M + SP_T - 1) / SP_T;
  if (per <= 4)
    sp_gram<T2, 4><<<gg, SP_T, 0, st>>>(d, p, mode);
  else if (per <= 8)
    sp_gram<T2, 8><<<gg, SP_T, 0, st>>>(d, p, mode);
  else
    sp_gram<T2, ACC_MAX><<<gg, SP_T, 0, st>>>(d, p, mode);
}

template <typename T2>
void launch_step_kernels(const lr_sparse* s, const SpDev& d, const SpParams& p, long step0, long n_steps, double dt,
                         cudaStream_t st) {
  const dim3 ge((unsigned)((p.NM + SP_T - 1) / SP_T), (unsigned)s->T);
  const int rb = SP_T / s->M;
  const dim3 gu((unsigned)((s->N + rb - 1) / rb), (unsigned)s->T);
  for (long i = 0; i <= n_steps; ++i) {
    const long step = step0 + i;
    const double t = (double)step * dt;
    const bool rec = step % s->pop_every == 0;
    sp_chi<<<s->T, 64, 0, st>>>(d, p, t, dt);
    if (i == n_steps) {   // observation of the final state
      const int mode = MODE_BETA | (rec ? MODE_OBS : 0);
      sp_apply<T2><<<ge, SP_T, 0, st>>>(d, p, 0, 1, 1);
      launch_gram<T2>(s, d, p, mode, st);
      sp_solve<<<s->T, SP_T, solve_smem(s), st>>>(d, p, step, mode);
      break;
    }
    for (int stg = 0; stg < 4; ++stg) {
      const int mode = MODE_SOLVE | (stg == 0 ? MODE_BETA | (rec ? MODE_OBS : 0) : 0);
      sp_apply<T2><<<ge, SP_T, 0, st>>>(d, p, stg, stg == 0, 0);
      launch_gram<T2>(s, d, p, mode, st);
      sp_solve<<<s->T, SP_T, solve_smem(s), st>>>(d, p, step, mode);
      sp_update<T2><<<gu, SP_T, 0, st>>>(d, p, stg, dt);
    }
  }
}

SpParams params(const lr_sparse* s) {
  SpParams p;
  p.N = s->N;
  p.M = s->M;
  p.K = s->K;
  p.T = s->T;
  p.n_levels = s->n_levels;
  p.nblk = s->nblk;
  p.ntile = s->ntile;
  p.NM = (long long)s->N * s->M;
  p.ps = (long long)2 * (1 + s->K) * s->M * s->M + 4 + s->n_levels;
  p.wd = s->wd;
  p.tau = s->tau;
  p.max_steps = s->max_steps;
  p.n_rec = s->n_rec;
  p.pop_every = s->pop_every;
  return p;
}

// Trajectory records for the initial-state kernel: with N_r = N_f = 1 its
// pure state is the basis state level0.
std::vector<TrajDev> trajectories(const lr_sparse* s, const int* psi) {
  std::vector<TrajDev> traj(s->T);
  for (int i = 0; i < s->T; ++i) {
    TrajDev t;
    memset(&t, 0, sizeof(t));
    t.N = s->N;
    t.M = s->M;
    t.ld = s->M;
    t.Nt = 1;
    t.Nr = 1;
    t.Nf = 1;
    t.n_modes = 3;
    t.cand = i;
    t.level0 = psi ? psi[i] : 0;
    t.z_off = (long long)i * s->N * s->M;
    traj[i] = t;
  }
  return traj;
}

}  // namespace

extern "C" lr_status lr_sparse_create(const lr_sparse_model* m, int n_traj, int M, lr_precision precision,
                                      const lr_pulse* pulses, double tau, long max_steps, int pop_every,
                                      lr_sparse** out) {
  if (!out) return LR_ERR_ARG;
  *out = nullptr;
  if (!m || !pulses || !m->rowptr || !m->col || !m->val || !m->chan || !m->level) return LR_ERR_ARG;
  if (m->N < 1 || m->N > (1 << 24) || m->n_jumps < 1 || m->n_jumps > LR_SPARSE_MAX_JUMPS) return LR_ERR_ARG;
  if (m->n_levels < 1 || m->n_levels > LR_MAX_NT || m->nnz < 0 || m->nnz > (1L << 31) - 1) return LR_ERR_ARG;
  if (n_traj < 1 || n_traj > 65535 || M < 1 || M > LR_MAX_RANK || M > m->N) return LR_ERR_ARG;
  if (!(tau > 0.0) || max_steps < 1 || pop_every < 1 || !isfinite(m->wd)) return LR_ERR_ARG;
  if (precision != LR_PREC_FP64 && precision != LR_PREC_FP32_G64) return LR_ERR_UNSUPPORTED;
  const int K = m->n_jumps, N = m->N;
  for (int o = 0; o < K + 2; ++o) {
    const int* rp = m->rowptr + (size_t)o * (N + 1);
    for (int n = 0; n < N; ++n)
      if (rp[n] < 0 || rp[n] > rp[n + 1] || rp[n + 1] > m->nnz) return LR_ERR_ARG;
  }
  for (long e = 0; e < m->nnz; ++e)
    if (m->col[e] < 0 || m->col[e] >= N || m->chan[e] >= NCH || !isfinite(m->val[2 * e]) || !isfinite(m->val[2 * e + 1]))
      return LR_ERR_ARG;
  for (int n = 0; n < N; ++n)
    if (m->level[n] < 0 || m->level[n] >= m->n_levels) return LR_ERR_ARG;
  for (int i = 0; i < n_traj; ++i) {
    const lr_pulse& P = pulses[i];
    if (P.kind != 0 && P.kind != 1) return LR_ERR_ARG;
    const double wdp = P.kind == 0 ? P.p[1] : P.p[6], phi = P.kind == 0 ? P.p[3] : P.p[7];
    if (phi != 0.0 || fabs(wdp - m->wd) > 1e-12 * fabs(m->wd)) return LR_ERR_ARG;
    for (int k = 0; k < 8; ++k)
      if (!isfinite(P.p[k])) return LR_ERR_ARG;
  }
  lr_sparse* s = new (std::nothrow) lr_sparse();
  if (!s) return LR_ERR_NOMEM;
  s->N = N;
  s->M = M;
  s->fp32 = precision == LR_PREC_FP32_G64;
  s->K = K;
  s->T = n_traj;
  s->n_levels = m->n_levels;
  const int R = s->fp32 ? rows_per_block<float2>() : rows_per_block<double2>();
  s->ntile = (N + R - 1) / R;
  // Gram blocks per trajectory: enough blocks for ~8 per SM over the batch, each
  // looping over ntile / nblk row tiles (fewer partial sums for the solve)
  const int want = (8 * 152 + n_traj - 1) / n_traj;
  s->nblk = std::min(s->ntile, std::max(8, want));
  s->nnz = m->nnz;
  s->max_steps = max_steps;
  s->pop_every = pop_every;
  s->n_rec = max_steps / pop_every + 1;
  s->step = 0;
  s->wd = m->wd;
  s->tau = tau;
  s->rowptr.assign(m->rowptr, m->rowptr + (size_t)(K + 2) * (N + 1));
  s->col.assign(m->col, m->col + m->nnz);
  s->val.assign(m->val, m->val + 2 * m->nnz);
  s->chan.assign(m->chan, m->chan + m->nnz);
  s->level.assign(m->level, m->level + N);
  s->pulses.resize(n_traj);
  for (int i = 0; i < n_traj; ++i) {
    s->pulses[i].kind = pulses[i].kind;
    for (int k = 0; k < 8; ++k) s->pulses[i].p[k] = pulses[i].p[k];
  }
  s->ws = nullptr;
  s->ws_bytes = 0;
  // the fused kernel: FP32_G64, unless LR_SPARSE_FUSED=0 selects the four-launch path;
  // one persistent CTA per SM (fewer when the batch is smaller)
  s->fused = 0;
  s->n_cta = s->n_team = s->team_c = 0;
  s->gram_tc = 0;
  const char* fz_env = getenv("LR_SPARSE_FUSED");
  if (s->fp32 && !(fz_env && strcmp(fz_env, "0") == 0)) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ==
                                                   cudaSuccess && sms > 0) {
      s->fused = 1;
      // LR_SPARSE_GRAM=tc: the Gram matrix on the tensor cores (rank padded to 20,
      // its slice layout); the default keeps the double-word CUDA-core sums, which
      // measured 1.8% faster on the 512-trajectory batch (this kernel waits on its
      // operator gathers, not on the Gram's FMAs)
      const char* gram_env = getenv("LR_SPARSE_GRAM");
      s->gram_tc = (s->M + 3) / 4 * 4 == 20 && gram_env && strcmp(gram_env, "tc") == 0;
      fused_teams(s, sms);
    } else {
      cudaGetLastError();
    }
  }
  layout(s);
  *out = s;
  return LR_OK;
}

extern "C" lr_status lr_sparse_workspace_size(const lr_sparse* s, size_t* bytes) {
  if (!s || !bytes) return LR_ERR_ARG;
  *bytes = s->total;
  return LR_OK;
}

extern "C" lr_status lr_sparse_bind_workspace(lr_sparse* s, void* workspace, size_t bytes, void* stream) {
  if (!s || !workspace) return LR_ERR_ARG;
  if (bytes < s->total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(s, LR_ERR_WORKSPACE, "workspace too small or not 256-byte aligned");
  s->ws = static_cast<char*>(workspace);
  s->ws_bytes = bytes;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const std::vector<TrajDev> traj = trajectories(s, nullptr);
  std::vector<double2> val(s->nnz);
  std::vector<float2> valf(s->nnz);
  for (long e = 0; e < s->nnz; ++e) {
    val[e] = make_double2(s->val[2 * e], s->val[2 * e + 1]);
    valf[e] = make_float2((float)s->val[2 * e], (float)s->val[2 * e + 1]);
  }
  cudaError_t e;
  if ((e = cudaMemsetAsync(s->ws, 0, s->total, st)) != cudaSuccess) return cuda_fail(s, e);
  struct Up {
    size_t off;
    const void* src;
    size_t bytes;
  } ups[] = {{s->o_rowptr, s->rowptr.data(), s->rowptr.size() * sizeof(int)},
             {s->o_col, s->col.data(), s->col.size() * sizeof(int)},
             {s->o_val, val.data(), val.size() * sizeof(double2)},
             {s->o_valf, valf.data(), valf.size() * sizeof(float2)},
             {s->o_chan, s->chan.data(), s->chan.size()},
             {s->o_level, s->level.data(), s->level.size() * sizeof(int)},
             {s->o_pulse, s->pulses.data(), s->pulses.size() * sizeof(PulseDev)},
             {s->o_traj, traj.data(), traj.size() * sizeof(TrajDev)}};
  for (const Up& u : ups)
    if (u.bytes && (e = cudaMemcpyAsync(s->ws + u.off, u.src, u.bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(s, e);
  std::vector<float2> vala;
  std::vector<float4> diag;
  if (s->fused) {
    // A's static (channel a = 0, q = 0) diagonal entries leave the gathered values
    // and go, summed per row in FP64, into hi + lo floats
    vala = valf;
    diag.assign(s->N, make_float4(0.f, 0.f, 0.f, 0.f));
    const int static_ch = 2;
    for (int n = 0; n < s->N; ++n) {
      double dr = 0.0, di = 0.0;
      for (int k = s->rowptr[n]; k < s->rowptr[n + 1]; ++k)
        if (s->col[k] == n && s->chan[k] == static_ch) {
          dr += s->val[2 * k];
          di += s->val[2 * k + 1];
          vala[k] = make_float2(0.f, 0.f);
        }
      const float hr = (float)dr, hi = (float)di;
      diag[n] = make_float4(hr, hi, (float)(dr - (double)hr), (float)(di - (double)hi));
    }
    if ((e = cudaMemcpyAsync(s->ws + s->o_fvala, vala.data(), vala.size() * sizeof(float2), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->ws + s->o_fdiag, diag.data(), diag.size() * sizeof(float4), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
      return cuda_fail(s, e);
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(s, e);
  if ((e = raise_solve_smem((int)solve_smem(s))) != cudaSuccess) return cuda_fail(s, e);
  s->step = 0;
  return LR_OK;
}

extern "C" lr_status lr_sparse_set_initial(lr_sparse* s, const int* psi, uint64_t seed, double eps, void* stream) {
  if (!s || !psi) return LR_ERR_ARG;
  if (!s->ws) return fail(s, LR_ERR_WORKSPACE, "no workspace bound");
  if (!(eps >= 0.0) || !((s->M - 1) * eps < 1.0)) return fail(s, LR_ERR_ARG, "eps out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < s->T; ++i)
    if (psi[i] < 0 || psi[i] >= s->N) return fail(s, LR_ERR_ARG, "psi index out of range");
  const std::vector<TrajDev> traj = trajectories(s, psi);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(s->ws + s->o_traj, traj.data(), traj.size() * sizeof(TrajDev), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return cuda_fail(s, e);
  SpDev d = dev(s);
  DevPtrs p;
  memset(&p, 0, sizeof(p));
  p.traj = reinterpret_cast<const TrajDev*>(s->ws + s->o_traj);
  p.Za = d.W;   // FP64 scratch of the state's layout
  p.Zn = d.Z;
  RunParams rp;
  memset(&rp, 0, sizeof(rp));
  rp.n_traj = s->T;
  if ((e = launch_initial_state(p, rp, s->N, s->fp32, seed, eps, st)) != cudaSuccess) return cuda_fail(s, e);
  if ((e = cudaMemcpyAsync(d.Zs, d.Z, state_bytes(s), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return cuda_fail(s, e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(s, e);
  s->step = 0;
  s->dt = 0.0;
  return LR_OK;
}

extern "C" lr_status lr_sparse_set_state(lr_sparse* s, const double* Z, long step, void* stream) {
  if (!s || !Z) return LR_ERR_ARG;
  if (!s->ws) return fail(s, LR_ERR_WORKSPACE, "no workspace bound");
  if (step < 0 || step > s->max_steps) return fail(s, LR_ERR_ARG, "step out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long n = (long long)s->T * s->N * s->M;
  cudaError_t e;
  if (s->fp32) {   // host complex128 -> FP64 scratch -> complex64 state
    if ((e = cudaMemcpyAsync(s->ws + s->o_W, Z, n * sizeof(double2), cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_fail(s, e);
    if ((e = launch_convert(s->ws + s->o_W, s->ws + s->o_Z, n, 1, st)) != cudaSuccess) return cuda_fail(s, e);
  } else if ((e = cudaMemcpyAsync(s->ws + s->o_Z, Z, n * sizeof(double2), cudaMemcpyHostToDevice, st)) !=
             cudaSuccess) {
    return cuda_fail(s, e);
  }
  if ((e = cudaMemcpyAsync(s->ws + s->o_Zs, s->ws + s->o_Z, state_bytes(s), cudaMemcpyDeviceToDevice, st)) !=
      cudaSuccess)
    return cuda_fail(s, e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(s, e);
  s->step = step;
  return LR_OK;
}

extern "C" lr_status lr_sparse_get_state(const lr_sparse* s, double* Z, void* stream) {
  if (!s || !Z || !s->ws) return LR_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long n = (long long)s->T * s->N * s->M;
  const char* src = s->ws + s->o_Z;
  if (s->fp32) {   // complex64 state -> FP64 scratch (W is only used within a stage)
    if (launch_convert(s->ws + s->o_Z, s->ws + s->o_W, n, 0, st) != cudaSuccess) return LR_ERR_CUDA;
    src = s->ws + s->o_W;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return LR_ERR_CUDA;
  if (cudaMemcpy(Z, src, n * sizeof(double2), cudaMemcpyDeviceToHost) != cudaSuccess) return LR_ERR_CUDA;
  return LR_OK;
}

extern "C" lr_status lr_sparse_integrate(lr_sparse* s, double dt, long n_steps, void* stream) {
  if (!s) return LR_ERR_ARG;
  if (!s->ws) return fail(s, LR_ERR_WORKSPACE, "no workspace bound");
  if (!(dt > 0.0) || !isfinite(dt) || n_steps < 0) return fail(s, LR_ERR_ARG, "bad dt or n_steps");
  if (s->step + n_steps > s->max_steps) return fail(s, LR_ERR_STATE, "integration past max_steps");
  if (s->step > 0 && s->dt > 0.0 && dt != s->dt) return fail(s, LR_ERR_ARG, "dt differs within one pulse run");
  s->dt = dt;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const SpDev d = dev(s);
  const SpParams p = params(s);
  if (s->fused) {
    const SfSmem L = sf_smem(s->M, s->K, s->gram_tc);
    cudaError_t e0 = raise_fused_smem(L.total);
    if (e0 != cudaSuccess) return cuda_fail(s, e0);
    sfz::Args a{};
    a.rowptr = d.rowptr;
    a.col = d.col;
    a.valf = d.valf;
    a.valf_a = reinterpret_cast<const float2*>(s->ws + s->o_fvala);
    a.diag_a = reinterpret_cast<const float4*>(s->ws + s->o_fdiag);
    a.chan = d.chan;
    a.level = d.level;
    a.pulse = d.pulse;
    a.err = d.err;
    a.Z = static_cast<float2*>(d.Z);
    a.flag = reinterpret_cast<int*>(s->ws + s->o_fflag);
    // equal spans of trajectory-steps per CTA when the batch has more
    // trajectories than CTAs (LR_SPARSE_SPLIT=0: whole trajectories per CTA)
    const char* sp_env = getenv("LR_SPARSE_SPLIT");
    a.split = s->team_c == 1 && s->T > s->n_cta && n_steps > 0 && !(sp_env && strcmp(sp_env, "0") == 0);
    a.C = a.split ? 1 : s->team_c;
    a.scratch = reinterpret_cast<float2*>(s->ws + s->o_fsc);
    a.beta = d.beta;
    a.pops = d.pops;
    a.nphot = d.nphot;
    a.trace = d.trace;
    a.N = s->N;
    a.M = s->M;
    a.Mp = (s->M + 3) / 4 * 4;
    a.K = s->K;
    a.T = s->T;
    a.n_levels = s->n_levels;
    a.wd = s->wd;
    a.tau = s->tau;
    a.dt = dt;
    a.max_steps = s->max_steps;
    a.n_rec = s->n_rec;
    a.pop_every = s->pop_every;
    a.step0 = s->step;
    a.n_steps = n_steps;
    a.o_gd = L.o_gd;
    a.o_w = L.o_w;
    a.o_tred = L.o_tred;
    a.o_xt = L.o_xt;
    a.o_misc = L.o_misc;
    a.o_gpart = L.o_gpart;
    a.o_tsum = L.o_tsum;
    a.o_gs = L.o_gs;
    a.o_gv = L.o_gv;
    if (a.split) {
      // the hand-over waits need every CTA resident: a cooperative launch
      // (refused, rather than run, when the grid does not fit)
      int per_sm = 0, dev = 0, sms = 0;
      const void* k1 = s->gram_tc ? (const void*)sfz::sf_kernel<false, true> : (const void*)sfz::sf_kernel<false, false>;
      cudaError_t e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1, sfz::NT, L.total);
      if (e1 == cudaSuccess) e1 = cudaGetDevice(&dev);
      if (e1 == cudaSuccess) e1 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e1 != cudaSuccess) return cuda_fail(s, e1);
      if (per_sm * sms < s->n_cta) return fail(s, LR_ERR_CUDA, "split schedule: CTAs do not fit at once");
      e1 = cudaMemsetAsync(a.flag, 0, (size_t)s->T * sizeof(int), st);
      if (e1 != cudaSuccess) return cuda_fail(s, e1);
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(s->n_cta);
      cfg.blockDim = dim3(sfz::NT);
      cfg.dynamicSmemBytes = L.total;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      e1 = s->gram_tc ? cudaLaunchKernelEx(&cfg, sfz::sf_kernel<false, true>, a)
                      : cudaLaunchKernelEx(&cfg, sfz::sf_kernel<false, false>, a);
      if (e1 != cudaSuccess) return cuda_fail(s, e1);
    } else {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(s->n_cta);
      cfg.blockDim = dim3(sfz::NT);
      cfg.dynamicSmemBytes = L.total;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = a.C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      const cudaError_t e1 =
          a.C > 1 ? (s->gram_tc ? cudaLaunchKernelEx(&cfg, sfz::sf_kernel<true, true>, a)
                                : cudaLaunchKernelEx(&cfg, sfz::sf_kernel<true, false>, a))
                  : (s->gram_tc ? cudaLaunchKernelEx(&cfg, sfz::sf_kernel<false, true>, a)
                                : cudaLaunchKernelEx(&cfg, sfz::sf_kernel<false, false>, a));
      if (e1 != cudaSuccess) return cuda_fail(s, e1);
    }
  } else if (s->fp32) {
    launch_step_kernels<float2>(s, d, p, s->step, n_steps, dt, st);
  } else {
    launch_step_kernels<double2>(s, d, p, s->step, n_steps, dt, st);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(s, e);
  s->step += n_steps;
  return LR_OK;
}

extern "C" lr_status lr_sparse_observables(lr_sparse* s, double* beta, double* pops, double* nphot, double* trace,
                                           void* stream) {
  if (!s) return LR_ERR_ARG;
  if (!s->ws) return fail(s, LR_ERR_WORKSPACE, "no workspace bound");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(s, e);
  unsigned err = 0;
  if ((e = cudaMemcpy(&err, s->ws + s->o_err, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(s, e);
  struct Down {
    void* dst;
    size_t off, bytes;
  } downs[] = {{beta, s->o_beta, (size_t)s->T * (s->max_steps + 1) * sizeof(double2)},
               {pops, s->o_pops, (size_t)s->T * s->n_rec * s->n_levels * sizeof(double)},
               {nphot, s->o_nphot, (size_t)s->T * s->n_rec * sizeof(double)},
               {trace, s->o_trace, (size_t)s->T * s->n_rec * sizeof(double)}};
  for (const Down& dn : downs)
    if (dn.dst && (e = cudaMemcpy(dn.dst, s->ws + dn.off, dn.bytes, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(s, e);
  if (err == DEV_NOT_PD) return fail(s, LR_ERR_NOT_PD, "Gram matrix not positive definite");
  if (err == DEV_NONFINITE) return fail(s, LR_ERR_NONFINITE, "non-finite state or signal");
  if (err) return fail(s, LR_ERR_CUDA, "device error");
  return LR_OK;
}

extern "C" lr_status lr_sparse_loss(lr_sparse* s, double eta, double kappa, double gamma, double* eps_a, double* ion,
                                    double* loss, void* stream) {
  if (!s) return LR_ERR_ARG;
  if (!s->ws) return fail(s, LR_ERR_WORKSPACE, "no workspace bound");
  if (s->T % 2) return fail(s, LR_ERR_ARG, "trajectories must come in (g, e) pairs");
  if (!(eta > 0.0) || !(kappa >= 0.0) || !(gamma >= 0.0) || !isfinite(eta + kappa + gamma))
    return fail(s, LR_ERR_ARG, "bad eta, kappa or gamma");
  if (s->step < 1 || !(s->dt > 0.0)) return fail(s, LR_ERR_STATE, "no integrated steps");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nc = s->T / 2;
  double* dout = reinterpret_cast<double*>(s->ws + s->o_loss);
  sp_loss<<<nc, SP_T, 0, st>>>(dev(s), params(s), s->step, s->dt, eta, kappa, gamma, dout);
  cudaError_t e;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(s, e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(s, e);
  std::vector<double> h((size_t)nc * 3);
  if ((e = cudaMemcpy(h.data(), dout, h.size() * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(s, e);
  for (int c = 0; c < nc; ++c) {
    if (eps_a) eps_a[c] = h[3 * c];
    if (ion) ion[c] = h[3 * c + 1];
    if (loss) loss[c] = h[3 * c + 2];
  }
  return LR_OK;
}

extern "C" lr_status lr_sparse_query(const lr_sparse* s, int* fused, int* team, int* gram_tc) {
  if (!s || !fused) return LR_ERR_ARG;
  *fused = s->fused;
  if (team) *team = s->fused ? s->team_c : 0;
  if (gram_tc) *gram_tc = s->fused ? s->gram_tc : 0;
  return LR_OK;
}

extern "C" const char* lr_sparse_last_error(const lr_sparse* s) { return s ? s->msg.c_str() : "null context"; }

extern "C" void lr_sparse_destroy(lr_sparse* s) { delete s; }
