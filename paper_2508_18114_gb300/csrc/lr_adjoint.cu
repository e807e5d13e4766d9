// Discrete adjoint of the RK4 integration of Eq. S5: gradient of the
// assignment errors (Sec. S3.A) with respect to the pulse parameters.
//
// Loss and cotangents. eps_a = erfc(SNR/2)/2 + tau gamma/2 with
// SNR = sqrt(2 eta kappa S), S = dt sum_n w_n |beta_e(n) - beta_g(n)|^2
// (trapezoid weights w_n). With d eps/d S = -exp(-SNR^2/4) eta kappa /
// (2 sqrt(pi) SNR), the readout signal beta(n) = tr(Z_n^dag r Z_n) of
// trajectory e receives the complex cotangent g(n) = dL/dRe + i dL/dIm =
// dL/d eps * d eps/d S * dt * w_n * 2 (beta_e - beta_g)(n), and g -> -g for g.
// For a real loss with dL = Re tr(Zbar^dag dZ), beta contributes
// Zbar += conj(g) r Z + g r^dag Z.
//
// RK4 (stage inputs U_0 = Z, U_1 = Z + h/2 K_1, U_2 = Z + h/2 K_2,
// U_3 = Z + h K_3, K_{s+1} = F(U_s)) reversed: with Zbar' = lambda,
//   Kbar_4 = h/6 lambda,               Ubar_3 = J(U_3)^dag Kbar_4
//   Kbar_3 = h/3 lambda + h   Ubar_3,  Ubar_2 = J(U_2)^dag Kbar_3
//   Kbar_2 = h/3 lambda + h/2 Ubar_2,  Ubar_1 = J(U_1)^dag Kbar_2
//   Kbar_1 = h/6 lambda + h/2 Ubar_1,  Ubar_0 = J(U_0)^dag Kbar_1
//   lambda_n = lambda + sum_s Ubar_s + (beta(n) cotangent).
//
// Vector-Jacobian product of F(U) = -i H_eff U + sum_k 1/2 a_k (l_k U) X_k'^dag,
// X_k' = G^-1 U^dag l_k U (L_k = sqrt(a_k) l_k, a = kappa, gamma), for a
// cotangent Fbar (derived from dF with dG = dU^dag U + U^dag dU):
//   E_k' = (l_k U)^dag Fbar G^-1,   P_k' = X_k' E_k' + (X_k' E_k')^dag,
//   Ubar = i H_eff^dag Fbar + sum_k a_k/2 [ l_k^dag (Fbar X_k' + U E_k'^dag)
//          + (l_k U) E_k' - U P_k' ].
// The pulse enters only through c(t) (r + r^dag): theta_bar_i +=
// Im tr(Fbar^dag (r + r^dag) U) dc/dtheta_i at the stage time.
//
// The forward recomputation uses the plain engine's kernels; states are stored
// every `ckpt_every` steps and each segment is recomputed step by step.
//
// Precision follows the context. FP64 context: everything in complex128 /
// FP64. FP32-bulk context: the states, stage inputs, cotangents and every
// per-element product (operator apply, projection terms, the VJP rows, the
// partial sums of (l_k U)^dag Fbar and T_k) in complex64 / FP32; the Gram
// matrix summed from exact products of the FP32 entries in double-word FP32;
// the Cholesky factor, G^-1, X_k', E_k', P_k' (M x M) in FP64 (rounded once to FP32 for the
// per-element kernels); the readout signal, the trapezoid weights and the
// pulse-parameter gradient accumulated in FP64.
#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "lr_internal.cuh"

namespace lr {
namespace adj {

constexpr int AT = 256;
constexpr int AR = 16;   // rows per partial block (as the plain engine)
constexpr int MR2 = LR_MAX_RANK * LR_MAX_RANK;

struct Ptrs {
  const TrajDev* traj;
  const PulseDev* pulse;
  unsigned* err;
  double2* Xs;      // [4][n_traj][2][MR2]  X_k' of each stage (row-major M x M)
  double2* Gi;      // [4][n_traj][MR2]     G^-1 of each stage
  double2* EP;      // [n_traj][4][MR2]     E_r', E_b', P_r', P_b'
  float2* Xs32;     // FP32-bulk adjoint: FP32 copies of Xs and EP (else null);
  float2* EP32;     // EP32 [n_traj][6][MR2] also holds E_r', E_b' transposed
  const double* part;
  double* bpart;
  double* thbar;    // [n_traj][8]
  const double2* beta;
  long bstride;     // beta entries per trajectory
  const double* gcoef;   // [n_cand]
  int n_traj;
  double tau, dt;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) { return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }  // conj(a) b
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return mk(s * a.x, s * a.y); }

// Reduce the plain partials of stage input U_s, factorise G, form G^-1 and X_k'.
__global__ void __launch_bounds__(AT) adj_factor(Ptrs a, int stage) {
  const int tj = blockIdx.x;
  const TrajDev d = a.traj[tj];
  const int M = d.M, MM = M * M, tid = threadIdx.x;
  __shared__ double2 L[LR_MAX_RANK][LR_MAX_RANK + 1];
  __shared__ double2 W[LR_MAX_RANK][LR_MAX_RANK + 1];
  __shared__ double2 T[2][LR_MAX_RANK][LR_MAX_RANK + 1];
  __shared__ double rinv[LR_MAX_RANK];
  __shared__ int bad;
  const double* P = a.part + d.p_off;
  const size_t ps = plain_pstride(M);
  if (tid == 0) bad = 0;
  for (int e = tid; e < 3 * MM; e += AT) {
    const int mat = e / MM, ij = e - mat * MM, i = ij / M, j = ij - (ij / M) * M;
    if (mat == 0 && i > j) continue;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < d.nblk; ++b) {
      re += P[b * ps + 2 * e];
      im += P[b * ps + 2 * e + 1];
    }
    if (mat == 0) {
      L[i][j] = mk(re, i == j ? 0.0 : im);
      L[j][i] = mk(re, i == j ? 0.0 : -im);
    } else {
      T[mat - 1][i][j] = mk(re, im);
    }
  }
  __syncthreads();
  for (int k = 0; k < M; ++k) {
    if (tid == 0) {
      double piv = L[k][k].x;
      if (!(piv > 0.0) || !isfinite(piv)) {
        bad = 1;
        piv = 1.0;
      }
      const double sd = sqrt(piv);
      L[k][k] = mk(sd, 0.0);
      rinv[k] = 1.0 / sd;
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < M; i += AT) L[i][k] = cscale(rinv[k], L[i][k]);
    __syncthreads();
    const int w = M - k - 1;
    for (int e = tid; e < w * w; e += AT) {
      const int i = k + 1 + e / w, j = k + 1 + e % w;
      if (j > i) continue;
      const double2 x = L[i][k], y = L[j][k];
      L[i][j] = mk(L[i][j].x - (x.x * y.x + x.y * y.y), L[i][j].y - (x.y * y.x - x.x * y.y));
    }
    __syncthreads();
  }
  if (tid == 0 && bad) set_error(a.err, DEV_NOT_PD);
  // W = L^-1
  for (int e = tid; e < MM; e += AT) {
    const int i = e / M, j = e - i * M;
    W[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < M; ++k) {
    for (int j = tid; j <= k; j += AT) W[k][j] = cscale(rinv[k], W[k][j]);
    __syncthreads();
    const int rows = M - k - 1;
    for (int e = tid; e < rows * (k + 1); e += AT) {
      const int i = k + 1 + e / (k + 1), j = e % (k + 1);
      W[i][j] = mk(W[i][j].x - (L[i][k].x * W[k][j].x - L[i][k].y * W[k][j].y),
                   W[i][j].y - (L[i][k].x * W[k][j].y + L[i][k].y * W[k][j].x));
    }
    __syncthreads();
  }
  double2* Gi = a.Gi + ((size_t)stage * a.n_traj + tj) * MR2;
  // G^-1 = W^dag W into L (reuse)
  for (int e = tid; e < MM; e += AT) {
    const int i = e / M, j = e - i * M;
    double2 s = mk(0.0, 0.0);
    for (int k = max(i, j); k < M; ++k) s = cadd(s, cmulc(W[k][i], W[k][j]));
    Gi[i * M + j] = s;
  }
  __syncthreads();
  // X_k' = G^-1 T_k
  double2* X = a.Xs + (((size_t)stage * a.n_traj + tj) * 2) * MR2;
  float2* X32 = a.Xs32 ? a.Xs32 + (((size_t)stage * a.n_traj + tj) * 2) * MR2 : nullptr;
  for (int e = tid; e < 2 * MM; e += AT) {
    const int k = e / MM, ij = e - k * MM, i = ij / M, j = ij - (ij / M) * M;
    double2 s = mk(0.0, 0.0);
    for (int l = 0; l < M; ++l) s = cadd(s, cmul(Gi[i * M + l], T[k][l][j]));
    X[k * MR2 + ij] = s;
    if (X32) X32[k * MR2 + ij] = make_float2((float)s.x, (float)s.y);
  }
}

// Partial sums of B_k' = (l_k U)^dag Fbar and w = tr(Fbar^dag (r + r^dag) U) per row block.
// Fbar = ca lam + cb Un (cb == 0: Un unused). B_k' in the bulk arithmetic, w in FP64.
template <typename T2>
__global__ void __launch_bounds__(AT) adj_bpart(Ptrs a, const T2* __restrict__ U, const T2* __restrict__ lam,
                                                const T2* __restrict__ Un, double ca_d, double cb_d) {
  using T = typename real_of<T2>::type;
  const TrajDev d = a.traj[blockIdx.y];
  const int b = blockIdx.x;
  if (b >= d.nblk) return;
  __shared__ T2 sF[AR][LR_MAX_RANK], sR[AR][LR_MAX_RANK], sB[AR][LR_MAX_RANK];
  __shared__ double2 wpart[AT];
  const int M = d.M, ld = d.ld, r0 = b * AR, rows = min(AR, d.N - r0);
  const size_t off = d.z_off;
  const int st = d.Nr * d.Nf;
  const T ca = (T)ca_d, cb = (T)cb_d;
  double2 wsum = mk(0.0, 0.0);
  for (int e = threadIdx.x; e < AR * M; e += AT) {
    const int i = e / M, m = e - (e / M) * M;
    T2 f = mkc<T2>(0, 0), zr = mkc<T2>(0, 0), zb = mkc<T2>(0, 0);
    if (i < rows) {
      const int n = r0 + i;
      const size_t o = off + (size_t)n * ld + m;
      const T2 l0 = lam[o];
      f = mkc<T2>(ca * l0.x, ca * l0.y);
      if (cb_d != 0.0) {
        const T2 u0 = Un[o];
        f = mkc<T2>(f.x + cb * u0.x, f.y + cb * u0.y);
      }
      const RowIdx ri = row_index(d, n);
      const int iro = readout_index(d, ri), dro = readout_dim(d);
      T2 xd = mkc<T2>(0, 0);
      if (iro + 1 < dro) {
        const T c = (T)sqrt(iro + 1.0);
        const T2 v = U[o + ld];
        zr = mkc<T2>(c * v.x, c * v.y);
        xd = zr;
      }
      if (iro >= 1) {
        const T c = (T)sqrt((double)iro);
        const T2 v = U[o - ld];
        xd = mkc<T2>(xd.x + c * v.x, xd.y + c * v.y);
      }
      if (ri.it + 1 < d.Nt) {
        const T c = (T)sqrt(ri.it + 1.0);
        const T2 v = U[o + (size_t)st * ld];
        zb = mkc<T2>(c * v.x, c * v.y);
      }
      // conj(f) xd, summed in FP64
      wsum = cadd(wsum, cmulc(mk((double)f.x, (double)f.y), mk((double)xd.x, (double)xd.y)));
    }
    sF[i][m] = f;
    sR[i][m] = zr;
    sB[i][m] = zb;
  }
  wpart[threadIdx.x] = wsum;
  __syncthreads();
  double* out = a.bpart + d.p_off + (size_t)b * plain_pstride(M);
  const int MM = M * M;
  for (int e = threadIdx.x; e < 2 * MM; e += AT) {
    const int k = e / MM, ij = e - k * MM, i = ij / M, j = ij - (ij / M) * M;
    T re = 0, im = 0;
    for (int r = 0; r < rows; ++r) {
      const T2 x = k == 0 ? sR[r][i] : sB[r][i], y = sF[r][j];   // conj(x) y
      re = fma(x.x, y.x, fma(x.y, y.y, re));
      im = fma(x.x, y.y, fma(-x.y, y.x, im));
    }
    out[2 * e] = (double)re;
    out[2 * e + 1] = (double)im;
  }
  if (threadIdx.x == 0) {
    double2 w = mk(0.0, 0.0);
    for (int t = 0; t < AT; ++t) w = cadd(w, wpart[t]);
    out[4 * MM] = w.x;
    out[4 * MM + 1] = w.y;
  }
}

// Reduce B_k' and w; E_k' = B_k' G^-1, P_k' = X_k' E_k' + (X_k' E_k')^dag;
// theta_bar += Im(w) dc/dtheta at the stage time.
__global__ void __launch_bounds__(AT) adj_bsolve(Ptrs a, int stage, double t_stage) {
  const int tj = blockIdx.x;
  const TrajDev d = a.traj[tj];
  const int M = d.M, MM = M * M, tid = threadIdx.x;
  __shared__ double2 B[2][LR_MAX_RANK][LR_MAX_RANK + 1];
  __shared__ double2 E[2][LR_MAX_RANK][LR_MAX_RANK + 1];
  __shared__ double2 XE[2][LR_MAX_RANK][LR_MAX_RANK + 1];
  const double* P = a.bpart + d.p_off;
  const size_t ps = plain_pstride(M);
  for (int e = tid; e < 2 * MM + 1; e += AT) {
    double re = 0.0, im = 0.0;
    for (int b = 0; b < d.nblk; ++b) {
      re += P[b * ps + 2 * e];
      im += P[b * ps + 2 * e + 1];
    }
    if (e < 2 * MM) {
      const int k = e / MM, ij = e - k * MM;
      B[k][ij / M][ij % M] = mk(re, im);
    } else {
      double dc[8];
      pulse_coefficient_grad(a.pulse[d.cand], a.tau, t_stage, dc);
      for (int i = 0; i < 8; ++i) a.thbar[(size_t)tj * 8 + i] += im * dc[i];
    }
  }
  __syncthreads();
  const double2* Gi = a.Gi + ((size_t)stage * a.n_traj + tj) * MR2;
  const double2* X = a.Xs + (((size_t)stage * a.n_traj + tj) * 2) * MR2;
  for (int e = tid; e < 2 * MM; e += AT) {
    const int k = e / MM, ij = e - k * MM, i = ij / M, j = ij - (ij / M) * M;
    double2 s = mk(0.0, 0.0);
    for (int l = 0; l < M; ++l) s = cadd(s, cmul(B[k][i][l], Gi[l * M + j]));
    E[k][i][j] = s;
  }
  __syncthreads();
  for (int e = tid; e < 2 * MM; e += AT) {
    const int k = e / MM, ij = e - k * MM, i = ij / M, j = ij - (ij / M) * M;
    double2 s = mk(0.0, 0.0);
    for (int l = 0; l < M; ++l) s = cadd(s, cmul(X[k * MR2 + i * M + l], E[k][l][j]));
    XE[k][i][j] = s;
  }
  __syncthreads();
  double2* EP = a.EP + (size_t)tj * 4 * MR2;
  float2* EP32 = a.EP32 ? a.EP32 + (size_t)tj * 6 * MR2 : nullptr;
  for (int e = tid; e < 2 * MM; e += AT) {
    const int k = e / MM, ij = e - k * MM, i = ij / M, j = ij - (ij / M) * M;
    const double2 ev = E[k][i][j];
    EP[k * MR2 + ij] = ev;
    const double2 p = XE[k][i][j], q = XE[k][j][i];
    const double2 pv = mk(p.x + q.x, p.y - q.y);
    EP[(2 + k) * MR2 + ij] = pv;
    if (EP32) {
      EP32[k * MR2 + ij] = make_float2((float)ev.x, (float)ev.y);
      EP32[(2 + k) * MR2 + ij] = make_float2((float)pv.x, (float)pv.y);
      EP32[(4 + k) * MR2 + j * M + i] = make_float2((float)ev.x, (float)ev.y);   // E_k' transposed
    }
  }
}

// Ubar_s per element (n, m) for the cotangent Fbar = ca lam + cb Un.
template <typename T2>
__global__ void __launch_bounds__(AT) adj_vjp(Ptrs a, const T2* __restrict__ U, const T2* __restrict__ lam,
                                              const T2* __restrict__ Un, double ca_d, double cb_d, double t_stage,
                                              T2* __restrict__ Ub) {
  using T = typename real_of<T2>::type;
  constexpr bool f32 = sizeof(T) == 4;
  const int tj = blockIdx.y;
  const TrajDev d = a.traj[tj];
  const int M = d.M, ld = d.ld;
  const size_t off = d.z_off;
  const int st = d.Nr * d.Nf, sr = d.Nf;
  __shared__ double coef;
  if (threadIdx.x == 0) coef = pulse_coefficient(a.pulse[d.cand], a.tau, t_stage);
  __syncthreads();
  // M x M factors of this trajectory and stage (FP64, or their FP32 copies)
  const T2* EP;
  const T2* Xt;
  if constexpr (f32) {
    EP = a.EP32 + (size_t)tj * 6 * MR2;    // E_r', E_b', P_r', P_b', then E_r', E_b' transposed
    Xt = a.Xs32 + (size_t)tj * 2 * MR2;    // a.Xs32 points at this stage's [traj][2][MR2]
  } else {
    EP = a.EP + (size_t)tj * 4 * MR2;
    Xt = a.Xs + (size_t)tj * 2 * MR2;
  }
  const T ca = (T)ca_d, cb = (T)cb_d, cf = (T)coef;
  const long total = (long)d.N * M;
  auto F = [&](size_t o) {
    const T2 l0 = lam[o];
    T2 f = mkc<T2>(ca * l0.x, ca * l0.y);
    if (cb_d != 0.0) {
      const T2 u0 = Un[o];
      f = mkc<T2>(f.x + cb * u0.x, f.y + cb * u0.y);
    }
    return f;
  };
  auto cmul_t = [](T2 x, T2 y) { return mkc<T2>(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); };
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int n = (int)(idx / M), m = (int)(idx - (long)n * M);
    const RowIdx ri = row_index(d, n);
    double dre, dim_;
    heff_diag(d, ri, 0.0, dre, dim_);   // the adjoint runs in the lab frame
    const size_t o = off + (size_t)n * ld + m;
    const T2 f0 = F(o);
    // i H_eff^dag Fbar: diagonal i conj(h) = i dre + dim
    T2 acc;
    if constexpr (f32) {
      const T dh = (T)dre, dl = (T)(dre - (double)dh), di = (T)dim_;
      acc = mkc<T2>(fma(-dh, f0.y, fma(-dl, f0.y, di * f0.x)), fma(dh, f0.x, fma(dl, f0.x, di * f0.y)));
    } else {
      acc = mkc<T2>(-dre * f0.y + dim_ * f0.x, dre * f0.x + dim_ * f0.y);
    }
    T hr = 0, hi = 0;   // sum of real off-diagonal H entries times Fbar
    for (int sa = -1; sa <= 1; sa += 2) {
      const int it2 = ri.it + sa;
      if (it2 < 0 || it2 >= d.Nt) continue;
      const double ct = sqrt((double)max(ri.it, it2));
      for (int sb = -1; sb <= 1; sb += 2) {
        const int ir2 = ri.ir + sb;
        if (ir2 < 0 || ir2 >= d.Nr) continue;
        const T w = (T)(d.g * ct * sqrt((double)max(ri.ir, ir2)));
        const T2 v = F(off + (size_t)(n + sa * st + sb * sr) * ld + m);
        hr += w * v.x;
        hi += w * v.y;
      }
    }
    if (d.n_modes == 3) {
      for (int sa = -1; sa <= 1; sa += 2) {
        const int ir2 = ri.ir + sa;
        if (ir2 < 0 || ir2 >= d.Nr) continue;
        const double cr = sqrt((double)max(ri.ir, ir2));
        for (int sb = -1; sb <= 1; sb += 2) {
          const int if2 = ri.iff + sb;
          if (if2 < 0 || if2 >= d.Nf) continue;
          const T w = (T)(d.J * cr * sqrt((double)max(ri.iff, if2)));
          const T2 v = F(off + (size_t)(n + sa * sr + sb) * ld + m);
          hr += w * v.x;
          hi += w * v.y;
        }
      }
    }
    const int iro = readout_index(d, ri), dro = readout_dim(d);
    for (int sa = -1; sa <= 1; sa += 2) {
      const int i2 = iro + sa;
      if (i2 < 0 || i2 >= dro) continue;
      const T w = cf * (T)sqrt((double)max(iro, i2));
      const T2 v = F(off + (size_t)(n + sa) * ld + m);
      hr += w * v.x;
      hi += w * v.y;
    }
    acc = mkc<T2>(acc.x - hi, acc.y + hr);   // i * (H_off Fbar)
    // projection terms, k = r (stride 1, readout index), k = b (stride st, transmon index)
    for (int k = 0; k < 2; ++k) {
      const double ak = k == 0 ? d.kappa : d.gamma;
      if (ak == 0.0) continue;
      const int idx_k = k == 0 ? iro : ri.it;
      const int dim_k = k == 0 ? dro : d.Nt;
      const int s_k = k == 0 ? 1 : st;
      const T2* Xk = Xt + (size_t)k * MR2;
      const T2* Ek = EP + (size_t)k * MR2;
      const T2* Pk = EP + (size_t)(2 + k) * MR2;
      // E_k'[m][l] for the lanes' consecutive m: the transposed copy (FP32) keeps
      // the loads of a warp contiguous
      const T2* EkT = f32 ? EP + (size_t)(4 + k) * MR2 : nullptr;
      T2 t = mkc<T2>(0, 0);
      if (idx_k >= 1) {          // l_k^dag (Fbar X_k' + U E_k'^dag) at row n - s_k
        const size_t om = off + (size_t)(n - s_k) * ld;
        T2 s1 = mkc<T2>(0, 0);
        for (int l = 0; l < M; ++l) {
          const T2 p1 = cmul_t(F(om + l), Xk[l * M + m]);
          const T2 e = f32 ? EkT[l * M + m] : Ek[m * M + l];
          const T2 p2 = cmul_t(U[om + l], mkc<T2>(e.x, -e.y));
          s1 = mkc<T2>(s1.x + p1.x + p2.x, s1.y + p1.y + p2.y);
        }
        const T c = (T)sqrt((double)idx_k);
        t = mkc<T2>(t.x + c * s1.x, t.y + c * s1.y);
      }
      if (idx_k + 1 < dim_k) {   // (l_k U) E_k'
        const size_t op = off + (size_t)(n + s_k) * ld;
        T2 s2 = mkc<T2>(0, 0);
        for (int l = 0; l < M; ++l) {
          const T2 p = cmul_t(U[op + l], Ek[l * M + m]);
          s2 = mkc<T2>(s2.x + p.x, s2.y + p.y);
        }
        const T c = (T)sqrt(idx_k + 1.0);
        t = mkc<T2>(t.x + c * s2.x, t.y + c * s2.y);
      }
      {                          // - U P_k'
        const size_t on = off + (size_t)n * ld;
        T2 s3 = mkc<T2>(0, 0);
        for (int l = 0; l < M; ++l) {
          const T2 p = cmul_t(U[on + l], Pk[l * M + m]);
          s3 = mkc<T2>(s3.x + p.x, s3.y + p.y);
        }
        t = mkc<T2>(t.x - s3.x, t.y - s3.y);
      }
      const T h = (T)(0.5 * ak);
      acc = mkc<T2>(acc.x + h * t.x, acc.y + h * t.y);
    }
    Ub[o] = acc;
  }
}

// lam_new = lam + sum_s Ubar_s + conj(g) r Z + g r^dag Z (readout cotangent of step n).
template <typename T2>
__global__ void __launch_bounds__(AT) adj_update(Ptrs a, const T2* __restrict__ Z, const T2* __restrict__ lam,
                                                 const T2* __restrict__ U0, const T2* __restrict__ U1,
                                                 const T2* __restrict__ U2, const T2* __restrict__ U3,
                                                 T2* __restrict__ lam_new, long step, long S, int with_sum) {
  using T = typename real_of<T2>::type;
  const int tj = blockIdx.y;
  const TrajDev d = a.traj[tj];
  const int M = d.M, ld = d.ld;
  const size_t off = d.z_off;
  const int c = d.cand;
  const double2 be = a.beta[(size_t)(2 * c + 1) * a.bstride + step];
  const double2 bg = a.beta[(size_t)(2 * c) * a.bstride + step];
  const double w = (step == 0 || step == S) ? 0.5 : 1.0;
  const double sg = (tj & 1) ? 1.0 : -1.0;
  const double gs = sg * a.gcoef[c] * w;
  const T gx = (T)(gs * (be.x - bg.x)), gy = (T)(gs * (be.y - bg.y));
  const long total = (long)d.N * M;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int n = (int)(idx / M), m = (int)(idx - (long)n * M);
    const size_t o = off + (size_t)n * ld + m;
    T vx = 0, vy = 0;
    if (with_sum) {
      const T2 l0 = lam[o], a0 = U0[o], a1 = U1[o], a2 = U2[o], a3 = U3[o];
      vx = l0.x + ((a0.x + a1.x) + (a2.x + a3.x));
      vy = l0.y + ((a0.y + a1.y) + (a2.y + a3.y));
    }
    const RowIdx ri = row_index(d, n);
    const int iro = readout_index(d, ri), dro = readout_dim(d);
    if (iro + 1 < dro) {   // conj(g) r Z
      const T cc = (T)sqrt(iro + 1.0);
      const T2 z = Z[o + ld];
      const T zx = cc * z.x, zy = cc * z.y;
      vx += gx * zx + gy * zy;
      vy += gx * zy - gy * zx;
    }
    if (iro >= 1) {        // g r^dag Z
      const T cc = (T)sqrt((double)iro);
      const T2 z = Z[o - ld];
      const T zx = cc * z.x, zy = cc * z.y;
      vx += gx * zx - gy * zy;
      vy += gx * zy + gy * zx;
    }
    lam_new[o] = mkc<T2>(vx, vy);
  }
}

// gcoef[c] = dL/deps_c * d eps/dS * dt * 2 from the recomputed readout signals.
__global__ void adj_gcoef(Ptrs a, const double* __restrict__ deps, double eta, long S, double* gcoef) {
  const int c = blockIdx.x;
  __shared__ double sh[AT];
  const double2* bg = a.beta + (size_t)(2 * c) * a.bstride;
  const double2* be = a.beta + (size_t)(2 * c + 1) * a.bstride;
  double acc = 0.0;
  for (long i = threadIdx.x; i <= S; i += AT) {
    const double dx = be[i].x - bg[i].x, dy = be[i].y - bg[i].y;
    acc += ((i == 0 || i == S) ? 0.5 : 1.0) * (dx * dx + dy * dy);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int t = 0; t < AT; ++t) s += sh[t];
    const TrajDev d = a.traj[2 * c];
    const double Sint = a.dt * s;
    const double snr = sqrt(2.0 * eta * d.kappa * Sint);
    double dEdS = 0.0;
    if (snr > 0.0) dEdS = -exp(-0.25 * snr * snr) * eta * d.kappa / (2.0 * sqrt(M_PI) * snr);
    gcoef[c] = deps[c] * dEdS * a.dt * 2.0;
  }
}

}  // namespace adj

// ------------------------------------------------------------------ driver

BwdLayout bwd_layout(long long tot, int n_traj, int n_cand, int nt_max, size_t part_doubles, long S, int K, int fp32) {
  BwdLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = (o + bytes + 255) / 256 * 256;
    return at;
  };
  const size_t T = (fp32 ? sizeof(float2) : sizeof(double2)) * (size_t)tot;
  L.K = K;
  L.fp32 = fp32;
  L.n_seg = (S + K - 1) / K;
  L.ck = take(T * L.n_seg);
  L.seg = take(T * (K + 1));
  L.cur = take(T);
  L.za = take(T);
  L.zb = take(T);
  L.acc = take(T);
  L.U = take(T * 4);
  L.Ub = take(T * 4);
  L.lam = take(T);
  L.lamn = take(T);
  L.X = take(sizeof(double2) * 2 * adj::MR2 * n_traj);
  L.part = take(sizeof(double) * part_doubles);
  L.Xs = take(sizeof(double2) * 4 * 2 * adj::MR2 * n_traj);
  L.Gi = take(sizeof(double2) * 4 * adj::MR2 * n_traj);
  L.EP = take(sizeof(double2) * 4 * adj::MR2 * n_traj);
  L.Xs32 = fp32 ? take(sizeof(float2) * 4 * 2 * adj::MR2 * n_traj) : 0;
  L.EP32 = fp32 ? take(sizeof(float2) * 6 * adj::MR2 * n_traj) : 0;
  L.bpart = take(sizeof(double) * part_doubles);
  L.beta = take(sizeof(double2) * n_traj * (size_t)(S + 1));
  L.pops = take(sizeof(double) * n_traj * nt_max);
  L.nphot = take(sizeof(double) * n_traj);
  L.trace = take(sizeof(double) * n_traj);
  L.gcoef = take(sizeof(double) * n_cand);
  L.deps = take(sizeof(double) * n_cand);
  L.thbar = take(sizeof(double) * 8 * n_traj);
  L.total = o;
  return L;
}

namespace {

template <typename T2>
cudaError_t backward_t(const DevPtrs& main, const RunParams& rp0, char* ws, const BwdLayout& L, long long tot,
                       int max_nblk, int max_N, long S, const void* z0, int z0_fp32, const double* deps_host,
                       double* dtheta_host, cudaStream_t s) {
  constexpr bool f32 = sizeof(T2) == sizeof(float2);
  const size_t T = sizeof(T2) * (size_t)tot;
  auto P2 = [&](size_t off) { return reinterpret_cast<double2*>(ws + off); };
  auto PS = [&](size_t off) { return reinterpret_cast<T2*>(ws + off); };
  cudaError_t e;
  // plain-engine pointers for the forward recomputation
  DevPtrs p{};
  p.traj = main.traj;
  p.pulse = main.pulse;
  p.err = main.err;
  p.Zn = ws + L.cur;
  p.Za = ws + L.za;
  p.Zb = ws + L.zb;
  p.acc = ws + L.acc;
  p.X = P2(L.X);
  p.part = reinterpret_cast<double*>(ws + L.part);
  p.beta = P2(L.beta);
  p.pops = reinterpret_cast<double*>(ws + L.pops);
  p.nphot = reinterpret_cast<double*>(ws + L.nphot);
  p.trace = reinterpret_cast<double*>(ws + L.trace);
  RunParams rp = rp0;
  rp.max_steps = S;
  rp.n_rec = 1;
  rp.pop_every = INT_MAX;
  adj::Ptrs a{};
  a.traj = main.traj;
  a.pulse = main.pulse;
  a.err = main.err;
  a.Xs = P2(L.Xs);
  a.Gi = P2(L.Gi);
  a.EP = P2(L.EP);
  a.Xs32 = f32 ? reinterpret_cast<float2*>(ws + L.Xs32) : nullptr;
  a.EP32 = f32 ? reinterpret_cast<float2*>(ws + L.EP32) : nullptr;
  a.part = p.part;
  a.bpart = reinterpret_cast<double*>(ws + L.bpart);
  a.thbar = reinterpret_cast<double*>(ws + L.thbar);
  a.beta = p.beta;
  a.bstride = S + 1;
  a.gcoef = reinterpret_cast<double*>(ws + L.gcoef);
  a.n_traj = rp.n_traj;
  a.tau = rp.tau;
  a.dt = rp.dt;
  const double h = rp.dt;

  // initial state into the first checkpoint (in the adjoint's state type)
  if (z0_fp32 == (int)f32)
    e = cudaMemcpyAsync(PS(L.ck), z0, T, cudaMemcpyDeviceToDevice, s);
  else
    e = launch_convert(z0, PS(L.ck), tot, f32 ? 1 : 0, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ws + L.thbar, 0, sizeof(double) * 8 * rp.n_traj, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(ws + L.deps, deps_host, sizeof(double) * rp.n_cand, cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  // forward pass: checkpoints and the readout signal
  for (long sg = 0; sg < L.n_seg; ++sg) {
    const long s0 = sg * L.K, len = std::min<long>(L.K, S - s0);
    if ((e = cudaMemcpyAsync(p.Zn, PS(L.ck) + (size_t)sg * tot, T, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    if ((e = plain_integrate(p, rp, max_nblk, max_N, s0, len, s, f32)) != cudaSuccess) return e;
    if (sg + 1 < L.n_seg &&
        (e = cudaMemcpyAsync(PS(L.ck) + (size_t)(sg + 1) * tot, p.Zn, T, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
  }
  adj::adj_gcoef<<<rp.n_cand, adj::AT, 0, s>>>(a, reinterpret_cast<double*>(ws + L.deps), rp.eta, S,
                                                reinterpret_cast<double*>(ws + L.gcoef));
  const dim3 egrid((unsigned)std::min<long>(((long)max_N * LR_MAX_RANK + adj::AT - 1) / adj::AT, 4096), rp.n_traj);
  const dim3 pgrid(max_nblk, rp.n_traj);
  T2* lam = PS(L.lam);
  T2* lamn = PS(L.lamn);
  // lambda_S: readout cotangent of the final state
  adj::adj_update<T2><<<egrid, adj::AT, 0, s>>>(a, reinterpret_cast<const T2*>(p.Zn), lam, lam, lam, lam, lam, lam,
                                                S, S, 0);
  T2* U[4] = {nullptr, PS(L.U) + tot, PS(L.U) + 2 * tot, PS(L.U) + 3 * tot};
  T2* Ub[4] = {PS(L.Ub), PS(L.Ub) + tot, PS(L.Ub) + 2 * tot, PS(L.Ub) + 3 * tot};
  const double ca[4] = {h / 6.0, h / 3.0, h / 3.0, h / 6.0};
  const double cb[4] = {h / 2.0, h / 2.0, h, 0.0};
  const double cs[4] = {0.0, 0.5, 0.5, 1.0};
  for (long sg = L.n_seg - 1; sg >= 0; --sg) {
    const long s0 = sg * L.K, len = std::min<long>(L.K, S - s0);
    T2* seg = PS(L.seg);
    if ((e = cudaMemcpyAsync(seg, PS(L.ck) + (size_t)sg * tot, T, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    for (long i = 1; i < len; ++i) {
      if ((e = cudaMemcpyAsync(p.Zn, seg + (size_t)(i - 1) * tot, T, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
      if ((e = plain_integrate(p, rp, max_nblk, max_N, s0 + i - 1, 1, s, f32)) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(seg + (size_t)i * tot, p.Zn, T, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    }
    for (long i = len - 1; i >= 0; --i) {
      const long n = s0 + i;
      const double tn = (double)n * h;
      T2* Z = seg + (size_t)i * tot;
      U[0] = Z;
      // forward stages: U_s, G^-1, X_k', next stage input
      DevPtrs q = p;
      q.Zn = Z;
      for (int st = 0; st < 4; ++st) {
        plain_gram_launch(q, rp, max_nblk, U[st], s);
        adj::adj_factor<<<rp.n_traj, adj::AT, 0, s>>>(a, st);
        if (st < 3) {
          q.X = a.Xs + (size_t)st * rp.n_traj * 2 * adj::MR2;
          plain_rhs_launch(q, rp, max_N, U[st], U[st + 1], st, tn + cs[st] * h, s);
        }
      }
      // reverse stages
      for (int st = 3; st >= 0; --st) {
        const T2* un = st < 3 ? Ub[st + 1] : Ub[0];
        const double cbs = st < 3 ? cb[st] : 0.0;
        const double ts = tn + cs[st] * h;
        adj::adj_bpart<T2><<<pgrid, adj::AT, 0, s>>>(a, U[st], lam, un, ca[st], cbs);
        adj::adj_bsolve<<<rp.n_traj, adj::AT, 0, s>>>(a, st, ts);
        adj::Ptrs as = a;
        as.Xs = a.Xs + (size_t)st * rp.n_traj * 2 * adj::MR2;
        if (f32) as.Xs32 = a.Xs32 + (size_t)st * rp.n_traj * 2 * adj::MR2;
        adj::adj_vjp<T2><<<egrid, adj::AT, 0, s>>>(as, U[st], lam, un, ca[st], cbs, ts, Ub[st]);
      }
      adj::adj_update<T2><<<egrid, adj::AT, 0, s>>>(a, Z, lam, Ub[0], Ub[1], Ub[2], Ub[3], lamn, n, S, 1);
      std::swap(lam, lamn);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  // theta_bar per candidate = g + e trajectories
  std::vector<double> th(8 * (size_t)rp.n_traj);
  if ((e = cudaMemcpyAsync(th.data(), ws + L.thbar, sizeof(double) * th.size(), cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  for (int c = 0; c < rp.n_cand; ++c)
    for (int i = 0; i < 8; ++i) dtheta_host[8 * c + i] = th[8 * (2 * c) + i] + th[8 * (2 * c + 1) + i];
  return cudaSuccess;
}

}  // namespace

cudaError_t backward_run(const DevPtrs& main, const RunParams& rp, char* ws, const BwdLayout& L, long long tot,
                         int max_nblk, int max_N, long S, const void* z0, int z0_fp32, const double* deps_host,
                         double* dtheta_host, cudaStream_t s) {
  if (L.fp32)
    return backward_t<float2>(main, rp, ws, L, tot, max_nblk, max_N, S, z0, z0_fp32, deps_host, dtheta_host, s);
  return backward_t<double2>(main, rp, ws, L, tot, max_nblk, max_N, S, z0, z0_fp32, deps_host, dtheta_host, s);
}

}  // namespace lr
