// PLAIN engine: straightforward FP64 kernels with the state in HBM.
//
// One RK4 stage of Eq. S5 is three launches:
//   plain_gram  - per row block, partial sums of G = Z^dag Z (upper triangle),
//                 T_r = Z^dag r Z and T_b = Z^dag b Z, plus level populations
//                 and readout photons at recording steps;
//   plain_solve - one block per trajectory: reduce the partials in a fixed
//                 order, record beta = tr(T_r) at stage 1 of each step, Cholesky
//                 G = L L^dag, solve X_r = G^-1 T_r, X_b = G^-1 T_b;
//   plain_rhs   - per element: F = -i H_eff Z + 1/2 kappa (rZ) X_r^dag
//                 + 1/2 gamma (bZ) X_b^dag, then the RK4 stage update.
// With Y_k = L_k Z the projection term of Eq. S5 is 1/2 sum_k Y_k (Z^+ Y_k)^dag
// = 1/2 kappa (rZ)(G^-1 Z^dag r Z)^dag + 1/2 gamma (bZ)(G^-1 Z^dag b Z)^dag,
// and -1/2 sum_k L_k^dag L_k Z is folded into the diagonal of H_eff.
//
// The state type is a template parameter: complex128 (the reference path), or
// complex64 for the FP32-bulk recomputation inside the adjoint. With complex64
// the Gram matrix is summed from the exact products of the FP32 entries in
// double-word FP32 (FP64-class), the Cholesky factor and the solves are FP64,
// and the operator apply, T_k, the projection term and the RK4 update run in
// FP32 (the diagonal energies and the step sizes split into hi + lo floats so
// that FP32 does not round the mode frequencies or dt).
#include "lr_internal.cuh"

namespace lr {

constexpr int PR = 16;        // rows per Gram block
constexpr int PT = 256;       // threads per block

__host__ __device__ inline size_t pstride(int M) { return plain_pstride(M); }

int plain_rows_per_block() { return PR; }
size_t plain_partial_doubles(int M) { return pstride(M); }

template <typename T2>
__global__ void __launch_bounds__(PT) plain_gram(const TrajDev* __restrict__ traj, const T2* __restrict__ Zin,
                                                 double* __restrict__ part, int with_obs) {
  using T = typename real_of<T2>::type;
  const TrajDev d = traj[blockIdx.y];
  const int b = blockIdx.x;
  if (b >= d.nblk) return;
  __shared__ T2 sZ[PR][LR_MAX_RANK], sR[PR][LR_MAX_RANK], sB[PR][LR_MAX_RANK];
  __shared__ double sw[PR];
  __shared__ int slev[PR], sro[PR];
  const int M = d.M, ld = d.ld;
  const int r0 = b * PR;
  const int rows = min(PR, d.N - r0);
  const T2* Z = Zin + d.z_off;
  const int st = d.Nr * d.Nf;
  for (int e = threadIdx.x; e < PR * M; e += blockDim.x) {
    const int i = e / M, m = e - (e / M) * M;
    T2 z = mkc<T2>(0, 0), zr = mkc<T2>(0, 0), zb = mkc<T2>(0, 0);
    if (i < rows) {
      const int n = r0 + i;
      z = Z[(size_t)n * ld + m];
      const RowIdx ri = row_index(d, n);
      const int iro = readout_index(d, ri);
      if (iro + 1 < readout_dim(d)) {
        const T c = (T)sqrt(iro + 1.0);
        const T2 v = Z[(size_t)(n + 1) * ld + m];
        zr = mkc<T2>(c * v.x, c * v.y);
      }
      if (ri.it + 1 < d.Nt) {
        const T c = (T)sqrt(ri.it + 1.0);
        const T2 v = Z[(size_t)(n + st) * ld + m];
        zb = mkc<T2>(c * v.x, c * v.y);
      }
      if (m == 0) {
        slev[i] = ri.it;
        sro[i] = iro;
      }
    }
    sZ[i][m] = z;
    sR[i][m] = zr;
    sB[i][m] = zb;
  }
  __syncthreads();
  double* out = part + d.p_off + (size_t)b * pstride(M);
  const int MM = M * M;
  for (int e = threadIdx.x; e < 3 * MM; e += blockDim.x) {
    const int mat = e / MM, ij = e - mat * MM, i = ij / M, j = ij - (ij / M) * M;
    if (mat == 0 && i > j) continue;
    if (sizeof(T) == 4 && mat == 0) {
      // FP32 state: exact FP32 products (FMA TwoProduct) in double-word sums
      // (Knuth TwoSum), ~2^-48 relative: the FP64-class Gram on the FP32 pipes
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      auto acc2 = [](float& hi, float& lo, float a, float b) {
        const float p = a * b, e = fmaf(a, b, -p), t = hi + p, bp = t - hi;
        lo += ((hi - (t - bp)) + (p - bp)) + e;
        hi = t;
      };
      for (int r = 0; r < rows; ++r) {
        const T2 a = sZ[r][i], c = sZ[r][j];
        acc2(rh, rl, (float)a.x, (float)c.x);      // conj(a) * c
        acc2(rh, rl, (float)a.y, (float)c.y);
        acc2(ih, il, (float)a.x, (float)c.y);
        acc2(ih, il, -(float)a.y, (float)c.x);
      }
      out[2 * e] = (double)rh + (double)rl;
      out[2 * e + 1] = (double)ih + (double)il;
    } else if (sizeof(T) == 8 || mat == 0) {
      // FP64 sums
      double re = 0.0, im = 0.0;
      for (int r = 0; r < rows; ++r) {
        const T2 a = sZ[r][i];
        const T2 c = mat == 0 ? sZ[r][j] : (mat == 1 ? sR[r][j] : sB[r][j]);
        const double ax = a.x, ay = a.y, cx = c.x, cy = c.y;
        re = fma(ax, cx, fma(ay, cy, re));      // conj(a) * c
        im = fma(ax, cy, fma(-ay, cx, im));
      }
      out[2 * e] = re;
      out[2 * e + 1] = im;
    } else {
      T re = 0, im = 0;
      for (int r = 0; r < rows; ++r) {
        const T2 a = sZ[r][i];
        const T2 c = mat == 1 ? sR[r][j] : sB[r][j];
        re = fma(a.x, c.x, fma(a.y, c.y, re));
        im = fma(a.x, c.y, fma(-a.y, c.x, im));
      }
      out[2 * e] = (double)re;
      out[2 * e + 1] = (double)im;
    }
  }
  if (with_obs) {
    for (int i = threadIdx.x; i < PR; i += blockDim.x) {
      double w = 0.0;
      if (i < rows)
        for (int m = 0; m < M; ++m) {
          const double x = sZ[i][m].x, y = sZ[i][m].y;
          w += x * x + y * y;
        }
      sw[i] = w;
    }
    __syncthreads();
    if (threadIdx.x < LR_MAX_NT + 1) {
      const int t = threadIdx.x;
      double acc = 0.0;
      for (int i = 0; i < rows; ++i) {
        if (t < LR_MAX_NT) acc += (slev[i] == t) ? sw[i] : 0.0;
        else acc += sro[i] * sw[i];
      }
      out[6 * MM + t] = acc;
    }
  }
}

__global__ void __launch_bounds__(PT) plain_solve(DevPtrs p, RunParams rp, long step, int stage, int record,
                                                  int do_solve) {
  const int tj = blockIdx.x;
  const TrajDev d = p.traj[tj];
  const int M = d.M, MM = M * M, tid = threadIdx.x;
  __shared__ double2 L[LR_MAX_RANK][LR_MAX_RANK + 1];
  __shared__ double2 B[LR_MAX_RANK][2 * LR_MAX_RANK + 1];
  __shared__ int bad;
  const double* P = p.part + d.p_off;
  const size_t ps = pstride(M);
  if (tid == 0) bad = 0;
  for (int e = tid; e < 3 * MM; e += blockDim.x) {
    const int mat = e / MM, ij = e - mat * MM, i = ij / M, j = ij - (ij / M) * M;
    if (mat == 0 && i > j) continue;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < d.nblk; ++b) {
      re += P[b * ps + 2 * e];
      im += P[b * ps + 2 * e + 1];
    }
    if (mat == 0) {
      if (i == j) {
        L[i][i] = mk(re, 0.0);
      } else {
        L[i][j] = mk(re, im);
        L[j][i] = mk(re, -im);
      }
    } else {
      B[i][(mat - 1) * M + j] = mk(re, im);
    }
  }
  __syncthreads();
  if (stage == 0) {
    if (tid == 0) {
      double br = 0.0, bi = 0.0;
      for (int i = 0; i < M; ++i) {
        br += B[i][i].x;
        bi += B[i][i].y;
      }
      p.beta[(size_t)tj * (rp.max_steps + 1) + step] = mk(br, bi);
      if (!isfinite(br) || !isfinite(bi)) set_error(p.err, DEV_NONFINITE);
    }
    if (record && tid < LR_MAX_NT + 1) {
      double acc = 0.0;
      for (int b = 0; b < d.nblk; ++b) acc += P[b * ps + 6 * MM + tid];
      const long rec = step / rp.pop_every;
      if (tid < rp.nt_max) p.pops[((size_t)tj * rp.n_rec + rec) * rp.nt_max + tid] = tid < d.Nt ? acc : 0.0;
      if (tid == LR_MAX_NT) p.nphot[(size_t)tj * rp.n_rec + rec] = acc;
    }
    if (record && tid == 32) {
      double tr = 0.0;
      for (int i = 0; i < M; ++i) tr += L[i][i].x;
      p.trace[(size_t)tj * rp.n_rec + step / rp.pop_every] = tr;
    }
    if (record && p.gsnap) {
      double2* gs = p.gsnap + ((size_t)tj * rp.n_rec + step / rp.pop_every) * rp.snap_m * rp.snap_m;
      for (int e = tid; e < MM; e += blockDim.x) gs[(e / M) * rp.snap_m + e % M] = L[e / M][e % M];
    }
  }
  __syncthreads();   // the trace above reads the diagonal before it is factorised
  if (!do_solve) return;
  // Cholesky G = L L^dag (right-looking, lower triangle in place).
  for (int k = 0; k < M; ++k) {
    if (tid == 0) {
      double piv = L[k][k].x;
      if (!(piv > 0.0) || !isfinite(piv)) {
        bad = 1;
        piv = 1.0;
      }
      L[k][k] = mk(sqrt(piv), 0.0);
    }
    __syncthreads();
    const double inv = 1.0 / L[k][k].x;
    for (int i = k + 1 + tid; i < M; i += blockDim.x) L[i][k] = mk(L[i][k].x * inv, L[i][k].y * inv);
    __syncthreads();
    const int w = M - k - 1;
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int i = k + 1 + e / w, j = k + 1 + e % w;
      if (j > i) continue;
      const double2 a = L[i][k], c = L[j][k];   // L[i][j] -= a * conj(c)
      L[i][j] = mk(L[i][j].x - (a.x * c.x + a.y * c.y), L[i][j].y - (a.y * c.x - a.x * c.y));
    }
    __syncthreads();
  }
  if (tid == 0 && bad) set_error(p.err, DEV_NOT_PD);
  const int nc = 2 * M;
  // forward: L W = B
  for (int k = 0; k < M; ++k) {
    const double inv = 1.0 / L[k][k].x;
    for (int c = tid; c < nc; c += blockDim.x) B[k][c] = mk(B[k][c].x * inv, B[k][c].y * inv);
    __syncthreads();
    for (int e = tid; e < (M - k - 1) * nc; e += blockDim.x) {
      const int i = k + 1 + e / nc, c = e % nc;
      const double2 a = L[i][k], w = B[k][c];
      B[i][c] = mk(B[i][c].x - (a.x * w.x - a.y * w.y), B[i][c].y - (a.x * w.y + a.y * w.x));
    }
    __syncthreads();
  }
  // backward: L^dag X = W, (L^dag)[i][k] = conj(L[k][i])
  for (int k = M - 1; k >= 0; --k) {
    const double inv = 1.0 / L[k][k].x;
    for (int c = tid; c < nc; c += blockDim.x) B[k][c] = mk(B[k][c].x * inv, B[k][c].y * inv);
    __syncthreads();
    for (int e = tid; e < k * nc; e += blockDim.x) {
      const int i = e / nc, c = e % nc;
      const double2 a = L[k][i], w = B[k][c];    // conj(a) * w
      B[i][c] = mk(B[i][c].x - (a.x * w.x + a.y * w.y), B[i][c].y - (a.x * w.y - a.y * w.x));
    }
    __syncthreads();
  }
  double2* X = p.X + (size_t)tj * 2 * LR_MAX_RANK * LR_MAX_RANK;
  for (int e = tid; e < 2 * MM; e += blockDim.x) {
    const int k = e / MM, ij = e - k * MM, i = ij / M, j = ij - (ij / M) * M;
    X[k * LR_MAX_RANK * LR_MAX_RANK + ij] = B[i][k * M + j];
  }
}

template <typename T2>
__global__ void __launch_bounds__(PT) plain_rhs(DevPtrs p, RunParams rp, const T2* __restrict__ Zin,
                                                T2* __restrict__ Zout, int stage, double t) {
  using T = typename real_of<T2>::type;
  constexpr bool f32 = sizeof(T) == 4;
  const int tj = blockIdx.y;
  const TrajDev d = p.traj[tj];
  __shared__ T2 sX[2][LR_MAX_RANK * LR_MAX_RANK];
  __shared__ double coef, coef_i, wfr;
  const int M = d.M, MM = M * M, ld = d.ld;
  const double2* X = p.X + (size_t)tj * 2 * LR_MAX_RANK * LR_MAX_RANK;
  // transposed in shared memory, sX[k][l * M + m] = X_k[m][l]: the threads of a
  // warp (consecutive m) then read consecutive words (no bank conflicts)
  for (int e = threadIdx.x; e < 2 * MM; e += blockDim.x) {
    const int k = e / MM, ij = e - k * MM, i = ij / M, j = ij - i * M;
    const double2 x = X[k * LR_MAX_RANK * LR_MAX_RANK + ij];
    sX[k][j * M + i] = mkc<T2>((T)x.x, (T)x.y);
  }
  if (threadIdx.x == 0) {
    const PulseDev P = p.pulse[d.cand];
    if (rp.frame) {
      const double2 w = pulse_rwa_drive(P, rp.tau, t);
      coef = w.x;
      coef_i = w.y;
      wfr = pulse_drive_frequency(P);
    } else {
      coef = pulse_coefficient(P, rp.tau, t);
      coef_i = 0.0;
      wfr = 0.0;
    }
  }
  __syncthreads();
  const T2* Z = Zin + d.z_off;
  T2* Zn = reinterpret_cast<T2*>(p.Zn) + d.z_off;
  T2* acc = reinterpret_cast<T2*>(p.acc) + d.z_off;
  T2* Zo = Zout ? Zout + d.z_off : nullptr;
  const int st = d.Nr * d.Nf, sr = d.Nf;
  const T c = (T)coef, ci = (T)coef_i;
  const double dt = rp.dt;
  // FP32 state: step sizes as hi + lo floats
  const double hsd = stage == 2 ? dt : 0.5 * dt, h6d = dt / 6.0;
  const T hs_hi = (T)hsd, hs_lo = (T)(hsd - (double)hs_hi), h6_hi = (T)h6d, h6_lo = (T)(h6d - (double)h6_hi);
  const bool rwa = rp.frame != 0;
  const long total = (long)d.N * M;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int n = (int)(idx / M), m = (int)(idx - (long)n * M);
    const RowIdx ri = row_index(d, n);
    double dre, dim_;
    heff_diag(d, ri, wfr, dre, dim_);
    const T2 z = Z[(size_t)n * ld + m];
    T hr, hi;
    if constexpr (f32) {
      // diagonal energy as hi + lo floats: FP32 does not round the mode frequencies
      const T dh = (T)dre, dl = (T)(dre - (double)dh), di = (T)dim_;
      hr = fma(dh, z.x, fma(dl, z.x, -di * z.y));
      hi = fma(dh, z.y, fma(dl, z.y, di * z.x));
    } else {
      hr = dre * z.x - dim_ * z.y;
      hi = dre * z.y + dim_ * z.x;
    }
    // g (b + b^dag)(a + a^dag)
    for (int a = -1; a <= 1; a += 2) {
      const int it2 = ri.it + a;
      if (it2 < 0 || it2 >= d.Nt) continue;
      const double ct = sqrt((double)max(ri.it, it2));
      for (int bb = -1; bb <= 1; bb += 2) {
        const int ir2 = ri.ir + bb;
        if (ir2 < 0 || ir2 >= d.Nr) continue;
        if (rwa && a == bb) continue;   // RWA keeps g (b^dag a + b a^dag) only
        const T w = (T)(d.g * ct * sqrt((double)max(ri.ir, ir2)));
        const T2 v = Z[(size_t)(n + a * st + bb * sr) * ld + m];
        hr += w * v.x;
        hi += w * v.y;
      }
    }
    if (d.n_modes == 3) {
      // J (a + a^dag)(f + f^dag)
      for (int a = -1; a <= 1; a += 2) {
        const int ir2 = ri.ir + a;
        if (ir2 < 0 || ir2 >= d.Nr) continue;
        const double cr = sqrt((double)max(ri.ir, ir2));
        for (int bb = -1; bb <= 1; bb += 2) {
          const int if2 = ri.iff + bb;
          if (if2 < 0 || if2 >= d.Nf) continue;
          if (rwa && a == bb) continue;   // RWA keeps J (a^dag f + a f^dag) only
          const T w = (T)(d.J * cr * sqrt((double)max(ri.iff, if2)));
          const T2 v = Z[(size_t)(n + a * sr + bb) * ld + m];
          hr += w * v.x;
          hi += w * v.y;
        }
      }
    }
    // drive on the readout mode (stride 1): lab frame c(t) (r + r^dag); RWA
    // w r + conj(w) r^dag with w = c + i ci (row n gets r from n+1, r^dag from n-1)
    const int iro = readout_index(d, ri), dro = readout_dim(d);
    for (int a = -1; a <= 1; a += 2) {
      const int i2 = iro + a;
      if (i2 < 0 || i2 >= dro) continue;
      const T s = (T)sqrt((double)max(iro, i2));
      const T wr = c * s, wi = (a > 0 ? ci : -ci) * s;
      const T2 v = Z[(size_t)(n + a) * ld + m];
      hr += wr * v.x - wi * v.y;
      hi += wr * v.y + wi * v.x;
    }
    // F = -i H_eff Z
    T fr = hi, fi = -hr;
    // + 1/2 kappa (rZ) X_r^dag + 1/2 gamma (bZ) X_b^dag
    if (iro + 1 < dro) {
      const T s = (T)(0.5 * d.kappa * sqrt(iro + 1.0));
      const T2* zr = Z + (size_t)(n + 1) * ld;
      T sr_ = 0, si_ = 0;
      for (int l = 0; l < M; ++l) {
        const T2 y = zr[l], x = sX[0][l * M + m];   // y * conj(x)
        sr_ += y.x * x.x + y.y * x.y;
        si_ += y.y * x.x - y.x * x.y;
      }
      fr += s * sr_;
      fi += s * si_;
    }
    if (ri.it + 1 < d.Nt) {
      const T s = (T)(0.5 * d.gamma * sqrt(ri.it + 1.0));
      const T2* zb = Z + (size_t)(n + st) * ld;
      T sr_ = 0, si_ = 0;
      for (int l = 0; l < M; ++l) {
        const T2 y = zb[l], x = sX[1][l * M + m];
        sr_ += y.x * x.x + y.y * x.y;
        si_ += y.y * x.x - y.x * x.y;
      }
      fr += s * sr_;
      fi += s * si_;
    }
    // RK4 (weights 1/6, 1/3, 1/3, 1/6)
    const size_t o = (size_t)n * ld + m;
    const T2 zn = Zn[o];
    if constexpr (f32) {
      if (stage < 3) {
        if (stage == 0) {
          acc[o] = mkc<T2>(fr, fi);
        } else {
          const T2 a = acc[o];
          acc[o] = mkc<T2>(fma((T)2, fr, a.x), fma((T)2, fi, a.y));
        }
        Zo[o] = mkc<T2>(zn.x + fma(hs_lo, fr, hs_hi * fr), zn.y + fma(hs_lo, fi, hs_hi * fi));
      } else {
        const T2 a = acc[o];
        const T s_r = a.x + fr, s_i = a.y + fi;
        Zn[o] = mkc<T2>(zn.x + fma(h6_lo, s_r, h6_hi * s_r), zn.y + fma(h6_lo, s_i, h6_hi * s_i));
      }
    } else {
      if (stage == 0) {
        acc[o] = mkc<T2>(fr, fi);
        Zo[o] = mkc<T2>(zn.x + 0.5 * dt * fr, zn.y + 0.5 * dt * fi);
      } else if (stage == 1) {
        const T2 a = acc[o];
        acc[o] = mkc<T2>(a.x + 2.0 * fr, a.y + 2.0 * fi);
        Zo[o] = mkc<T2>(zn.x + 0.5 * dt * fr, zn.y + 0.5 * dt * fi);
      } else if (stage == 2) {
        const T2 a = acc[o];
        acc[o] = mkc<T2>(a.x + 2.0 * fr, a.y + 2.0 * fi);
        Zo[o] = mkc<T2>(zn.x + dt * fr, zn.y + dt * fi);
      } else {
        const T2 a = acc[o];
        const double h = dt / 6.0;
        Zn[o] = mkc<T2>(zn.x + h * (a.x + fr), zn.y + h * (a.y + fi));
      }
    }
  }
}

void plain_gram_launch(const DevPtrs& p, const RunParams& rp, int max_nblk, const double2* zin, cudaStream_t s) {
  plain_gram<double2><<<dim3(max_nblk, rp.n_traj), PT, 0, s>>>(p.traj, zin, p.part, 0);
}
void plain_gram_launch(const DevPtrs& p, const RunParams& rp, int max_nblk, const float2* zin, cudaStream_t s) {
  plain_gram<float2><<<dim3(max_nblk, rp.n_traj), PT, 0, s>>>(p.traj, zin, p.part, 0);
}

template <typename T2>
void rhs_launch(const DevPtrs& p, const RunParams& rp, int max_N, const T2* zin, T2* zout, int stage, double t,
                cudaStream_t s) {
  const int rhs_blocks = (int)((long)max_N * LR_MAX_RANK / PT / 2 + 1);
  plain_rhs<T2><<<dim3(rhs_blocks, rp.n_traj), PT, 0, s>>>(p, rp, zin, zout, stage, t);
}
void plain_rhs_launch(const DevPtrs& p, const RunParams& rp, int max_N, const double2* zin, double2* zout, int stage,
                      double t, cudaStream_t s) {
  rhs_launch(p, rp, max_N, zin, zout, stage, t, s);
}
void plain_rhs_launch(const DevPtrs& p, const RunParams& rp, int max_N, const float2* zin, float2* zout, int stage,
                      double t, cudaStream_t s) {
  rhs_launch(p, rp, max_N, zin, zout, stage, t, s);
}

template <typename T2>
cudaError_t integrate_t(const DevPtrs& p, const RunParams& rp, int max_nblk, int max_N, long step0, long n_steps,
                        cudaStream_t s) {
  T2* Zn = reinterpret_cast<T2*>(p.Zn);
  T2* Za = reinterpret_cast<T2*>(p.Za);
  T2* Zb = reinterpret_cast<T2*>(p.Zb);
  const dim3 ggrid(max_nblk, rp.n_traj);
  const int rhs_blocks = (int)((long)max_N * LR_MAX_RANK / PT / 2 + 1);
  const dim3 rgrid(rhs_blocks < 1 ? 1 : rhs_blocks, rp.n_traj);
  for (long st = step0; st < step0 + n_steps; ++st) {
    const double tn = (double)st * rp.dt;
    const int record = (st % rp.pop_every) == 0;
    for (int stage = 0; stage < 4; ++stage) {
      const T2* zin = stage == 0 ? Zn : (stage == 2 ? Zb : Za);
      T2* zout = stage == 1 ? Zb : (stage == 3 ? nullptr : Za);
      const double ts = tn + (stage == 0 ? 0.0 : (stage == 3 ? rp.dt : 0.5 * rp.dt));
      plain_gram<T2><<<ggrid, PT, 0, s>>>(p.traj, zin, p.part, stage == 0 && record);
      plain_solve<<<rp.n_traj, PT, 0, s>>>(p, rp, st, stage, stage == 0 && record, 1);
      plain_rhs<T2><<<rgrid, PT, 0, s>>>(p, rp, zin, zout, stage, ts);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // observables of the final state
  const long se = step0 + n_steps;
  const int record = (se % rp.pop_every) == 0;
  plain_gram<T2><<<ggrid, PT, 0, s>>>(p.traj, Zn, p.part, record);
  plain_solve<<<rp.n_traj, PT, 0, s>>>(p, rp, se, 0, record, 0);
  return cudaGetLastError();
}

cudaError_t plain_integrate(const DevPtrs& p, const RunParams& rp, int max_nblk, int max_N, long step0,
                            long n_steps, cudaStream_t s, int fp32) {
  return fp32 ? integrate_t<float2>(p, rp, max_nblk, max_N, step0, n_steps, s)
              : integrate_t<double2>(p, rp, max_nblk, max_N, step0, n_steps, s);
}

}  // namespace lr
