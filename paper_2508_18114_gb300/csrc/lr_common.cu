// Kernels shared by the engines: fixed-rank initial state (Sec. S1.A),
// assignment-error epilogue (Sec. S3.A) and state precision conversion.
#include "lr_internal.cuh"

namespace lr {

constexpr int IT = 512;   // threads of the initial-state kernel
constexpr int ET = 256;   // threads of the epilogue kernel
constexpr unsigned long long GOLDEN = 0x9E3779B97F4A7C15ull;

// SplitMix64 (Steele, Lea & Flood 2014): k-th output for a seed.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long k) {
  return mix64(seed + (k + 1ull) * GOLDEN);
}
__device__ __forceinline__ double uniform_open0(unsigned long long seed, unsigned long long k) {
  return ((double)(splitmix64(seed, k) >> 11) + 1.0) * 0x1.0p-53;
}

// Fixed-order block reduction (deterministic for a fixed block size).
template <int NT>
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < NT / 32; ++w) r += sh[w];
    sh[32] = r;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

// One block per trajectory: Gaussian padding columns, modified Gram-Schmidt
// (two passes) against psi and each other, weights 1-(M-1)eps and eps.
// Works in FP64 in `W` (layout of the state), writes the state as T2.
template <typename T2>
__global__ void __launch_bounds__(IT) initial_state_kernel(const TrajDev* __restrict__ traj, double2* __restrict__ Wbase,
                                                           T2* __restrict__ Zbase, unsigned long long seed, double eps) {
  __shared__ double sh[33];
  const int tj = blockIdx.x;
  const TrajDev d = traj[tj];
  const int N = d.N, M = d.M, ld = d.ld;
  double2* W = Wbase + d.z_off;
  T2* Z = Zbase + d.z_off;
  const int psi = d.level0 * d.Nr * d.Nf;
  const unsigned long long ts = splitmix64(seed, (unsigned long long)tj);
  for (int n = threadIdx.x; n < N; n += IT) {
    W[(size_t)n * ld] = mk(n == psi ? 1.0 : 0.0, 0.0);
    for (int j = 1; j < M; ++j) {
      const unsigned long long pidx = (unsigned long long)(j - 1) * N + n;
      const double u1 = uniform_open0(ts, 2ull * pidx), u2 = uniform_open0(ts, 2ull * pidx + 1ull);
      const double r = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      W[(size_t)n * ld + j] = mk(r * cs, r * sn);
    }
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 1; j < M; ++j) {
      for (int i = 0; i < j; ++i) {
        double re = 0.0, im = 0.0;
        for (int n = threadIdx.x; n < N; n += IT) {
          const double2 a = W[(size_t)n * ld + i], b = W[(size_t)n * ld + j];   // conj(a) b
          re += a.x * b.x + a.y * b.y;
          im += a.x * b.y - a.y * b.x;
        }
        re = block_sum<IT>(re, sh);
        im = block_sum<IT>(im, sh);
        for (int n = threadIdx.x; n < N; n += IT) {
          const double2 a = W[(size_t)n * ld + i], b = W[(size_t)n * ld + j];
          W[(size_t)n * ld + j] = mk(b.x - (re * a.x - im * a.y), b.y - (re * a.y + im * a.x));
        }
        __syncthreads();
      }
      double nn = 0.0;
      for (int n = threadIdx.x; n < N; n += IT) {
        const double2 b = W[(size_t)n * ld + j];
        nn += b.x * b.x + b.y * b.y;
      }
      nn = block_sum<IT>(nn, sh);
      const double inv = 1.0 / sqrt(nn);
      for (int n = threadIdx.x; n < N; n += IT) {
        const double2 b = W[(size_t)n * ld + j];
        W[(size_t)n * ld + j] = mk(b.x * inv, b.y * inv);
      }
      __syncthreads();
    }
  }
  const double w0 = sqrt(1.0 - (M - 1) * eps), we = sqrt(eps);
  for (int n = threadIdx.x; n < N; n += IT) {
    for (int j = 0; j < ld; ++j) {
      double2 v = mk(0.0, 0.0);
      if (j < M) {
        const double2 q = W[(size_t)n * ld + j];
        const double s = j == 0 ? w0 : we;
        v = mk(s * q.x, s * q.y);
      }
      if constexpr (sizeof(T2) == sizeof(double2)) {
        Z[(size_t)n * ld + j] = v;
      } else {
        Z[(size_t)n * ld + j] = make_float2((float)v.x, (float)v.y);
      }
    }
  }
}

// Rank growth (adaptive rank): one block per trajectory. The source state's
// columns are kept; columns M_src .. M_dst-1 are sqrt(eps) q_j with q_j the
// normalised component of a complex Gaussian vector xi_j (same generator as the
// initial state, pair index (j - M_src) N + n) orthogonal to span(Z_src) and to
// q_{M_src} .. q_{j-1}. The projection onto span(Z_src) is Z G^-1 Z^dag with
// G = Z^dag Z (Cholesky, FP64), applied twice (reorthogonalisation).
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }

template <typename T2>
__global__ void __launch_bounds__(IT) grow_kernel(const TrajDev* __restrict__ dtraj, const TrajDev* __restrict__ straj,
                                                  const T2* __restrict__ Zsrc, double2* __restrict__ Wbase,
                                                  T2* __restrict__ Zdst, unsigned long long seed, double eps,
                                                  unsigned* err) {
  __shared__ double sh[33];
  __shared__ double2 L[LR_MAX_RANK][LR_MAX_RANK + 1];
  __shared__ double2 y[LR_MAX_RANK];
  __shared__ int bad;
  const int tj = blockIdx.x;
  const TrajDev d = dtraj[tj], sr = straj[tj];
  const int N = d.N, Ms = sr.M, Md = d.M, lds = sr.ld, ldd = d.ld;
  double2* W = Wbase + d.z_off;
  const T2* Zs = Zsrc + sr.z_off;
  T2* Z = Zdst + d.z_off;
  const unsigned long long ts = splitmix64(seed, (unsigned long long)tj);
  if (threadIdx.x == 0) bad = 0;
  for (int n = threadIdx.x; n < N; n += IT) {
    for (int j = 0; j < Ms; ++j) W[(size_t)n * ldd + j] = to_d2(Zs[(size_t)n * lds + j]);
    for (int j = Ms; j < Md; ++j) {
      const unsigned long long pidx = (unsigned long long)(j - Ms) * N + n;
      const double u1 = uniform_open0(ts, 2ull * pidx), u2 = uniform_open0(ts, 2ull * pidx + 1ull);
      const double r = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      W[(size_t)n * ldd + j] = mk(r * cs, r * sn);
    }
  }
  __syncthreads();
  // inner product <W_i, W_j> = sum_n conj(W_ni) W_nj (fixed-order block sums)
  auto dot = [&](int i, int j) {
    double re = 0.0, im = 0.0;
    for (int n = threadIdx.x; n < N; n += IT) {
      const double2 a = W[(size_t)n * ldd + i], b = W[(size_t)n * ldd + j];
      re += a.x * b.x + a.y * b.y;
      im += a.x * b.y - a.y * b.x;
    }
    re = block_sum<IT>(re, sh);
    im = block_sum<IT>(im, sh);
    return mk(re, im);
  };
  // G = Z^dag Z, lower triangle: G_ij = <W_i, W_j> for i >= j
  for (int i = 0; i < Ms; ++i)
    for (int j = 0; j <= i; ++j) {
      const double2 g = dot(i, j);
      if (threadIdx.x == 0) L[i][j] = g;
    }
  __syncthreads();
  if (threadIdx.x == 0) {   // Cholesky G = L L^dag (serial, M <= 32)
    for (int k = 0; k < Ms && !bad; ++k) {
      double piv = L[k][k].x;
      for (int q = 0; q < k; ++q) piv -= L[k][q].x * L[k][q].x + L[k][q].y * L[k][q].y;
      if (!(piv > 0.0)) {
        bad = 1;
        break;
      }
      const double lkk = sqrt(piv);
      L[k][k] = mk(lkk, 0.0);
      for (int i = k + 1; i < Ms; ++i) {
        double re = L[i][k].x, im = L[i][k].y;   // G_ik - sum_q L_iq conj(L_kq)
        for (int q = 0; q < k; ++q) {
          re -= L[i][q].x * L[k][q].x + L[i][q].y * L[k][q].y;
          im -= L[i][q].y * L[k][q].x - L[i][q].x * L[k][q].y;
        }
        L[i][k] = mk(re / lkk, im / lkk);
      }
    }
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) set_error(err, DEV_NOT_PD);
    return;
  }
  for (int j = Ms; j < Md; ++j) {
    for (int pass = 0; pass < 2; ++pass) {
      // remove the span(Z) component: c = Z^dag w, G y = c, w -= Z y
      for (int i = 0; i < Ms; ++i) {
        const double2 c = dot(i, j);
        if (threadIdx.x == 0) y[i] = c;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int i = 0; i < Ms; ++i) {   // L u = c
          double re = y[i].x, im = y[i].y;
          for (int q = 0; q < i; ++q) {
            re -= L[i][q].x * y[q].x - L[i][q].y * y[q].y;
            im -= L[i][q].x * y[q].y + L[i][q].y * y[q].x;
          }
          y[i] = mk(re / L[i][i].x, im / L[i][i].x);
        }
        for (int i = Ms - 1; i >= 0; --i) {   // L^dag y = u
          double re = y[i].x, im = y[i].y;
          for (int q = i + 1; q < Ms; ++q) {
            re -= L[q][i].x * y[q].x + L[q][i].y * y[q].y;
            im -= L[q][i].x * y[q].y - L[q][i].y * y[q].x;
          }
          y[i] = mk(re / L[i][i].x, im / L[i][i].x);
        }
      }
      __syncthreads();
      for (int n = threadIdx.x; n < N; n += IT) {
        double2 w = W[(size_t)n * ldd + j];
        for (int i = 0; i < Ms; ++i) {
          const double2 a = W[(size_t)n * ldd + i], c = y[i];
          w = mk(w.x - (a.x * c.x - a.y * c.y), w.y - (a.x * c.y + a.y * c.x));
        }
        W[(size_t)n * ldd + j] = w;
      }
      __syncthreads();
      // and the components along the new orthonormal columns so far
      for (int k = Ms; k < j; ++k) {
        const double2 r = dot(k, j);
        for (int n = threadIdx.x; n < N; n += IT) {
          const double2 a = W[(size_t)n * ldd + k], b = W[(size_t)n * ldd + j];
          W[(size_t)n * ldd + j] = mk(b.x - (r.x * a.x - r.y * a.y), b.y - (r.x * a.y + r.y * a.x));
        }
        __syncthreads();
      }
    }
    const double nn = dot(j, j).x;
    const double inv = 1.0 / sqrt(nn);
    for (int n = threadIdx.x; n < N; n += IT) {
      const double2 b = W[(size_t)n * ldd + j];
      W[(size_t)n * ldd + j] = mk(b.x * inv, b.y * inv);
    }
    __syncthreads();
  }
  const double we = sqrt(eps);
  for (int n = threadIdx.x; n < N; n += IT)
    for (int j = 0; j < ldd; ++j) {
      T2 v;
      if (j < Ms) {
        v = Zs[(size_t)n * lds + j];   // the kept columns, unchanged
      } else if (j < Md) {
        const double2 q = W[(size_t)n * ldd + j];
        v.x = q.x * we;
        v.y = q.y * we;
      } else {
        v.x = 0;
        v.y = 0;
      }
      Z[(size_t)n * ldd + j] = v;
    }
}

cudaError_t launch_grow(const DevPtrs& dst, const DevPtrs& src, int n_traj, int prec_fp32, uint64_t seed, double eps,
                        cudaStream_t s) {
  double2* W = reinterpret_cast<double2*>(dst.Za);
  if (prec_fp32)
    grow_kernel<float2><<<n_traj, IT, 0, s>>>(dst.traj, src.traj, reinterpret_cast<const float2*>(src.Zn), W,
                                              reinterpret_cast<float2*>(dst.Zn), seed, eps, dst.err);
  else
    grow_kernel<double2><<<n_traj, IT, 0, s>>>(dst.traj, src.traj, reinterpret_cast<const double2*>(src.Zn), W,
                                               reinterpret_cast<double2*>(dst.Zn), seed, eps, dst.err);
  return cudaGetLastError();
}

cudaError_t launch_initial_state(const DevPtrs& p, const RunParams& rp, int /*max_N*/, int prec_fp32,
                                 uint64_t seed, double eps, cudaStream_t s) {
  double2* W = reinterpret_cast<double2*>(p.Za);
  if (prec_fp32)
    initial_state_kernel<float2><<<rp.n_traj, IT, 0, s>>>(p.traj, W, reinterpret_cast<float2*>(p.Zn), seed, eps);
  else
    initial_state_kernel<double2><<<rp.n_traj, IT, 0, s>>>(p.traj, W, reinterpret_cast<double2*>(p.Zn), seed, eps);
  return cudaGetLastError();
}

// One block per candidate: trapezoid of |beta_e - beta_g|^2 over the step grid,
// SNR = sqrt(2 eta kappa S), eps_a = erfc(SNR/2)/2 + tau gamma/2.
__global__ void __launch_bounds__(ET) eps_a_kernel(DevPtrs p, RunParams rp, long n_added) {
  __shared__ double sh[33];
  const int c = blockIdx.x;
  const long step = (long)*p.dstep + n_added;
  if (step < 0 || step > rp.max_steps) {   // the integrate before it refused to run past capacity
    if (c == 0 && threadIdx.x == 0) set_error(p.err, DEV_CAPACITY);
    return;
  }
  const TrajDev d = p.traj[2 * c];
  const double2* bg = p.beta + (size_t)(2 * c) * (rp.max_steps + 1);
  const double2* be = p.beta + (size_t)(2 * c + 1) * (rp.max_steps + 1);
  double acc = 0.0;
  for (long i = threadIdx.x; i <= step; i += ET) {
    const double dx = be[i].x - bg[i].x, dy = be[i].y - bg[i].y;
    const double w = (i == 0 || i == step) ? 0.5 : 1.0;
    acc += w * (dx * dx + dy * dy);
  }
  acc = block_sum<ET>(acc, sh);
  // ionization penalty (Sec. S3.B): populations of transmon levels k >= 2 of
  // both trajectories, trapezoid over the recorded grid up to the last record
  const long last = step / rp.pop_every;
  const int Nt = d.Nt;
  double ion = 0.0;
  for (long r = threadIdx.x; r <= last; r += ET) {
    const double w = (r == 0 || r == last) ? 0.5 : 1.0;
    double sum = 0.0;
    for (int tj = 2 * c; tj <= 2 * c + 1; ++tj)
      for (int k = 2; k < Nt; ++k) sum += p.pops[((size_t)tj * rp.n_rec + r) * rp.nt_max + k];
    ion += w * sum;
  }
  ion = block_sum<ET>(ion, sh);
  if (threadIdx.x == 0) {
    const double S = step > 0 ? rp.dt * acc : 0.0;
    const double snr = sqrt(2.0 * rp.eta * d.kappa * S);
    const double tau = (double)step * rp.dt;
    const double e = 0.5 * erfc(0.5 * snr) + 0.5 * tau * d.gamma;
    p.eps_a[c] = e;
    const double T = (step > 0 && last > 0) ? ion * rp.pop_every * rp.dt / tau : 0.0;
    p.ion[c] = T;
    p.loss[c] = log10(e + T);
    if (!isfinite(e)) set_error(p.err, DEV_NONFINITE);
  }
}

// Advance the device step counter once every block of eps_a_kernel has read it
// (a kernel of its own, ordered after it in the stream); a run past capacity
// leaves the counter where it was.
__global__ void advance_step_kernel(long long* dstep, long n_added, long max_steps) {
  const long long s = *dstep + n_added;
  if (s >= 0 && s <= max_steps) *dstep = s;
}

cudaError_t launch_eps_a(const DevPtrs& p, const RunParams& rp, long n_added, cudaStream_t s) {
  eps_a_kernel<<<rp.n_cand, ET, 0, s>>>(p, rp, n_added);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  advance_step_kernel<<<1, 1, 0, s>>>(p.dstep, n_added, rp.max_steps);
  return cudaGetLastError();
}

__global__ void convert_kernel(const void* __restrict__ src, void* __restrict__ dst, long long n, int to_fp32) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (to_fp32) {
      const double2 v = reinterpret_cast<const double2*>(src)[i];
      reinterpret_cast<float2*>(dst)[i] = make_float2((float)v.x, (float)v.y);
    } else {
      const float2 v = reinterpret_cast<const float2*>(src)[i];
      reinterpret_cast<double2*>(dst)[i] = make_double2(v.x, v.y);
    }
  }
}

cudaError_t launch_convert(const void* src, void* dst, long long n, int to_fp32, cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  convert_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, s>>>(src, dst, n, to_fp32);
  return cudaGetLastError();
}

}  // namespace lr
