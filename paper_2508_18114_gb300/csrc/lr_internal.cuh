// Internal declarations shared by the library's translation units.
// Device data layout, small complex helpers, model stencil and pulse.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lr.h"

namespace lr {

// ------------------------------------------------------------------ tables

// One trajectory as the kernels see it. Rows of Z are basis states with
// flat index n = (i_t * N_r + i_r) * N_f + i_f (N_f = 1 with two modes);
// Z is row-major [n][m] with row stride `ld` (complex elements).
struct TrajDev {
  int N, M, ld;
  int Nt, Nr, Nf;
  int n_modes;
  int cand;         // candidate index (pulse)
  int level0;       // initial transmon level (0 = g, 1 = e)
  int nblk;         // plain engine: row blocks of the Gram kernel
  long long z_off;  // offset of this trajectory in the state arrays (complex elements)
  long long p_off;  // plain engine: offset in the partial-sum array (doubles)
  double wq, alpha, wr, wf, g, J, kappa, gamma;
};

struct PulseDev {
  int kind;
  double p[8];
};

// Device error word values (first error wins).
enum DevErr : unsigned { DEV_OK = 0, DEV_NOT_PD = 1, DEV_NONFINITE = 2, DEV_TIMEOUT = 3 };

__device__ __forceinline__ void set_error(unsigned* err, unsigned code) {
  atomicCAS(err, 0u, code);
}

// ------------------------------------------------------------------ complex

template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };

__host__ __device__ __forceinline__ double2 mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ float2 mkf(float r, float i) { return make_float2(r, i); }

// ------------------------------------------------------------------ pulse

// Logistic step f(t, t0, s) of Sec. S2.C.
__device__ __forceinline__ double logistic(double t, double t0, double s) {
  return 1.0 / (1.0 + exp(-(t - t0) / s));
}

// Omega(t) cos(w_d t + phi): the coefficient of (r + r^dag) in H(t).
__device__ __forceinline__ double pulse_coefficient(const PulseDev& P, double tau, double t) {
  double env, wd, phi;
  if (P.kind == 0) {
    const double s = P.p[2] / 5.0, t0 = 6.0 * s;
    env = P.p[0] * logistic(t, t0, s) * (1.0 - logistic(t, tau - t0, s));
    wd = P.p[1];
    phi = P.p[3];
  } else {
    const double sr = P.p[3] / 5.0, sf = P.p[4] / 5.0, sm = P.p[5] / 5.0;
    env = P.p[0] * logistic(t, 6.0 * sr, sr) + (P.p[1] - P.p[0]) * logistic(t, P.p[2], sm) -
          P.p[1] * logistic(t, tau - 6.0 * sf, sf);
    wd = P.p[6];
    phi = P.p[7];
  }
  return env * cos(wd * t + phi);
}

// ------------------------------------------------------------------ stencil

// Mode indices of a row.
struct RowIdx {
  int it, ir, iff;
};

__device__ __forceinline__ RowIdx row_index(const TrajDev& d, int n) {
  RowIdx r;
  const int st = d.Nr * d.Nf;
  r.it = n / st;
  const int rem = n - r.it * st;
  r.ir = rem / d.Nf;
  r.iff = rem - r.ir * d.Nf;
  return r;
}

// Occupation of the readout (last) mode.
__device__ __forceinline__ int readout_index(const TrajDev& d, const RowIdx& r) {
  return d.n_modes == 3 ? r.iff : r.ir;
}
__device__ __forceinline__ int readout_dim(const TrajDev& d) {
  return d.n_modes == 3 ? d.Nf : d.Nr;
}

// Diagonal of H_eff = H - (i/2) sum_k L_k^dag L_k (real and imaginary part).
__device__ __forceinline__ void heff_diag(const TrajDev& d, const RowIdx& r, double& re, double& im) {
  const double it = r.it;
  re = d.wq * it + 0.5 * d.alpha * it * (it - 1.0) + d.wr * r.ir + (d.n_modes == 3 ? d.wf * r.iff : 0.0);
  im = -0.5 * (d.kappa * readout_index(d, r) + d.gamma * it);
}

// ------------------------------------------------------------------ launches

struct Layout;  // defined in lr_api.cu

// Workspace pointers handed to the kernels.
struct DevPtrs {
  const TrajDev* traj;
  const PulseDev* pulse;
  unsigned* err;
  void* Zn;        // state Z_n
  void* Za;        // stage buffer A
  void* Zb;        // stage buffer B
  void* acc;       // RK4 accumulator
  double2* X;      // [n_traj][2][LR_MAX_RANK^2] solved projections (plain)
  double* part;    // plain partial sums
  double2* beta;   // [n_traj][max_steps+1]
  double* pops;    // [n_traj][n_rec][nt_max]
  double* nphot;   // [n_traj][n_rec]
  double* trace;   // [n_traj][n_rec]
  double* eps_a;   // [n_cand]
  void* scratch;   // engine scratch
  long long scratch_bytes;
};

struct RunParams {
  int n_traj, n_cand;
  int nt_max;
  long max_steps;
  long n_rec;
  int pop_every;
  double tau;   // pulse duration (falling edge placement)
  double dt;
  double eta;
};

// lr_common.cu
cudaError_t launch_initial_state(const DevPtrs& p, const RunParams& rp, int max_N, int prec_fp32,
                                 uint64_t seed, double eps, cudaStream_t s);
cudaError_t launch_eps_a(const DevPtrs& p, const RunParams& rp, long step, cudaStream_t s);
// Elementwise complex128 <-> complex64 conversion of n elements.
cudaError_t launch_convert(const void* src, void* dst, long long n, int to_fp32, cudaStream_t s);

// lr_plain.cu
int plain_rows_per_block();
size_t plain_partial_doubles(int M);
cudaError_t plain_integrate(const DevPtrs& p, const RunParams& rp, int max_nblk, int max_N, long step0,
                            long n_steps, cudaStream_t s);

}  // namespace lr
