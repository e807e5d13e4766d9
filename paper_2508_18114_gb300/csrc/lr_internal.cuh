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
enum DevErr : unsigned { DEV_OK = 0, DEV_NOT_PD = 1, DEV_NONFINITE = 2, DEV_TIMEOUT = 3, DEV_CAPACITY = 4 };

__device__ __forceinline__ void set_error(unsigned* err, unsigned code) {
  atomicCAS(err, 0u, code);
}

// ------------------------------------------------------------------ complex

template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };

__host__ __device__ __forceinline__ double2 mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ float2 mkf(float r, float i) { return make_float2(r, i); }

// Real type of a complex storage type, and a constructor generic over both.
template <typename T2> struct real_of;
template <> struct real_of<double2> { using type = double; };
template <> struct real_of<float2> { using type = float; };
template <typename T2>
__host__ __device__ __forceinline__ T2 mkc(typename real_of<T2>::type r, typename real_of<T2>::type i) {
  T2 v;
  v.x = r;
  v.y = i;
  return v;
}

// ------------------------------------------------------------------ pulse

// Logistic step f(t, t0, s) of Sec. S2.C.
__device__ __forceinline__ double logistic(double t, double t0, double s) {
  return 1.0 / (1.0 + exp(-(t - t0) / s));
}

// Envelope Omega(t) of Sec. S2.C.
__device__ __forceinline__ double pulse_envelope(const PulseDev& P, double tau, double t) {
  if (P.kind == 0) {
    const double s = P.p[2] / 5.0, t0 = 6.0 * s;
    return P.p[0] * logistic(t, t0, s) * (1.0 - logistic(t, tau - t0, s));
  }
  const double sr = P.p[3] / 5.0, sf = P.p[4] / 5.0, sm = P.p[5] / 5.0;
  return P.p[0] * logistic(t, 6.0 * sr, sr) + (P.p[1] - P.p[0]) * logistic(t, P.p[2], sm) -
         P.p[1] * logistic(t, tau - 6.0 * sf, sf);
}
__device__ __forceinline__ double pulse_drive_frequency(const PulseDev& P) { return P.kind == 0 ? P.p[1] : P.p[6]; }
__device__ __forceinline__ double pulse_phase(const PulseDev& P) { return P.kind == 0 ? P.p[3] : P.p[7]; }

// Omega(t) cos(w_d t + phi): the coefficient of (r + r^dag) in H(t).
__device__ __forceinline__ double pulse_coefficient(const PulseDev& P, double tau, double t) {
  const double env = pulse_envelope(P, tau, t);
  return env * cos(pulse_drive_frequency(P) * t + pulse_phase(P));
}

// Drive in the frame rotating at w_d with the rotating-wave approximation
// (the RWA Hamiltonian of Sec. S2): (Omega(t)/2)(e^{i phi} r + e^{-i phi} r^dag).
// Returns the weight of the r term, w = (Omega/2) e^{i phi}; the r^dag term
// carries conj(w).
__device__ __forceinline__ double2 pulse_rwa_drive(const PulseDev& P, double tau, double t) {
  const double h = 0.5 * pulse_envelope(P, tau, t);
  double sn, cs;
  sincos(pulse_phase(P), &sn, &cs);
  return make_double2(h * cs, h * sn);
}

// d c(t) / d theta_i for the pulse parameters (kind 0: 4 entries, kind 1: 8),
// written into dc[8]; returns c(t). With f = logistic(u), df/du = f (1 - f):
//  flat-top   u1 = 5t/t_r - 6, u2 = 5(t - tau)/t_r + 6, Omega = A f1 (1 - f2);
//  two-segment u_r = 5t/t_rise - 6, u_m = 5(t - t_sw)/t_sm,
//              u_f = 5(t - tau)/t_fall + 6,
//              Omega = A1 f_r + (A2 - A1) f_m - A2 f_f;
//  c = Omega cos(w_d t + phi).
__device__ __forceinline__ double pulse_coefficient_grad(const PulseDev& P, double tau, double t, double* dc) {
  double env, wd, phi;
  double denv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int iw, ip;
  if (P.kind == 0) {
    const double A = P.p[0], tr = P.p[2];
    const double s = tr / 5.0, t0 = 6.0 * s;
    const double f1 = logistic(t, t0, s), f2 = logistic(t, tau - t0, s);
    env = A * f1 * (1.0 - f2);
    const double du1 = -5.0 * t / (tr * tr), du2 = -5.0 * (t - tau) / (tr * tr);
    denv[0] = f1 * (1.0 - f2);
    denv[2] = A * (f1 * (1.0 - f1) * du1 * (1.0 - f2) - f1 * f2 * (1.0 - f2) * du2);
    iw = 1;
    ip = 3;
  } else {
    const double A1 = P.p[0], A2 = P.p[1], tsw = P.p[2], trs = P.p[3], tfl = P.p[4], tsm = P.p[5];
    const double fr = logistic(t, 1.2 * trs, 0.2 * trs), fm = logistic(t, tsw, 0.2 * tsm),
                 ff = logistic(t, tau - 1.2 * tfl, 0.2 * tfl);
    env = A1 * fr + (A2 - A1) * fm - A2 * ff;
    denv[0] = fr - fm;
    denv[1] = fm - ff;
    denv[2] = (A2 - A1) * fm * (1.0 - fm) * (-5.0 / tsm);
    denv[3] = A1 * fr * (1.0 - fr) * (-5.0 * t / (trs * trs));
    denv[4] = -A2 * ff * (1.0 - ff) * (-5.0 * (t - tau) / (tfl * tfl));
    denv[5] = (A2 - A1) * fm * (1.0 - fm) * (-5.0 * (t - tsw) / (tsm * tsm));
    iw = 6;
    ip = 7;
  }
  wd = P.p[iw];
  phi = P.p[ip];
  double sn, cs;
  sincos(wd * t + phi, &sn, &cs);
  for (int i = 0; i < 8; ++i) dc[i] = denv[i] * cs;
  dc[iw] = -env * t * sn;
  dc[ip] = -env * sn;
  return env * cs;
}

// Doubles per row block of the plain engine's partial sums: G, Z^dag r Z,
// Z^dag b Z (M x M complex each) then level populations and photons.
__host__ __device__ inline size_t plain_pstride(int M) { return (size_t)6 * M * M + LR_MAX_NT + 2; }

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
// wfr: frame frequency (0 in the lab frame, w_d in the rotating frame, where
// every mode frequency becomes a detuning w - w_d).
__device__ __forceinline__ void heff_diag(const TrajDev& d, const RowIdx& r, double wfr, double& re, double& im) {
  const double it = r.it;
  re = (d.wq - wfr) * it + 0.5 * d.alpha * it * (it - 1.0) + (d.wr - wfr) * r.ir +
       (d.n_modes == 3 ? (d.wf - wfr) * r.iff : 0.0);
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
  double* ion;     // [n_cand] ionization penalty T(tau)
  double* loss;    // [n_cand] log10(eps_a + T)
  void* scratch;   // engine scratch
  long long scratch_bytes;
  double2* gsnap;  // [n_traj][n_rec][snap_m][snap_m] Gram matrices at record steps, or null
  long long* dstep;  // RK4 steps taken in the pulse run (device copy), or null
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
  int snap_m;   // leading dimension of the Gram snapshots (max M), 0 when not recorded
  int frame;    // 0: lab frame; 1: frame rotating at each candidate's w_d, rotating-wave approximation
};

// lr_common.cu
cudaError_t launch_initial_state(const DevPtrs& p, const RunParams& rp, int max_N, int prec_fp32,
                                 uint64_t seed, double eps, cudaStream_t s);
// Rank growth: dst's states = src's columns plus orthonormal padding columns of
// weight eps, one block per trajectory (both contexts hold the same trajectories).
cudaError_t launch_grow(const DevPtrs& dst, const DevPtrs& src, int n_traj, int prec_fp32, uint64_t seed, double eps,
                        cudaStream_t s);
// eps_a, T(tau) and Lambda at step *p.dstep + n_added (the integrate that
// precedes it in the stream took n_added steps), then *p.dstep += n_added.
cudaError_t launch_eps_a(const DevPtrs& p, const RunParams& rp, long n_added, cudaStream_t s);
// seeded single-shot readout (lr_shots.cu)
int shots_max_bins();
cudaError_t launch_shots(const DevPtrs& p, const RunParams& rp, long step, double eta, long n_shots, int bin,
                         unsigned long long seed, unsigned long long* counts, double* snr, double* eps_shots,
                         double* eps_bin, cudaStream_t s);
// Elementwise complex128 <-> complex64 conversion of n elements.
cudaError_t launch_convert(const void* src, void* dst, long long n, int to_fp32, cudaStream_t s);

// lr_diag.cu: eigenvalues and purity of the recorded Gram matrices, records
// [0, n_valid) of every trajectory
cudaError_t launch_diagnostics(const DevPtrs& p, const RunParams& rp, long n_valid, double* purity, double* eig,
                               cudaStream_t s);

// lr_plain.cu
int plain_rows_per_block();
size_t plain_partial_doubles(int M);
// The plain engine on complex128 state (the reference GPU path), or on
// complex64 state (fp32 = 1: the adjoint's FP32-bulk recomputation; the Gram
// matrix is summed from exact products in double-word FP32, Cholesky and solves
// in FP64, the rest in FP32).
cudaError_t plain_integrate(const DevPtrs& p, const RunParams& rp, int max_nblk, int max_N, long step0,
                            long n_steps, cudaStream_t s, int fp32 = 0);
// single kernels of the plain engine (used by the adjoint's recomputation)
void plain_gram_launch(const DevPtrs& p, const RunParams& rp, int max_nblk, const double2* zin, cudaStream_t s);
void plain_gram_launch(const DevPtrs& p, const RunParams& rp, int max_nblk, const float2* zin, cudaStream_t s);
void plain_rhs_launch(const DevPtrs& p, const RunParams& rp, int max_N, const double2* zin, double2* zout, int stage,
                      double t, cudaStream_t s);
void plain_rhs_launch(const DevPtrs& p, const RunParams& rp, int max_N, const float2* zin, float2* zout, int stage,
                      double t, cudaStream_t s);

// lr_adjoint.cu
struct BwdLayout {
  size_t ck, seg, cur, za, zb, acc, U, Ub, lam, lamn, X, part, Xs, Gi, EP, Xs32, EP32, bpart, beta, pops, nphot,
      trace, gcoef, deps, thbar, total;
  long n_seg, K;
  int fp32;   // 1: FP32-bulk adjoint (complex64 states and cotangents)
};
BwdLayout bwd_layout(long long tot, int n_traj, int n_cand, int nt_max, size_t part_doubles, long S, int K, int fp32);
cudaError_t backward_run(const DevPtrs& main, const RunParams& rp, char* ws, const BwdLayout& L, long long tot,
                         int max_nblk, int max_N, long S, const void* z0, int z0_fp32, const double* deps_host,
                         double* dtheta_host, cudaStream_t s);

}  // namespace lr
