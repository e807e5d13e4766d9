// Single-shot readout with seeded Gaussian measurement noise (Sec. S3.A): the
// Monte Carlo counterpart of the assignment error, from the recorded readout
// fields beta_g, beta_e of every candidate.
//
// One block per (candidate, state j, 256 shots). The block forms the bin
// coefficients a_b = conj(q_b) / sqrt(W_b) in shared memory and the separation
// D; every thread then draws one shot: N = sum_b Re(a_b xi_b) over the bins in
// order (FP64), xi_b = (n1 + i n2) / sqrt 2 by Box-Muller on two counter-based
// SplitMix64 uniforms, and counts the shot as misassigned when the matched
// filter's statistic +-D/2 + N lies on the wrong side of zero.
#include "lr_internal.cuh"

namespace lr {
namespace {

constexpr int ST = 256;                     // shots per block
constexpr int MAX_BINS = 2048;              // bins held in shared memory
constexpr unsigned long long GOLDEN = 0x9E3779B97F4A7C15ull;

// SplitMix64 (Steele, Lea & Flood 2014): output k of the stream of `seed`
__device__ __forceinline__ unsigned long long sm64(unsigned long long seed, unsigned long long k) {
  unsigned long long z = seed + (k + 1ull) * GOLDEN;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform_open0(unsigned long long seed, unsigned long long k) {
  return ((double)(sm64(seed, k) >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
}

struct ShotArgs {
  const TrajDev* traj;
  const double2* beta;   // [n_traj][ld]
  long ld;               // max_steps + 1
  long step;             // steps integrated (n)
  double dt, eta;
  long n_shots;
  int bin;               // steps per bin
  int n_bins;
  unsigned long long seed;
  unsigned long long* counts;   // [n_cand][2] misassigned shots of g and e
  double* snr;                  // [n_cand] binned SNR
};

__global__ void __launch_bounds__(ST) shots_kernel(ShotArgs a) {
  __shared__ double2 coef[MAX_BINS];
  __shared__ double red[ST / 32];
  __shared__ unsigned int nerr;
  const int c = blockIdx.x, j = blockIdx.y, tid = threadIdx.x;
  const double2* bg = a.beta + (size_t)(2 * c) * a.ld;
  const double2* be = a.beta + (size_t)(2 * c + 1) * a.ld;
  // bins: q_b and W_b (trapezoid weights over steps 0..n), a_b = conj(q_b) / sqrt(W_b)
  double dpart = 0.0;
  for (int b = tid; b < a.n_bins; b += ST) {
    const long k0 = (long)b * a.bin, k1 = k0 + a.bin <= a.step + 1 ? k0 + a.bin : a.step + 1;
    double qx = 0.0, qy = 0.0, W = 0.0;
    for (long k = k0; k < k1; ++k) {
      const double w = (k == 0 || k == a.step) ? 0.5 * a.dt : a.dt;
      qx += w * (be[k].x - bg[k].x);
      qy += w * (be[k].y - bg[k].y);
      W += w;
    }
    const double r = rsqrt(W);
    coef[b] = make_double2(qx * r, -qy * r);
    dpart += (qx * qx + qy * qy) / W;
  }
  if (tid == 0) nerr = 0u;
  // fixed-order block sum of |q_b|^2 / W_b
  for (int o = 16; o > 0; o >>= 1) dpart += __shfl_down_sync(0xffffffffu, dpart, o);
  if ((tid & 31) == 0) red[tid >> 5] = dpart;
  __syncthreads();
  double sum = 0.0;
  for (int w = 0; w < ST / 32; ++w) sum += red[w];
  const double kappa = a.traj[2 * c].kappa;
  const double D = sqrt(2.0 * a.eta * kappa) * sum;
  if (j == 0 && blockIdx.z == 0 && tid == 0) a.snr[c] = sqrt(2.0 * a.eta * kappa * sum);
  const long s = (long)blockIdx.z * ST + tid;
  if (s < a.n_shots) {
    const unsigned long long key = sm64(a.seed, (unsigned long long)(2 * c + j) * (unsigned long long)a.n_shots +
                                                    (unsigned long long)s);
    double N = 0.0;
    for (int b = 0; b < a.n_bins; ++b) {
      const double u1 = uniform_open0(key, 2ull * b), u2 = uniform_open0(key, 2ull * b + 1ull);
      const double r = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      const double2 q = coef[b];
      N += (q.x * (r * cs) - q.y * (r * sn)) * 0.70710678118654752440;
    }
    const bool wrong = j == 1 ? (0.5 * D + N <= 0.0) : (-0.5 * D + N > 0.0);
    if (wrong) atomicAdd(&nerr, 1u);
  }
  __syncthreads();
  if (tid == 0 && nerr) atomicAdd(a.counts + 2 * c + j, (unsigned long long)nerr);
}

// eps_shots = misassigned / (2 n_shots) + tau gamma / 2, eps_bin = erfc(SNR_b/2)/2 + tau gamma / 2
__global__ void shots_finish_kernel(const TrajDev* traj, const unsigned long long* counts, const double* snr, int n_cand,
                                    long n_shots, double tau, double* eps_shots, double* eps_bin) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cand) return;
  const double dec = 0.5 * tau * traj[2 * c].gamma;
  eps_shots[c] = (double)(counts[2 * c] + counts[2 * c + 1]) / (2.0 * (double)n_shots) + dec;
  eps_bin[c] = 0.5 * erfc(0.5 * snr[c]) + dec;
}

}  // namespace

int shots_max_bins() { return MAX_BINS; }

cudaError_t launch_shots(const DevPtrs& p, const RunParams& rp, long step, double eta, long n_shots, int bin,
                         unsigned long long seed, unsigned long long* counts, double* snr, double* eps_shots,
                         double* eps_bin, cudaStream_t s) {
  ShotArgs a{};
  a.traj = p.traj;
  a.beta = p.beta;
  a.ld = rp.max_steps + 1;
  a.step = step;
  a.dt = rp.dt;
  a.eta = eta;
  a.n_shots = n_shots;
  a.bin = bin;
  a.n_bins = (int)((step + 1 + bin - 1) / bin);
  a.seed = seed;
  a.counts = counts;
  a.snr = snr;
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * 2 * rp.n_cand, s);
  if (e != cudaSuccess) return e;
  const dim3 grid(rp.n_cand, 2, (unsigned)((n_shots + ST - 1) / ST));
  shots_kernel<<<grid, ST, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  shots_finish_kernel<<<(rp.n_cand + 127) / 128, 128, 0, s>>>(p.traj, counts, snr, rp.n_cand, n_shots,
                                                              (double)step * rp.dt, eps_shots, eps_bin);
  return cudaGetLastError();
}

}  // namespace lr
