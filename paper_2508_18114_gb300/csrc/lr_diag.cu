// Validity diagnostics (Sec. S1.B, Fig. S1): spectrum and purity of
// rho = Z Z^dag from the FP64 Gram matrices G = Z^dag Z recorded by the
// engines. rho and G share their nonzero eigenvalues, and tr(rho^2) = tr(G^2).
//
// One block per (trajectory, record). The complex Hermitian M x M matrix G
// is embedded as the real symmetric 2M x 2M matrix S = [[Re G, -Im G],
// [Im G, Re G]] (eigenvalues of G, each twice) and diagonalised by cyclic
// Jacobi rotations (Golub & Van Loan, Matrix Computations, Sec. 8.5): sweeps
// of 2M - 1 rounds, each round rotating the M disjoint index pairs of the
// round-robin ("circle") ordering in parallel, until the off-diagonal mass is
// below 1e-28 of the total (1e-14 relative in norm). Every reduction runs in a
// fixed order, so the output is deterministic.
#include "lr_internal.cuh"

namespace lr {
namespace {

constexpr int DT = 256;
constexpr int NMAX = 2 * LR_MAX_RANK;
constexpr int MAX_SWEEPS = 30;

__device__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < DT / 32; ++w) r += red[w];
    red[DT / 32] = r;
  }
  __syncthreads();
  const double r = red[DT / 32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(DT) diag_kernel(DevPtrs p, RunParams rp, long n_valid, double* purity, double* eig) {
  __shared__ double S[NMAX][NMAX + 1];
  __shared__ double rc[NMAX / 2], rs[NMAX / 2];
  __shared__ int rp_[NMAX / 2], rq_[NMAX / 2];
  __shared__ double red[DT / 32 + 1];
  __shared__ double ev[NMAX];
  const long b = blockIdx.x;
  const int tj = (int)(b / n_valid);
  const long rec = b - (long)tj * n_valid;
  const int M = p.traj[tj].M, n = 2 * M, sm = rp.snap_m, tid = threadIdx.x;
  const double2* G = p.gsnap + ((size_t)tj * rp.n_rec + rec) * sm * sm;

  double pur = 0.0, fro = 0.0;
  for (int e = tid; e < M * M; e += DT) {
    const int i = e / M, j = e - i * M;
    const double2 g = G[i * sm + j];
    S[i][j] = g.x;
    S[i + M][j + M] = g.x;
    S[i][j + M] = -g.y;
    S[i + M][j] = g.y;
    pur += g.x * g.x + g.y * g.y;
  }
  pur = block_sum_d(pur, red);   // tr(G^2) = sum |G_ij|^2 (G Hermitian)
  fro = 2.0 * pur;               // ||S||_F^2

  for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
    double off = 0.0;
    for (int e = tid; e < n * n; e += DT) {
      const int i = e / n, j = e - i * n;
      if (i != j) off += S[i][j] * S[i][j];
    }
    off = block_sum_d(off, red);
    if (!(off > 1e-28 * fro)) break;
    for (int round = 0; round < n - 1; ++round) {
      // pair k of this round: (n-1, round) for k = 0, else ((round+k), (round-k)) mod (n-1)
      if (tid < M) {
        const int k = tid;
        int pp, qq;
        if (k == 0) {
          pp = round;
          qq = n - 1;
        } else {
          pp = (round + k) % (n - 1);
          qq = (round - k + (n - 1)) % (n - 1);
        }
        if (pp > qq) {
          const int t = pp;
          pp = qq;
          qq = t;
        }
        const double apq = S[pp][qq];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double tau = (S[qq][qq] - S[pp][pp]) / (2.0 * apq);
          const double t = tau >= 0.0 ? 1.0 / (tau + hypot(1.0, tau)) : -1.0 / (-tau + hypot(1.0, tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        rp_[k] = pp;
        rq_[k] = qq;
        rc[k] = c;
        rs[k] = s;
      }
      __syncthreads();
      // rows: S <- J^T S
      for (int e = tid; e < M * n; e += DT) {
        const int k = e / n, col = e - k * n;
        const int pp = rp_[k], qq = rq_[k];
        const double c = rc[k], s = rs[k];
        const double a = S[pp][col], bb = S[qq][col];
        S[pp][col] = c * a - s * bb;
        S[qq][col] = s * a + c * bb;
      }
      __syncthreads();
      // columns: S <- S J
      for (int e = tid; e < M * n; e += DT) {
        const int k = e / n, row = e - k * n;
        const int pp = rp_[k], qq = rq_[k];
        const double c = rc[k], s = rs[k];
        const double a = S[row][pp], bb = S[row][qq];
        S[row][pp] = c * a - s * bb;
        S[row][qq] = s * a + c * bb;
      }
      __syncthreads();
    }
  }
  if (tid < n) ev[tid] = S[tid][tid];
  __syncthreads();
  if (tid == 0) {
    // descending insertion sort; eigenvalue k of G = mean of the equal pair 2k, 2k+1
    for (int i = 1; i < n; ++i) {
      const double v = ev[i];
      int j = i - 1;
      while (j >= 0 && ev[j] < v) {
        ev[j + 1] = ev[j];
        --j;
      }
      ev[j + 1] = v;
    }
    double* out = eig + ((size_t)tj * rp.n_rec + rec) * sm;
    for (int k = 0; k < sm; ++k) out[k] = k < M ? 0.5 * (ev[2 * k] + ev[2 * k + 1]) : 0.0;
    purity[(size_t)tj * rp.n_rec + rec] = pur;
  }
}

}  // namespace

cudaError_t launch_diagnostics(const DevPtrs& p, const RunParams& rp, long n_valid, double* purity, double* eig,
                               cudaStream_t s) {
  if (!p.gsnap || rp.snap_m < 1 || n_valid < 1) return cudaSuccess;
  const long blocks = (long)rp.n_traj * n_valid;
  diag_kernel<<<(unsigned)blocks, DT, 0, s>>>(p, rp, n_valid, purity, eig);
  return cudaGetLastError();
}

}  // namespace lr
