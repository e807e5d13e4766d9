// Full master equation on the device (FP64): the N x N density matrix under
// Eq. 2 / Eq. S4 for an operator set given as CSR rows with time channels
// (lr_sparse_model: A = -i H_eff, the jump operators L_k and the readout r),
// integrated with the classical RK4 scheme of the low-rank engines. It is the
// reference that the low-rank run of the same model is compared with (Fig. 2
// of the paper) and timed against (Table 1).
//
// With A = -i H_eff = -i H - 1/2 sum_k L_k^dag L_k and rho Hermitian,
//     d rho / dt = A rho + (A rho)^dag + sum_k L_k rho L_k^dag,
// and L_k rho L_k^dag = L_k (L_k rho)^dag. One RK4 stage is:
//   fm_opvals   the operator values at the stage time (val * chi[channel]);
//   fm_apply    B = A rho and Y_k = L_k rho, one thread per element (i, j),
//               gathering rows rho[col][j] over the CSR entries of row i;
//   fm_transp   Bt = B^dag, Yt_k = Y_k^dag (32 x 32 shared-memory tiles);
//   fm_update   F = B + Bt + sum_k L_k Yt_k (gathers of rows of Yt_k), and the
//               RK4 stage update of the accumulator and the next stage input,
//               from the upper triangle, mirrored: rho stays exactly Hermitian.
// Observables at the start of every step (fm_obs, one block, fixed order):
// beta = tr(rho r), and at recording steps the level populations, the photon
// number tr(r rho r^dag) and tr rho.
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "lr_internal.cuh"

namespace lr {
namespace {

constexpr int FT = 256;
constexpr int NCHF = 10;

struct FmDev {
  const int* rowptr;   // [(K + 2) (N + 1)]
  const int* col;
  const double2* val;
  const unsigned char* chan;
  const int* level;
  const PulseDev* pulse;
  unsigned* err;
  double2* opv;       // [nnz] operator values at the current stage time
  double2* rho;       // state rho_n [N][N]
  double2* rs;        // stage input
  double2* acc;       // RK4 accumulator
  double2* B;         // A rs
  double2* Bt;        // B^dag
  double2* Y;         // [K][N][N]  L_k rs
  double2* Yt;        // [K][N][N]  Y_k^dag
  double2* beta;      // [max_steps + 1]
  double *pops, *nphot, *trace;
};

struct FmParams {
  int N, K, n_levels;
  long long nnz;
  double wd, tau;
  long max_steps, n_rec;
  int pop_every;
};

__device__ __forceinline__ double2 cmulf(double2 a, double2 b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

__global__ void __launch_bounds__(FT) fm_opvals(FmDev d, FmParams p, double t) {
  __shared__ double2 chi[NCHF];
  if (threadIdx.x < NCHF) {
    const int a = threadIdx.x / 5, q = threadIdx.x % 5 - 2;
    const double om = a ? pulse_envelope(d.pulse[0], p.tau, t) : 1.0;
    double sn, cs;
    sincos((double)q * p.wd * t, &sn, &cs);
    chi[threadIdx.x] = mk(om * cs, om * sn);
  }
  __syncthreads();
  for (long long e = (long long)blockIdx.x * FT + threadIdx.x; e < p.nnz; e += (long long)gridDim.x * FT)
    d.opv[e] = cmulf(chi[d.chan[e]], d.val[e]);
}

// out[o][i][j] = sum over the CSR row i of operator 1 + o' (o' = o - 1 for the
// jumps, A for o = 0) of opv * in[col][j]; grid (ceil(N / FT), N, 1 + K).
__global__ void __launch_bounds__(FT) fm_apply(FmDev d, FmParams p, const double2* __restrict__ in) {
  const int j = blockIdx.x * FT + threadIdx.x, i = blockIdx.y, o = blockIdx.z;
  if (j >= p.N) return;
  const int* rp = d.rowptr + (size_t)o * (p.N + 1);
  double2 acc = mk(0.0, 0.0);
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const double2 v = d.opv[e], z = in[(size_t)d.col[e] * p.N + j];
    acc.x = fma(v.x, z.x, fma(-v.y, z.y, acc.x));
    acc.y = fma(v.x, z.y, fma(v.y, z.x, acc.y));
  }
  double2* out = o == 0 ? d.B : d.Y + (size_t)(o - 1) * p.N * p.N;
  out[(size_t)i * p.N + j] = acc;
}

// out = in^dag for the 1 + K matrices (B and the Y_k); 32 x 32 tiles.
__global__ void __launch_bounds__(FT) fm_transp(FmDev d, FmParams p) {
  __shared__ double2 tile[32][33];
  const int o = blockIdx.z;
  const double2* in = o == 0 ? d.B : d.Y + (size_t)(o - 1) * p.N * p.N;
  double2* out = o == 0 ? d.Bt : d.Yt + (size_t)(o - 1) * p.N * p.N;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += FT / 32) {
    const int i = y0 + r, j = x0 + tx;
    if (i < p.N && j < p.N) tile[r][tx] = in[(size_t)i * p.N + j];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += FT / 32) {
    const int i = x0 + r, j = y0 + tx;   // out[i][j] = conj(in[j][i])
    if (i < p.N && j < p.N) {
      const double2 v = tile[tx][r];
      out[(size_t)i * p.N + j] = mk(v.x, -v.y);
    }
  }
}

// F = B + Bt + sum_k L_k Yt_k, then the RK4 stage (weights 1/6, 1/3, 1/3, 1/6).
// The thread of (i, j), i <= j, writes entry (i, j) and its conjugate at (j, i):
// rho, the accumulator and the stage inputs stay exactly Hermitian. (The form
// A rho + (A rho)^dag + L (L rho)^dag equals the generator only for Hermitian
// rho; a rounding-level anti-Hermitian part would evolve under -sum_k L_k K
// L_k^dag and grow exponentially.)
__global__ void __launch_bounds__(FT) fm_update(FmDev d, FmParams p, int stage, double dt) {
  const int j = blockIdx.x * FT + threadIdx.x, i = blockIdx.y;
  if (j >= p.N || j < i) return;
  const size_t ij = (size_t)i * p.N + j, ji = (size_t)j * p.N + i;
  const double2 b = d.B[ij], bt = d.Bt[ij];
  double2 f = mk(b.x + bt.x, b.y + bt.y);
  for (int k = 0; k < p.K; ++k) {
    const int* rp = d.rowptr + (size_t)(1 + k) * (p.N + 1);
    const double2* yt = d.Yt + (size_t)k * p.N * p.N;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const double2 v = d.opv[e], z = yt[(size_t)d.col[e] * p.N + j];
      f.x = fma(v.x, z.x, fma(-v.y, z.y, f.x));
      f.y = fma(v.x, z.y, fma(v.y, z.x, f.y));
    }
  }
  if (i == j) f.y = 0.0;
  const double2 r0 = d.rho[ij];
  auto put = [&](double2* a, double2 v) {
    a[ij] = v;
    if (i != j) a[ji] = mk(v.x, -v.y);
  };
  if (stage == 0) {
    put(d.acc, f);
  } else if (stage < 3) {
    const double2 a = d.acc[ij];
    put(d.acc, mk(a.x + 2.0 * f.x, a.y + 2.0 * f.y));
  }
  if (stage < 3) {
    const double c = stage == 2 ? dt : 0.5 * dt;
    put(d.rs, mk(r0.x + c * f.x, r0.y + c * f.y));
  } else {
    const double2 a = d.acc[ij];
    const double h = dt / 6.0;
    const double2 rn = mk(r0.x + h * (a.x + f.x), r0.y + h * (a.y + f.y));
    if (!isfinite(rn.x) || !isfinite(rn.y)) set_error(d.err, DEV_NONFINITE);
    put(d.rho, rn);
    put(d.rs, rn);
  }
}

// rho = (rho + rho^dag) / 2 from its upper triangle (entries (i, j), i <= j, kept,
// the lower triangle their conjugates, the diagonal real).
__global__ void __launch_bounds__(FT) fm_hermitian(double2* rho, int N) {
  const int j = blockIdx.x * FT + threadIdx.x, i = blockIdx.y;
  if (j >= N || j < i) return;
  double2 v = rho[(size_t)i * N + j];
  if (i == j) v.y = 0.0;
  rho[(size_t)i * N + j] = v;
  rho[(size_t)j * N + i] = mk(v.x, -v.y);
}

// beta = tr(rho r) = sum_j sum_e r[j][c] rho[c][j]; at recording steps also the
// populations, tr(r rho r^dag) = sum_j sum_{e, e'} r[j][c] rho[c][c'] conj(r[j][c'])
// and tr rho. One block of 1024 threads; fixed-order reduction.
__global__ void __launch_bounds__(1024) fm_obs(FmDev d, FmParams p, long step, int record) {
  __shared__ double red[32][3 + LR_MAX_NT];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int* rp = d.rowptr + (size_t)(1 + p.K) * (p.N + 1);
  double v[3 + LR_MAX_NT];
  for (int c = 0; c < 3 + LR_MAX_NT; ++c) v[c] = 0.0;
  for (int j = tid; j < p.N; j += 1024) {
    for (int e = rp[j]; e < rp[j + 1]; ++e) {
      const double2 z = cmulf(d.opv[e], d.rho[(size_t)d.col[e] * p.N + j]);
      v[0] += z.x;
      v[1] += z.y;
    }
    if (record) {
      double2 s = mk(0.0, 0.0);
      for (int e = rp[j]; e < rp[j + 1]; ++e)
        for (int e2 = rp[j]; e2 < rp[j + 1]; ++e2) {
          const double2 a = d.opv[e], b = d.opv[e2];
          const double2 t = cmulf(cmulf(a, d.rho[(size_t)d.col[e] * p.N + d.col[e2]]), mk(b.x, -b.y));
          s.x += t.x;
          s.y += t.y;
        }
      v[2] += s.x;
      v[3 + d.level[j]] += d.rho[(size_t)j * p.N + j].x;
    }
  }
  for (int c = 0; c < 3 + LR_MAX_NT; ++c) {
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    if (lane == 0) red[warp][c] = v[c];
  }
  __syncthreads();
  if (tid == 0) {
    double t[3 + LR_MAX_NT];
    for (int c = 0; c < 3 + LR_MAX_NT; ++c) {
      t[c] = 0.0;
      for (int w = 0; w < 32; ++w) t[c] += red[w][c];
    }
    d.beta[step] = mk(t[0], t[1]);
    if (!isfinite(t[0]) || !isfinite(t[1])) set_error(d.err, DEV_NONFINITE);
    if (record) {
      const long rec = step / p.pop_every;
      double tr = 0.0;
      for (int l = 0; l < p.n_levels; ++l) {
        d.pops[rec * p.n_levels + l] = t[3 + l];
        tr += t[3 + l];
      }
      d.nphot[rec] = t[2];
      d.trace[rec] = tr;
    }
  }
}

__global__ void fm_pure(double2* rho, int N, int psi) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)N * N;
       e += (long long)gridDim.x * blockDim.x)
    rho[e] = mk(e == (long long)psi * N + psi ? 1.0 : 0.0, 0.0);
}

// rho = Z Z^dag for a low-rank factor Z [N][M] (the initial state of a low-rank run)
__global__ void __launch_bounds__(FT) fm_from_lowrank(double2* rho, const double2* __restrict__ Z, int N, int M) {
  const int j = blockIdx.x * FT + threadIdx.x, i = blockIdx.y;
  if (j >= N) return;
  double2 s = mk(0.0, 0.0);
  for (int m = 0; m < M; ++m) {
    const double2 a = Z[(size_t)i * M + m], b = Z[(size_t)j * M + m];   // a conj(b)
    s.x = fma(a.x, b.x, fma(a.y, b.y, s.x));
    s.y = fma(a.y, b.x, fma(-a.x, b.y, s.y));
  }
  rho[(size_t)i * N + j] = s;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace lr

using namespace lr;

struct lr_full {
  int N, K, n_levels;
  long nnz, max_steps, n_rec, step;
  int pop_every;
  double wd, tau, dt;
  std::vector<int> rowptr, col, level;
  std::vector<double> val;
  std::vector<unsigned char> chan;
  PulseDev pulse;
  char* ws;
  size_t o_rowptr, o_col, o_val, o_chan, o_level, o_pulse, o_err, o_opv, o_rho, o_rs, o_acc, o_B, o_Bt, o_Y, o_Yt,
      o_beta, o_pops, o_nphot, o_trace, total;
  std::string msg;
};

namespace {

lr_status ffail(lr_full* f, lr_status st, const char* m) {
  if (f) f->msg = m;
  return st;
}
lr_status fcuda(lr_full* f, cudaError_t e) {
  if (f) f->msg = cudaGetErrorString(e);
  return LR_ERR_CUDA;
}

FmDev fdev(const lr_full* f) {
  char* w = f->ws;
  FmDev d;
  d.rowptr = reinterpret_cast<const int*>(w + f->o_rowptr);
  d.col = reinterpret_cast<const int*>(w + f->o_col);
  d.val = reinterpret_cast<const double2*>(w + f->o_val);
  d.chan = reinterpret_cast<const unsigned char*>(w + f->o_chan);
  d.level = reinterpret_cast<const int*>(w + f->o_level);
  d.pulse = reinterpret_cast<const PulseDev*>(w + f->o_pulse);
  d.err = reinterpret_cast<unsigned*>(w + f->o_err);
  d.opv = reinterpret_cast<double2*>(w + f->o_opv);
  d.rho = reinterpret_cast<double2*>(w + f->o_rho);
  d.rs = reinterpret_cast<double2*>(w + f->o_rs);
  d.acc = reinterpret_cast<double2*>(w + f->o_acc);
  d.B = reinterpret_cast<double2*>(w + f->o_B);
  d.Bt = reinterpret_cast<double2*>(w + f->o_Bt);
  d.Y = reinterpret_cast<double2*>(w + f->o_Y);
  d.Yt = reinterpret_cast<double2*>(w + f->o_Yt);
  d.beta = reinterpret_cast<double2*>(w + f->o_beta);
  d.pops = reinterpret_cast<double*>(w + f->o_pops);
  d.nphot = reinterpret_cast<double*>(w + f->o_nphot);
  d.trace = reinterpret_cast<double*>(w + f->o_trace);
  return d;
}

FmParams fparams(const lr_full* f) {
  FmParams p;
  p.N = f->N;
  p.K = f->K;
  p.n_levels = f->n_levels;
  p.nnz = f->nnz;
  p.wd = f->wd;
  p.tau = f->tau;
  p.max_steps = f->max_steps;
  p.n_rec = f->n_rec;
  p.pop_every = f->pop_every;
  return p;
}

}  // namespace

extern "C" lr_status lr_full_create(const lr_sparse_model* m, const lr_pulse* pulse, double tau, long max_steps,
                                    int pop_every, lr_full** out) {
  if (!out) return LR_ERR_ARG;
  *out = nullptr;
  if (!m || !pulse || !m->rowptr || !m->col || !m->val || !m->chan || !m->level) return LR_ERR_ARG;
  if (m->N < 1 || m->N > 16384 || m->n_jumps < 1 || m->n_jumps > LR_SPARSE_MAX_JUMPS) return LR_ERR_ARG;
  if (m->n_levels < 1 || m->n_levels > LR_MAX_NT || m->nnz < 0 || m->nnz > (1L << 31) - 1) return LR_ERR_ARG;
  if (!(tau > 0.0) || max_steps < 1 || pop_every < 1 || !isfinite(m->wd)) return LR_ERR_ARG;
  if (pulse->kind != 0 && pulse->kind != 1) return LR_ERR_ARG;
  const int K = m->n_jumps, N = m->N;
  for (int o = 0; o < K + 2; ++o) {
    const int* rp = m->rowptr + (size_t)o * (N + 1);
    for (int n = 0; n < N; ++n)
      if (rp[n] < 0 || rp[n] > rp[n + 1] || rp[n + 1] > m->nnz) return LR_ERR_ARG;
  }
  for (long e = 0; e < m->nnz; ++e)
    if (m->col[e] < 0 || m->col[e] >= N || m->chan[e] >= NCHF || !isfinite(m->val[2 * e]) ||
        !isfinite(m->val[2 * e + 1]))
      return LR_ERR_ARG;
  for (int n = 0; n < N; ++n)
    if (m->level[n] < 0 || m->level[n] >= m->n_levels) return LR_ERR_ARG;
  for (int k = 0; k < 8; ++k)
    if (!isfinite(pulse->p[k])) return LR_ERR_ARG;
  lr_full* f = new (std::nothrow) lr_full();
  if (!f) return LR_ERR_NOMEM;
  f->N = N;
  f->K = K;
  f->n_levels = m->n_levels;
  f->nnz = m->nnz;
  f->max_steps = max_steps;
  f->pop_every = pop_every;
  f->n_rec = max_steps / pop_every + 1;
  f->step = 0;
  f->wd = m->wd;
  f->tau = tau;
  f->dt = 0.0;
  f->rowptr.assign(m->rowptr, m->rowptr + (size_t)(K + 2) * (N + 1));
  f->col.assign(m->col, m->col + m->nnz);
  f->val.assign(m->val, m->val + 2 * m->nnz);
  f->chan.assign(m->chan, m->chan + m->nnz);
  f->level.assign(m->level, m->level + N);
  f->pulse.kind = pulse->kind;
  for (int k = 0; k < 8; ++k) f->pulse.p[k] = pulse->p[k];
  f->ws = nullptr;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o = al256(o + bytes);
    return r;
  };
  const size_t NN = (size_t)N * N * sizeof(double2);
  f->o_rowptr = take(f->rowptr.size() * sizeof(int));
  f->o_col = take((size_t)f->nnz * sizeof(int));
  f->o_val = take((size_t)f->nnz * sizeof(double2));
  f->o_chan = take((size_t)f->nnz);
  f->o_level = take((size_t)N * sizeof(int));
  f->o_pulse = take(sizeof(PulseDev));
  f->o_err = take(sizeof(unsigned));
  f->o_opv = take((size_t)f->nnz * sizeof(double2));
  f->o_rho = take(NN);
  f->o_rs = take(NN);
  f->o_acc = take(NN);
  f->o_B = take(NN);
  f->o_Bt = take(NN);
  f->o_Y = take(NN * K);
  f->o_Yt = take(NN * K);
  f->o_beta = take((size_t)(max_steps + 1) * sizeof(double2));
  f->o_pops = take((size_t)f->n_rec * f->n_levels * sizeof(double));
  f->o_nphot = take((size_t)f->n_rec * sizeof(double));
  f->o_trace = take((size_t)f->n_rec * sizeof(double));
  f->total = o;
  *out = f;
  return LR_OK;
}

extern "C" lr_status lr_full_workspace_size(const lr_full* f, size_t* bytes) {
  if (!f || !bytes) return LR_ERR_ARG;
  *bytes = f->total;
  return LR_OK;
}

extern "C" lr_status lr_full_bind_workspace(lr_full* f, void* workspace, size_t bytes, void* stream) {
  if (!f || !workspace) return LR_ERR_ARG;
  if (bytes < f->total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return ffail(f, LR_ERR_WORKSPACE, "workspace too small or not 256-byte aligned");
  f->ws = static_cast<char*>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<double2> val(f->nnz);
  for (long e = 0; e < f->nnz; ++e) val[e] = make_double2(f->val[2 * e], f->val[2 * e + 1]);
  cudaError_t e;
  if ((e = cudaMemsetAsync(f->ws, 0, f->total, st)) != cudaSuccess) return fcuda(f, e);
  struct Up {
    size_t off;
    const void* src;
    size_t bytes;
  } ups[] = {{f->o_rowptr, f->rowptr.data(), f->rowptr.size() * sizeof(int)},
             {f->o_col, f->col.data(), f->col.size() * sizeof(int)},
             {f->o_val, val.data(), val.size() * sizeof(double2)},
             {f->o_chan, f->chan.data(), f->chan.size()},
             {f->o_level, f->level.data(), f->level.size() * sizeof(int)},
             {f->o_pulse, &f->pulse, sizeof(PulseDev)}};
  for (const Up& u : ups)
    if (u.bytes && (e = cudaMemcpyAsync(f->ws + u.off, u.src, u.bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return fcuda(f, e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fcuda(f, e);
  return LR_OK;
}

extern "C" lr_status lr_full_set_initial(lr_full* f, int psi, void* stream) {
  if (!f) return LR_ERR_ARG;
  if (!f->ws) return ffail(f, LR_ERR_WORKSPACE, "no workspace bound");
  if (psi < 0 || psi >= f->N) return ffail(f, LR_ERR_ARG, "psi index out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const FmDev d = fdev(f);
  fm_pure<<<1024, FT, 0, st>>>(d.rho, f->N, psi);
  cudaError_t e = cudaMemsetAsync(d.err, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fcuda(f, e);
  f->step = 0;
  f->dt = 0.0;
  return LR_OK;
}

extern "C" lr_status lr_full_set_state(lr_full* f, const double* rho, long step, void* stream) {
  if (!f || !rho) return LR_ERR_ARG;
  if (!f->ws) return ffail(f, LR_ERR_WORKSPACE, "no workspace bound");
  if (step < 0 || step > f->max_steps) return ffail(f, LR_ERR_ARG, "step out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(f->ws + f->o_rho, rho, (size_t)f->N * f->N * sizeof(double2),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    fm_hermitian<<<dim3((f->N + FT - 1) / FT, f->N), FT, 0, st>>>(reinterpret_cast<double2*>(f->ws + f->o_rho), f->N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(f->ws + f->o_err, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fcuda(f, e);
  f->step = step;
  return LR_OK;
}

extern "C" lr_status lr_full_set_state_lowrank(lr_full* f, const double* Z, int M, long step, void* stream) {
  if (!f || !Z) return LR_ERR_ARG;
  if (!f->ws) return ffail(f, LR_ERR_WORKSPACE, "no workspace bound");
  if (M < 1 || M > f->N || step < 0 || step > f->max_steps) return ffail(f, LR_ERR_ARG, "bad rank or step");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double2* zdev = reinterpret_cast<double2*>(f->ws + f->o_B);   // scratch: B holds N^2 >= N M entries
  cudaError_t e = cudaMemcpyAsync(zdev, Z, (size_t)f->N * M * sizeof(double2), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fcuda(f, e);
  fm_from_lowrank<<<dim3((f->N + FT - 1) / FT, f->N), FT, 0, st>>>(reinterpret_cast<double2*>(f->ws + f->o_rho), zdev,
                                                                  f->N, M);
  fm_hermitian<<<dim3((f->N + FT - 1) / FT, f->N), FT, 0, st>>>(reinterpret_cast<double2*>(f->ws + f->o_rho), f->N);
  if ((e = cudaGetLastError()) == cudaSuccess) e = cudaMemsetAsync(f->ws + f->o_err, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fcuda(f, e);
  f->step = step;
  return LR_OK;
}

extern "C" lr_status lr_full_get_state(const lr_full* f, double* rho, void* stream) {
  if (!f || !rho || !f->ws) return LR_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return LR_ERR_CUDA;
  if (cudaMemcpy(rho, f->ws + f->o_rho, (size_t)f->N * f->N * sizeof(double2), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return LR_ERR_CUDA;
  return LR_OK;
}

extern "C" lr_status lr_full_integrate(lr_full* f, double dt, long n_steps, void* stream) {
  if (!f) return LR_ERR_ARG;
  if (!f->ws) return ffail(f, LR_ERR_WORKSPACE, "no workspace bound");
  if (!(dt > 0.0) || !isfinite(dt) || n_steps < 0) return ffail(f, LR_ERR_ARG, "bad dt or n_steps");
  if (f->step + n_steps > f->max_steps) return ffail(f, LR_ERR_STATE, "integration past max_steps");
  if (f->step > 0 && f->dt > 0.0 && dt != f->dt) return ffail(f, LR_ERR_ARG, "dt differs within one pulse run");
  f->dt = dt;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const FmDev d = fdev(f);
  const FmParams p = fparams(f);
  const int N = f->N, K = f->K;
  const unsigned ob = (unsigned)std::min<long long>((f->nnz + FT - 1) / FT, 1024);
  const dim3 ga((N + FT - 1) / FT, N, 1 + K), gt((N + 31) / 32, (N + 31) / 32, 1 + K), gu((N + FT - 1) / FT, N);
  for (long i = 0; i <= n_steps; ++i) {
    const long step = f->step + i;
    const double t = (double)step * dt;
    // observables of rho at the start of this step (r(t) at the step time)
    fm_opvals<<<ob, FT, 0, st>>>(d, p, t);
    fm_obs<<<1, 1024, 0, st>>>(d, p, step, step % f->pop_every == 0);
    if (i == n_steps) break;
    for (int stage = 0; stage < 4; ++stage) {
      const double ts = t + (stage == 0 ? 0.0 : (stage == 3 ? dt : 0.5 * dt));
      if (stage > 0) fm_opvals<<<ob, FT, 0, st>>>(d, p, ts);
      fm_apply<<<ga, FT, 0, st>>>(d, p, stage == 0 ? d.rho : d.rs);
      fm_transp<<<gt, FT, 0, st>>>(d, p);
      fm_update<<<gu, FT, 0, st>>>(d, p, stage, dt);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fcuda(f, e);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fcuda(f, e);
  f->step += n_steps;
  return LR_OK;
}

extern "C" lr_status lr_full_observables(lr_full* f, double* beta, double* pops, double* nphot, double* trace,
                                         void* stream) {
  if (!f) return LR_ERR_ARG;
  if (!f->ws) return ffail(f, LR_ERR_WORKSPACE, "no workspace bound");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  struct Dn {
    void* dst;
    size_t off, bytes;
  } dn[] = {{beta, f->o_beta, (size_t)(f->max_steps + 1) * sizeof(double2)},
            {pops, f->o_pops, (size_t)f->n_rec * f->n_levels * sizeof(double)},
            {nphot, f->o_nphot, (size_t)f->n_rec * sizeof(double)},
            {trace, f->o_trace, (size_t)f->n_rec * sizeof(double)}};
  for (const Dn& x : dn)
    if (x.dst && (e = cudaMemcpyAsync(x.dst, f->ws + x.off, x.bytes, cudaMemcpyDefault, st)) != cudaSuccess)
      return fcuda(f, e);
  unsigned err = 0;
  if ((e = cudaMemcpyAsync(&err, f->ws + f->o_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fcuda(f, e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fcuda(f, e);
  if (err == DEV_NONFINITE) return ffail(f, LR_ERR_NONFINITE, "non-finite value in rho or the signal");
  if (err != 0) return ffail(f, LR_ERR_CUDA, "device error");
  return LR_OK;
}

extern "C" const char* lr_full_last_error(const lr_full* f) { return f ? f->msg.c_str() : "null context"; }
extern "C" void lr_full_destroy(lr_full* f) { delete f; }
