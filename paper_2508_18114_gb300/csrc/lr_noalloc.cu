// lr_integrate_plain_noalloc: the plain FP64 engine for one trajectory with
// its scratch memory in a fixed, file-scope device array instead of a
// caller-bound workspace, for callers that cannot allocate device memory.
#include <climits>
#include <mutex>

#include "lr_internal.cuh"

namespace lr {
namespace {

// Limits of the static scratch (see include/lr.h).
constexpr int NA_MAX_N = 4096;
constexpr long long NA_MAX_NM = 65536;
constexpr int NA_MAX_M = LR_MAX_RANK;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Byte layout of the scratch array.
constexpr size_t NA_OFF_TRAJ = 0;
constexpr size_t NA_OFF_PULSE = align256(NA_OFF_TRAJ + sizeof(TrajDev));
constexpr size_t NA_OFF_ERR = align256(NA_OFF_PULSE + sizeof(PulseDev));
constexpr size_t NA_OFF_POPS = align256(NA_OFF_ERR + sizeof(unsigned));
constexpr size_t NA_OFF_NPHOT = align256(NA_OFF_POPS + sizeof(double) * LR_MAX_NT);
constexpr size_t NA_OFF_TRACE = align256(NA_OFF_NPHOT + sizeof(double));
constexpr size_t NA_OFF_X = align256(NA_OFF_TRACE + sizeof(double));
constexpr size_t NA_OFF_ZA = align256(NA_OFF_X + sizeof(double2) * 2 * LR_MAX_RANK * LR_MAX_RANK);
constexpr size_t NA_OFF_ZB = align256(NA_OFF_ZA + sizeof(double2) * NA_MAX_NM);
constexpr size_t NA_OFF_ACC = align256(NA_OFF_ZB + sizeof(double2) * NA_MAX_NM);
constexpr size_t NA_OFF_PART = align256(NA_OFF_ACC + sizeof(double2) * NA_MAX_NM);
constexpr size_t NA_PART_BLOCKS = (NA_MAX_N + 15) / 16;
constexpr size_t NA_PART_STRIDE = (size_t)6 * NA_MAX_M * NA_MAX_M + LR_MAX_NT + 2;   // doubles per block
constexpr size_t NA_BYTES = align256(NA_OFF_PART + sizeof(double) * NA_PART_BLOCKS * NA_PART_STRIDE);

// The scratch array. Host code must not take its address directly: the
// symbol's host-side name is only a stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
// Device address of the array per device, guarded by g_scratch_mu. Outside
// stream capture every call looks the address up again (cheap, and not a
// stream operation), so a device reset or context teardown that reloads the
// module and moves the array cannot leave a stale pointer; inside a capture
// the address of the last call made outside capture is used.
static void* g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};
static std::mutex g_scratch_mu;

// Write the one-trajectory tables into the scratch and clear the error word
// (no host-to-device copy is needed: the tables travel as kernel arguments).
__global__ void noalloc_tables_kernel(TrajDev d, PulseDev pd, unsigned char* base) {
  *reinterpret_cast<TrajDev*>(base + NA_OFF_TRAJ) = d;
  *reinterpret_cast<PulseDev*>(base + NA_OFF_PULSE) = pd;
  *reinterpret_cast<unsigned*>(base + NA_OFF_ERR) = 0u;
}

}  // namespace
}  // namespace lr

extern "C" lr_status lr_integrate_plain_noalloc(const lr_model* m, int M, const lr_pulse* pulse, double tau,
                                                double* Z, double* beta, double dt, long step0, long n_steps,
                                                void* stream) {
  using namespace lr;
  if (!m || !pulse || !Z || !beta) return LR_ERR_ARG;
  if (m->n_modes != 2 && m->n_modes != 3) return LR_ERR_ARG;
  const int Nt = m->dims[0], Nr = m->dims[1], Nf = m->n_modes == 3 ? m->dims[2] : 1;
  if (Nt < 1 || Nt > LR_MAX_NT || Nr < 1 || Nf < 1) return LR_ERR_ARG;
  const long long N = (long long)Nt * Nr * Nf;
  if (M < 1 || M > N) return LR_ERR_ARG;
  if (N > NA_MAX_N || M > NA_MAX_M || N * M > NA_MAX_NM) return LR_ERR_UNSUPPORTED;
  if (!(dt > 0.0) || !(tau > 0.0) || step0 < 0 || n_steps < 0 || step0 + n_steps >= (long)INT_MAX)
    return LR_ERR_ARG;
  if (pulse->kind != 0 && pulse->kind != 1) return LR_ERR_ARG;
  if (m->kappa < 0.0 || m->gamma < 0.0) return LR_ERR_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return LR_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return LR_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cs == cudaStreamCaptureStatusNone) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return LR_ERR_CUDA;
      g_scratch_ptr[dev] = ptr;
    } else if (!g_scratch_ptr[dev]) {
      return LR_ERR_STATE;   // the first call on a device must come before any capture
    }
    base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  }

  TrajDev d{};
  d.N = (int)N;
  d.M = M;
  d.ld = M;
  d.Nt = Nt;
  d.Nr = Nr;
  d.Nf = Nf;
  d.n_modes = m->n_modes;
  d.cand = 0;
  d.level0 = 0;
  d.nblk = (int)((N + 15) / 16);
  d.z_off = 0;
  d.p_off = 0;
  d.wq = m->wq;
  d.alpha = m->alpha;
  d.wr = m->wr;
  d.wf = m->n_modes == 3 ? m->wf : 0.0;
  d.g = m->g;
  d.J = m->n_modes == 3 ? m->J : 0.0;
  d.kappa = m->kappa;
  d.gamma = m->gamma;
  PulseDev pd{};
  pd.kind = pulse->kind;
  for (int i = 0; i < 8; ++i) pd.p[i] = pulse->p[i];

  noalloc_tables_kernel<<<1, 1, 0, s>>>(d, pd, base);
  if (cudaGetLastError() != cudaSuccess) return LR_ERR_CUDA;

  DevPtrs p{};
  p.traj = reinterpret_cast<const TrajDev*>(base + NA_OFF_TRAJ);
  p.pulse = reinterpret_cast<const PulseDev*>(base + NA_OFF_PULSE);
  p.err = reinterpret_cast<unsigned*>(base + NA_OFF_ERR);
  p.Zn = Z;
  p.Za = base + NA_OFF_ZA;
  p.Zb = base + NA_OFF_ZB;
  p.acc = base + NA_OFF_ACC;
  p.X = reinterpret_cast<double2*>(base + NA_OFF_X);
  p.part = reinterpret_cast<double*>(base + NA_OFF_PART);
  // the engine indexes beta by absolute step; the caller's buffer starts at step0
  p.beta = reinterpret_cast<double2*>(beta) - step0;
  p.pops = reinterpret_cast<double*>(base + NA_OFF_POPS);
  p.nphot = reinterpret_cast<double*>(base + NA_OFF_NPHOT);
  p.trace = reinterpret_cast<double*>(base + NA_OFF_TRACE);
  p.eps_a = nullptr;
  p.ion = nullptr;
  p.loss = nullptr;

  RunParams rp{};
  rp.n_traj = 1;
  rp.n_cand = 1;
  rp.nt_max = Nt;
  rp.max_steps = step0 + n_steps;
  rp.n_rec = 1;
  rp.pop_every = INT_MAX;   // populations only at step 0, into the scratch
  rp.tau = tau;
  rp.dt = dt;
  rp.eta = 0.6;
  if (plain_integrate(p, rp, d.nblk, d.N, step0, n_steps, s) != cudaSuccess) return LR_ERR_CUDA;

  unsigned err = 0;
  if (cudaMemcpyAsync(&err, base + NA_OFF_ERR, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return LR_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LR_ERR_CUDA;
  switch (err) {
    case DEV_OK: return LR_OK;
    case DEV_NOT_PD: return LR_ERR_NOT_PD;
    case DEV_NONFINITE: return LR_ERR_NONFINITE;
    default: return LR_ERR_TIMEOUT;
  }
}
