// C ABI of the library: context, validation, workspace layout, launches.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lr_internal.cuh"
#include "lr_fused.cuh"

using lr::DevPtrs;
using lr::PulseDev;
using lr::RunParams;
using lr::TrajDev;

struct lr_ctx {
  int n_cand = 0, n_traj = 0;
  lr_options opt{};
  lr_engine engine = LR_ENGINE_PLAIN;
  std::vector<TrajDev> traj;
  std::vector<PulseDev> pulses;
  int nt_max = 0, max_N = 0, max_M = 0, max_nblk = 0;
  long n_rec = 0;
  long long tot_elems = 0;
  lr::FusedPlan fused{};
  // workspace layout (byte offsets)
  size_t o_traj = 0, o_pulse = 0, o_err = 0, o_zn = 0, o_za = 0, o_zb = 0, o_acc = 0, o_x = 0, o_part = 0,
         o_beta = 0, o_pops = 0, o_nphot = 0, o_trace = 0, o_eps = 0, o_ion = 0, o_loss = 0, o_scratch = 0,
         o_gsnap = 0, o_dpur = 0, o_deig = 0, o_dstep = 0, o_shots = 0, total = 0;
  size_t scratch_bytes = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool have_pulse = false, have_state = false;
  bool z0_valid = false;   // the state at step 0 is kept for lr_backward
  size_t o_z0 = 0;
  double tau = 0.0, dt = 0.0;
  long step = 0;
  std::string last_error;
};

namespace {

lr_status fail(lr_ctx* c, lr_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

lr_status cuda_fail(lr_ctx* c, cudaError_t e, const char* where) {
  return fail(c, LR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

DevPtrs dev_ptrs(const lr_ctx* c) {
  DevPtrs p{};
  char* w = c->ws;
  p.traj = reinterpret_cast<const TrajDev*>(w + c->o_traj);
  p.pulse = reinterpret_cast<const PulseDev*>(w + c->o_pulse);
  p.err = reinterpret_cast<unsigned*>(w + c->o_err);
  p.Zn = w + c->o_zn;
  p.Za = w + c->o_za;
  p.Zb = c->o_zb ? w + c->o_zb : nullptr;
  p.acc = c->o_acc ? w + c->o_acc : nullptr;
  p.X = reinterpret_cast<double2*>(w + c->o_x);
  p.part = c->o_part ? reinterpret_cast<double*>(w + c->o_part) : nullptr;
  p.beta = reinterpret_cast<double2*>(w + c->o_beta);
  p.pops = reinterpret_cast<double*>(w + c->o_pops);
  p.nphot = reinterpret_cast<double*>(w + c->o_nphot);
  p.trace = reinterpret_cast<double*>(w + c->o_trace);
  p.eps_a = reinterpret_cast<double*>(w + c->o_eps);
  p.ion = reinterpret_cast<double*>(w + c->o_ion);
  p.loss = reinterpret_cast<double*>(w + c->o_loss);
  p.scratch = c->scratch_bytes ? w + c->o_scratch : nullptr;
  p.scratch_bytes = (long long)c->scratch_bytes;
  p.gsnap = c->opt.record_gram ? reinterpret_cast<double2*>(w + c->o_gsnap) : nullptr;
  p.dstep = reinterpret_cast<long long*>(w + c->o_dstep);
  return p;
}

RunParams run_params(const lr_ctx* c) {
  RunParams r{};
  r.n_traj = c->n_traj;
  r.n_cand = c->n_cand;
  r.nt_max = c->nt_max;
  r.max_steps = c->opt.max_steps;
  r.n_rec = c->n_rec;
  r.pop_every = c->opt.pop_every;
  r.tau = c->tau;
  r.dt = c->dt;
  r.eta = c->opt.eta;
  r.snap_m = c->opt.record_gram ? c->max_M : 0;
  r.frame = c->opt.frame;
  return r;
}

bool ready(lr_ctx* c) { return c->ws != nullptr; }

// The host copy of the step counter from the device one (graph replays advance
// only the device counter).
cudaError_t refresh_step(lr_ctx* c) {
  long long v = 0;
  cudaError_t e = cudaMemcpy(&v, c->ws + c->o_dstep, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) c->step = (long)v;
  return e;
}

lr_status check_device_error(lr_ctx* c) {
  unsigned e = 0;
  cudaError_t ce = cudaMemcpy(&e, c->ws + c->o_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) return cuda_fail(c, ce, "reading device error word");
  switch (e) {
    case lr::DEV_OK: return LR_OK;
    case lr::DEV_NOT_PD: return fail(c, LR_ERR_NOT_PD, "Gram matrix lost positive definiteness (Cholesky breakdown)");
    case lr::DEV_NONFINITE: return fail(c, LR_ERR_NONFINITE, "non-finite value in the state or readout signal");
    case lr::DEV_TIMEOUT: return fail(c, LR_ERR_TIMEOUT, "a device-side wait ran out of its budget");
    case lr::DEV_CAPACITY:
      return fail(c, LR_ERR_STATE, "an integrate (e.g. a replayed graph) would have passed max_steps; it did not run");
    default: return fail(c, LR_ERR_CUDA, "unknown device error word");
  }
}

}  // namespace

extern "C" {

lr_status lr_create(int n_cand, const lr_model* models, const int* ranks, const lr_options* opt, lr_ctx** out) {
  if (!out) return LR_ERR_ARG;
  *out = nullptr;
  if (n_cand <= 0 || !models || !ranks || !opt) return LR_ERR_ARG;
  if (opt->max_steps < 1 || opt->pop_every < 1 || !(opt->eta > 0.0 && opt->eta <= 1.0)) return LR_ERR_ARG;
  if (opt->precision != LR_PREC_FP64 && opt->precision != LR_PREC_FP32_G64 && opt->precision != LR_PREC_FP32 &&
      opt->precision != LR_PREC_TF32_G64)
    return LR_ERR_ARG;
  if (opt->engine != LR_ENGINE_AUTO && opt->engine != LR_ENGINE_PLAIN && opt->engine != LR_ENGINE_FUSED)
    return LR_ERR_ARG;
  if (opt->record_gram != 0 && opt->record_gram != 1) return LR_ERR_ARG;
  if (opt->frame != 0 && opt->frame != 1) return LR_ERR_ARG;
  lr_ctx* c = new (std::nothrow) lr_ctx();
  if (!c) return LR_ERR_NOMEM;
  c->n_cand = n_cand;
  c->n_traj = 2 * n_cand;
  c->opt = *opt;
  c->n_rec = opt->max_steps / opt->pop_every + 1;
  const int PR = lr::plain_rows_per_block();
  long long z_off = 0, p_off = 0;
  for (int k = 0; k < n_cand; ++k) {
    const lr_model& m = models[k];
    if (m.n_modes != 2 && m.n_modes != 3) { delete c; return LR_ERR_ARG; }
    const int Nt = m.dims[0], Nr = m.dims[1], Nf = m.n_modes == 3 ? m.dims[2] : 1;
    if (Nt < 1 || Nt > LR_MAX_NT || Nr < 1 || Nf < 1) { delete c; return LR_ERR_ARG; }
    const long long N = (long long)Nt * Nr * Nf;
    const int M = ranks[k];
    if (N > (1 << 24) || M < 1 || M > LR_MAX_RANK || M > N) { delete c; return LR_ERR_ARG; }
    const double vals[] = {m.wq, m.alpha, m.wr, m.wf, m.g, m.J, m.kappa, m.gamma};
    for (double v : vals)
      if (!std::isfinite(v)) { delete c; return LR_ERR_ARG; }
    if (m.kappa < 0.0 || m.gamma < 0.0) { delete c; return LR_ERR_ARG; }
    for (int lvl = 0; lvl < 2; ++lvl) {
      TrajDev d{};
      d.N = (int)N;
      d.M = M;
      d.ld = M;
      d.Nt = Nt;
      d.Nr = Nr;
      d.Nf = Nf;
      d.n_modes = m.n_modes;
      d.cand = k;
      d.level0 = lvl < Nt ? lvl : 0;
      d.nblk = (int)((N + PR - 1) / PR);
      d.z_off = z_off;
      d.p_off = p_off;
      d.wq = m.wq;
      d.alpha = m.alpha;
      d.wr = m.wr;
      d.wf = m.n_modes == 3 ? m.wf : 0.0;
      d.g = m.g;
      d.J = m.n_modes == 3 ? m.J : 0.0;
      d.kappa = m.kappa;
      d.gamma = m.gamma;
      z_off += N * M;
      p_off += (long long)d.nblk * (long long)lr::plain_partial_doubles(M);
      c->nt_max = std::max(c->nt_max, Nt);
      c->max_N = std::max(c->max_N, (int)N);
      c->max_M = std::max(c->max_M, M);
      c->max_nblk = std::max(c->max_nblk, d.nblk);
      c->traj.push_back(d);
    }
  }
  c->tot_elems = z_off;
  c->pulses.assign(n_cand, PulseDev{});
  // engine selection
  const bool fused_ok = lr::fused_plan(c->traj, opt->precision, opt->frame, &c->fused);
  if (opt->engine == LR_ENGINE_FUSED && !fused_ok) {
    delete c;
    return LR_ERR_UNSUPPORTED;
  }
  if (opt->engine == LR_ENGINE_PLAIN && opt->precision != LR_PREC_FP64) {
    delete c;
    return LR_ERR_UNSUPPORTED;
  }
  c->engine = opt->engine == LR_ENGINE_PLAIN ? LR_ENGINE_PLAIN
              : (fused_ok ? LR_ENGINE_FUSED : LR_ENGINE_PLAIN);
  // AUTO in FP64 with teams of more than two CTAs per trajectory (a batch far
  // smaller than the GPU): every CTA of a team repeats the FP64 M x M phase, a
  // chain of ~M dependent eliminations on the FP64 pipe, so the plain kernels,
  // which spread that phase over the batch, are faster (GB300, N = 2000, M = 20,
  // 2 trajectories: plain 1471, fused on teams of 10 853 traj*steps/s)
  if (opt->engine == LR_ENGINE_AUTO && fused_ok && opt->precision == LR_PREC_FP64 && c->fused.C > 2)
    c->engine = LR_ENGINE_PLAIN;
  if (c->engine == LR_ENGINE_PLAIN && opt->precision != LR_PREC_FP64) {
    delete c;
    return LR_ERR_UNSUPPORTED;
  }
  // workspace layout
  const size_t A = 256;
  const size_t es = opt->precision == LR_PREC_FP64 ? sizeof(double2) : sizeof(float2);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, A);
    return at;
  };
  c->o_traj = take(sizeof(TrajDev) * c->n_traj);
  c->o_pulse = take(sizeof(PulseDev) * n_cand);
  c->o_err = take(sizeof(unsigned));
  c->o_zn = take(es * c->tot_elems);
  c->o_z0 = take(es * c->tot_elems);
  c->o_za = take(sizeof(double2) * c->tot_elems);
  if (c->engine == LR_ENGINE_PLAIN) {
    c->o_zb = take(sizeof(double2) * c->tot_elems);
    c->o_acc = take(sizeof(double2) * c->tot_elems);
    c->o_part = take(sizeof(double) * (size_t)p_off);
  }
  c->o_x = take(sizeof(double2) * 2 * LR_MAX_RANK * LR_MAX_RANK * c->n_traj);
  c->o_beta = take(sizeof(double2) * (size_t)c->n_traj * (opt->max_steps + 1));
  c->o_pops = take(sizeof(double) * (size_t)c->n_traj * c->n_rec * c->nt_max);
  c->o_nphot = take(sizeof(double) * (size_t)c->n_traj * c->n_rec);
  c->o_trace = take(sizeof(double) * (size_t)c->n_traj * c->n_rec);
  c->o_dstep = take(sizeof(long long));
  c->o_eps = take(sizeof(double) * n_cand);
  c->o_ion = take(sizeof(double) * n_cand);
  c->o_loss = take(sizeof(double) * n_cand);
  // lr_assignment_shots: counts [n_cand][2] (u64), SNR, eps_shots, eps_bin [n_cand]
  c->o_shots = take(sizeof(double) * 5 * n_cand);
  if (opt->record_gram) {
    const size_t nr = (size_t)c->n_traj * c->n_rec;
    c->o_gsnap = take(sizeof(double2) * nr * c->max_M * c->max_M);
    c->o_dpur = take(sizeof(double) * nr);
    c->o_deig = take(sizeof(double) * nr * c->max_M);
  }
  if (c->engine == LR_ENGINE_FUSED) {
    c->scratch_bytes = lr::fused_scratch_bytes(c->fused, c->n_traj);
    if (c->scratch_bytes) c->o_scratch = take(c->scratch_bytes);
  }
  c->total = o;
  *out = c;
  return LR_OK;
}

lr_status lr_workspace_size(const lr_ctx* c, size_t* bytes) {
  if (!c || !bytes) return LR_ERR_ARG;
  *bytes = c->total;
  return LR_OK;
}

lr_status lr_bind_workspace(lr_ctx* c, void* dev_ptr, size_t bytes) {
  if (!c) return LR_ERR_ARG;
  if (!dev_ptr || bytes < c->total) return fail(c, LR_ERR_WORKSPACE, "workspace missing or too small");
  if (reinterpret_cast<uintptr_t>(dev_ptr) % 256 != 0) return fail(c, LR_ERR_WORKSPACE, "workspace not 256-byte aligned");
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, dev_ptr);
  if (e != cudaSuccess || (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return fail(c, LR_ERR_WORKSPACE, "workspace is not device memory");
  }
  c->ws = static_cast<char*>(dev_ptr);
  c->ws_bytes = bytes;
  e = cudaMemcpy(c->ws + c->o_traj, c->traj.data(), sizeof(TrajDev) * c->n_traj, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying trajectory table");
  e = cudaMemset(c->ws + c->o_err, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(c, e, "clearing error word");
  e = cudaMemset(c->ws + c->o_dstep, 0, sizeof(long long));
  if (e != cudaSuccess) return cuda_fail(c, e, "clearing the step counter");
  if (c->engine == LR_ENGINE_FUSED) {
    e = lr::fused_prepare(c->fused, c->opt.precision, c->ws + c->o_scratch, c->n_traj);
    if (e != cudaSuccess) return cuda_fail(c, e, "preparing the fused engine");
  }
  if (c->opt.record_gram) {
    // records that no run writes stay zero matrices
    e = cudaMemset(c->ws + c->o_gsnap, 0,
                   sizeof(double2) * (size_t)c->n_traj * c->n_rec * c->max_M * c->max_M);
    if (e != cudaSuccess) return cuda_fail(c, e, "clearing Gram snapshots");
  }
  c->have_state = false;
  c->have_pulse = false;
  return LR_OK;
}

lr_status lr_set_pulse(lr_ctx* c, const lr_pulse* pulses, double tau, void* stream) {
  if (!c || !pulses) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  if (!(tau > 0.0) || !std::isfinite(tau)) return fail(c, LR_ERR_ARG, "tau must be positive");
  for (int k = 0; k < c->n_cand; ++k) {
    const lr_pulse& P = pulses[k];
    if (P.kind != 0 && P.kind != 1) return fail(c, LR_ERR_ARG, "unknown pulse kind");
    const int np = P.kind == 0 ? 4 : 8;
    for (int i = 0; i < np; ++i)
      if (!std::isfinite(P.p[i])) return fail(c, LR_ERR_ARG, "non-finite pulse parameter");
    const bool widths_ok = P.kind == 0 ? P.p[2] > 0.0 : (P.p[3] > 0.0 && P.p[4] > 0.0 && P.p[5] > 0.0);
    if (!widths_ok) return fail(c, LR_ERR_ARG, "pulse rise/fall/smoothing times must be positive");
    c->pulses[k].kind = P.kind;
    for (int i = 0; i < 8; ++i) c->pulses[k].p[i] = i < np ? P.p[i] : 0.0;
  }
  cudaError_t e = cudaMemcpyAsync(c->ws + c->o_pulse, c->pulses.data(), sizeof(PulseDev) * c->n_cand,
                                  cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "copying pulses");
  e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "copying pulses");
  c->tau = tau;
  c->have_pulse = true;
  return LR_OK;
}

lr_status lr_set_initial(lr_ctx* c, uint64_t seed, double eps, void* stream) {
  if (!c) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  if (!(eps > 0.0) || !((c->max_M - 1) * eps < 1.0)) return fail(c, LR_ERR_ARG, "need eps > 0 and (M-1) eps < 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevPtrs p = dev_ptrs(c);
  RunParams rp = run_params(c);
  cudaError_t e = lr::launch_initial_state(p, rp, c->max_N, c->opt.precision != LR_PREC_FP64, seed, eps, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "initial state kernel");
  e = cudaMemsetAsync(c->ws + c->o_err, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "clearing error word");
  e = cudaMemsetAsync(c->ws + c->o_dstep, 0, sizeof(long long), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "clearing the step counter");
  const size_t es = c->opt.precision == LR_PREC_FP64 ? sizeof(double2) : sizeof(float2);
  e = cudaMemcpyAsync(c->ws + c->o_z0, c->ws + c->o_zn, es * c->tot_elems, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "keeping the initial state");
  c->step = 0;
  c->dt = 0.0;
  c->have_state = true;
  c->z0_valid = true;
  return LR_OK;
}

lr_status lr_set_state(lr_ctx* c, int traj, const double* host_Z, long step, void* stream) {
  if (!c || !host_Z || traj < 0 || traj >= c->n_traj || step < 0 || step > c->opt.max_steps) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const TrajDev& d = c->traj[traj];
  const long long n = (long long)d.N * d.M;
  cudaError_t e;
  if (c->opt.precision == LR_PREC_FP64) {
    e = cudaMemcpyAsync(c->ws + c->o_zn + sizeof(double2) * d.z_off, host_Z, sizeof(double2) * n,
                        cudaMemcpyHostToDevice, s);
  } else {
    char* tmp = c->ws + c->o_za + sizeof(double2) * d.z_off;
    e = cudaMemcpyAsync(tmp, host_Z, sizeof(double2) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = lr::launch_convert(tmp, c->ws + c->o_zn + sizeof(float2) * d.z_off, n, 1, s);
  }
  if (e == cudaSuccess && step == 0) {
    const size_t es = c->opt.precision == LR_PREC_FP64 ? sizeof(double2) : sizeof(float2);
    e = cudaMemcpyAsync(c->ws + c->o_z0 + es * d.z_off, c->ws + c->o_zn + es * d.z_off, es * n,
                        cudaMemcpyDeviceToDevice, s);
  }
  const long long dstep = step;
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->ws + c->o_dstep, &dstep, sizeof(dstep), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "setting state");
  if (step != c->step) c->step = step;
  if (step != 0) c->z0_valid = false;
  if (step == 0) c->dt = 0.0;
  c->have_state = true;
  return LR_OK;
}

lr_status lr_grow_rank(lr_ctx* dst, const lr_ctx* src, uint64_t seed, double eps, void* stream) {
  if (!dst || !src || dst == src) return LR_ERR_ARG;
  if (!ready(dst) || !src->ws) return fail(dst, LR_ERR_WORKSPACE, "no workspace bound");
  if (!src->have_state || !src->have_pulse) return fail(dst, LR_ERR_STATE, "the source has no pulse run");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(dst, LR_ERR_ARG, "need eps > 0");
  if (dst->n_cand != src->n_cand || dst->n_traj != src->n_traj || dst->opt.precision != src->opt.precision ||
      dst->opt.max_steps != src->opt.max_steps || dst->opt.pop_every != src->opt.pop_every ||
      dst->opt.frame != src->opt.frame || dst->nt_max != src->nt_max)
    return fail(dst, LR_ERR_ARG, "the contexts differ in batch, precision, capacity, records or frame");
  for (int t = 0; t < dst->n_traj; ++t) {
    const TrajDev &a = dst->traj[t], &b = src->traj[t];
    if (a.N != b.N || a.Nt != b.Nt || a.Nr != b.Nr || a.Nf != b.Nf || a.n_modes != b.n_modes || a.wq != b.wq ||
        a.alpha != b.alpha || a.wr != b.wr || a.wf != b.wf || a.g != b.g || a.J != b.J || a.kappa != b.kappa ||
        a.gamma != b.gamma)
      return fail(dst, LR_ERR_ARG, "the contexts hold different models");
    if (a.M < b.M) return fail(dst, LR_ERR_ARG, "the destination rank is below the source rank");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dst->pulses = src->pulses;
  cudaError_t e = cudaMemcpyAsync(dst->ws + dst->o_pulse, dst->pulses.data(), sizeof(PulseDev) * dst->n_cand,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dst->ws + dst->o_err, 0, sizeof(unsigned), s);
  if (e == cudaSuccess)
    e = lr::launch_grow(dev_ptrs(dst), dev_ptrs(src), dst->n_traj, dst->opt.precision != LR_PREC_FP64, seed, eps, s);
  // the records of the run so far, and the step counter
  const size_t nt = dst->n_traj, nr = dst->n_rec;
  const struct {
    size_t d, s, bytes;
  } cp[] = {{dst->o_beta, src->o_beta, sizeof(double2) * nt * (dst->opt.max_steps + 1)},
            {dst->o_pops, src->o_pops, sizeof(double) * nt * nr * dst->nt_max},
            {dst->o_nphot, src->o_nphot, sizeof(double) * nt * nr},
            {dst->o_trace, src->o_trace, sizeof(double) * nt * nr},
            {dst->o_eps, src->o_eps, sizeof(double) * dst->n_cand},
            {dst->o_ion, src->o_ion, sizeof(double) * dst->n_cand},
            {dst->o_loss, src->o_loss, sizeof(double) * dst->n_cand},
            {dst->o_dstep, src->o_dstep, sizeof(long long)}};
  for (const auto& x : cp)
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst->ws + x.d, src->ws + x.s, x.bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(dst, e, "growing the rank");
  dst->tau = src->tau;
  dst->dt = src->dt;
  dst->step = src->step;
  dst->have_pulse = true;
  dst->have_state = true;
  dst->z0_valid = false;
  return check_device_error(dst);
}

lr_status lr_get_state(lr_ctx* c, int traj, double* host_Z, void* stream) {
  if (!c || !host_Z || traj < 0 || traj >= c->n_traj) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  if (!c->have_state) return fail(c, LR_ERR_STATE, "no state set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const TrajDev& d = c->traj[traj];
  const long long n = (long long)d.N * d.M;
  cudaError_t e;
  if (c->opt.precision == LR_PREC_FP64) {
    e = cudaMemcpyAsync(host_Z, c->ws + c->o_zn + sizeof(double2) * d.z_off, sizeof(double2) * n,
                        cudaMemcpyDeviceToHost, s);
  } else {
    char* tmp = c->ws + c->o_za + sizeof(double2) * d.z_off;
    e = lr::launch_convert(c->ws + c->o_zn + sizeof(float2) * d.z_off, tmp, n, 0, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_Z, tmp, sizeof(double2) * n, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "reading state");
  return LR_OK;
}

lr_status lr_integrate(lr_ctx* c, double dt, long n_steps, void* stream) {
  if (!c) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  if (!c->have_pulse) return fail(c, LR_ERR_STATE, "lr_set_pulse not called");
  if (!c->have_state) return fail(c, LR_ERR_STATE, "no initial state");
  if (!(dt > 0.0) || !std::isfinite(dt) || n_steps < 0) return fail(c, LR_ERR_ARG, "need dt > 0 and n_steps >= 0");
  if (c->step + n_steps > c->opt.max_steps) return fail(c, LR_ERR_ARG, "n_steps exceeds max_steps capacity");
  if (c->step > 0 && c->dt != 0.0 && c->dt != dt) return fail(c, LR_ERR_STATE, "dt changed within a pulse run");
  c->dt = dt;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "capture status");
  if (cap != cudaStreamCaptureStatusNone && c->engine != LR_ENGINE_FUSED)
    return fail(c, LR_ERR_UNSUPPORTED, "graph capture of lr_integrate needs the fused engine");
  DevPtrs p = dev_ptrs(c);
  RunParams rp = run_params(c);
  cudaError_t e;
  if (c->engine == LR_ENGINE_PLAIN)
    e = lr::plain_integrate(p, rp, c->max_nblk, c->max_N, c->step, n_steps, s);
  else
    e = lr::fused_integrate(c->fused, p, rp, c->opt.precision, c->step, n_steps, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "integrate launch");
  c->step += n_steps;
  e = lr::launch_eps_a(p, rp, n_steps, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "eps_a launch");
  return LR_OK;
}

lr_status lr_observables(lr_ctx* c, double* beta, double* pops, double* nphot, double* trace, double* eps_a,
                         void* stream) {
  if (!c) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  struct Item { void* dst; size_t off, bytes; };
  const Item items[] = {
      {beta, c->o_beta, sizeof(double2) * (size_t)c->n_traj * (c->opt.max_steps + 1)},
      {pops, c->o_pops, sizeof(double) * (size_t)c->n_traj * c->n_rec * c->nt_max},
      {nphot, c->o_nphot, sizeof(double) * (size_t)c->n_traj * c->n_rec},
      {trace, c->o_trace, sizeof(double) * (size_t)c->n_traj * c->n_rec},
      {eps_a, c->o_eps, sizeof(double) * c->n_cand},
  };
  for (const Item& it : items) {
    if (!it.dst) continue;
    cudaError_t e = cudaMemcpyAsync(it.dst, c->ws + it.off, it.bytes, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "copying observables");
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = refresh_step(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronising");
  return check_device_error(c);
}

lr_status lr_loss(lr_ctx* c, double* ionization, double* loss, void* stream) {
  if (!c) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (ionization) e = cudaMemcpyAsync(ionization, c->ws + c->o_ion, sizeof(double) * c->n_cand, cudaMemcpyDefault, s);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, c->ws + c->o_loss, sizeof(double) * c->n_cand, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying the loss");
  return check_device_error(c);
}

lr_status lr_assignment_shots(lr_ctx* c, double eta, long n_shots, int bin_steps, unsigned long long seed,
                              double* eps_shots, double* eps_bin, long long* errors, void* stream) {
  if (!c) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  if (n_shots < 1 || n_shots > 65535L * 256 || bin_steps < 1 || !(eta > 0.0))
    return fail(c, LR_ERR_ARG, "bad n_shots (1 .. 65535 x 256), bin_steps or eta");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = refresh_step(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronising");
  if (c->step < 1) return fail(c, LR_ERR_STATE, "lr_assignment_shots before the first step");
  if ((c->step + bin_steps) / bin_steps > lr::shots_max_bins())
    return fail(c, LR_ERR_ARG, "more than 2048 bins: raise bin_steps");
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(c->ws + c->o_shots);
  double* snr = reinterpret_cast<double*>(c->ws + c->o_shots) + 2 * c->n_cand;
  double* es = snr + c->n_cand;
  double* eb = es + c->n_cand;
  e = lr::launch_shots(dev_ptrs(c), run_params(c), c->step, eta, n_shots, bin_steps, seed, counts, snr, es, eb, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "launching the shot simulation");
  std::vector<unsigned long long> cnt(2 * (size_t)c->n_cand);
  if ((e = cudaMemcpyAsync(cnt.data(), counts, sizeof(unsigned long long) * cnt.size(), cudaMemcpyDeviceToHost, s)) ==
          cudaSuccess &&
      eps_shots)
    e = cudaMemcpyAsync(eps_shots, es, sizeof(double) * c->n_cand, cudaMemcpyDefault, s);
  if (e == cudaSuccess && eps_bin) e = cudaMemcpyAsync(eps_bin, eb, sizeof(double) * c->n_cand, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying the shot results");
  if (errors)
    for (size_t i = 0; i < cnt.size(); ++i) errors[i] = (long long)cnt[i];
  return check_device_error(c);
}

lr_status lr_diagnostics(lr_ctx* c, double* purity, double* eig, void* stream) {
  if (!c) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  if (!c->opt.record_gram) return fail(c, LR_ERR_STATE, "lr_diagnostics needs lr_options.record_gram = 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    cudaError_t e0 = cudaStreamSynchronize(s);
    if (e0 == cudaSuccess) e0 = refresh_step(c);
    if (e0 != cudaSuccess) return cuda_fail(c, e0, "synchronising");
  }
  const size_t nr = (size_t)c->n_traj * c->n_rec;
  double* dpur = reinterpret_cast<double*>(c->ws + c->o_dpur);
  double* deig = reinterpret_cast<double*>(c->ws + c->o_deig);
  cudaError_t e = cudaMemsetAsync(dpur, 0, sizeof(double) * nr, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(deig, 0, sizeof(double) * nr * c->max_M, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "clearing diagnostics");
  const long n_valid = std::min(c->n_rec, c->step / c->opt.pop_every + 1);
  e = lr::launch_diagnostics(dev_ptrs(c), run_params(c), n_valid, dpur, deig, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics kernel");
  if (purity) e = cudaMemcpyAsync(purity, dpur, sizeof(double) * nr, cudaMemcpyDefault, s);
  if (e == cudaSuccess && eig) e = cudaMemcpyAsync(eig, deig, sizeof(double) * nr * c->max_M, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying diagnostics");
  return check_device_error(c);
}

lr_status lr_sync(lr_ctx* c, void* stream) {
  if (!c) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = refresh_step(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronising");
  return check_device_error(c);
}

lr_status lr_backward_workspace_size(const lr_ctx* c, int ckpt_every, size_t* bytes) {
  if (!c || !bytes || ckpt_every < 1) return LR_ERR_ARG;
  if (c->step < 1) return LR_ERR_STATE;
  size_t part = 0;
  for (const TrajDev& d : c->traj) part += (size_t)d.nblk * lr::plain_pstride(d.M);
  const lr::BwdLayout L = lr::bwd_layout(c->tot_elems, c->n_traj, c->n_cand, c->nt_max, part, c->step, ckpt_every,
                                         c->opt.precision != LR_PREC_FP64);
  *bytes = L.total;
  return LR_OK;
}

lr_status lr_backward(lr_ctx* c, void* dev_ws, size_t ws_bytes, const double* d_eps_a, double* d_theta,
                      int ckpt_every, void* stream) {
  if (!c || !d_eps_a || !d_theta || ckpt_every < 1) return LR_ERR_ARG;
  if (!ready(c)) return fail(c, LR_ERR_WORKSPACE, "no workspace bound");
  {
    cudaError_t e0 = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e0 == cudaSuccess) e0 = refresh_step(c);
    if (e0 != cudaSuccess) return cuda_fail(c, e0, "synchronising");
  }
  if (!c->have_pulse || !c->z0_valid || c->step < 1 || !(c->dt > 0.0))
    return fail(c, LR_ERR_STATE, "lr_backward needs a pulse run integrated from step 0 of a kept initial state");
  if (c->opt.frame != 0) return fail(c, LR_ERR_UNSUPPORTED, "lr_backward supports the lab frame only");
  for (int k = 0; k < c->n_cand; ++k)
    if (!std::isfinite(d_eps_a[k])) return fail(c, LR_ERR_ARG, "non-finite cotangent");
  size_t part = 0;
  for (const TrajDev& d : c->traj) part += (size_t)d.nblk * lr::plain_pstride(d.M);
  const lr::BwdLayout L = lr::bwd_layout(c->tot_elems, c->n_traj, c->n_cand, c->nt_max, part, c->step, ckpt_every,
                                         c->opt.precision != LR_PREC_FP64);
  if (!dev_ws || ws_bytes < L.total) return fail(c, LR_ERR_WORKSPACE, "backward workspace missing or too small");
  if (reinterpret_cast<uintptr_t>(dev_ws) % 256 != 0) return fail(c, LR_ERR_WORKSPACE, "backward workspace misaligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevPtrs p = dev_ptrs(c);
  RunParams rp = run_params(c);
  cudaError_t e = lr::backward_run(p, rp, static_cast<char*>(dev_ws), L, c->tot_elems, c->max_nblk, c->max_N, c->step,
                                   c->ws + c->o_z0, c->opt.precision != LR_PREC_FP64, d_eps_a, d_theta, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "backward");
  return check_device_error(c);
}

lr_status lr_query(const lr_ctx* c, lr_info* info) {
  if (!c || !info) return LR_ERR_ARG;
  info->n_cand = c->n_cand;
  info->n_traj = c->n_traj;
  info->nt_max = c->nt_max;
  info->n_rec = c->n_rec;
  info->max_steps = c->opt.max_steps;
  info->step = c->step;
  info->engine = c->engine;
  info->team_size = c->engine == LR_ENGINE_FUSED ? c->fused.C : 0;
  info->stage_in_smem = c->engine == LR_ENGINE_FUSED ? c->fused.zs_smem : 0;
  info->tensor_passes = c->engine == LR_ENGINE_FUSED ? c->fused.tc : 0;
  info->gram_tc = c->engine == LR_ENGINE_FUSED && c->fused.gram_mode == 2 ? 1 : 0;
  return LR_OK;
}

const char* lr_status_string(lr_status s) {
  switch (s) {
    case LR_OK: return "ok";
    case LR_ERR_ARG: return "invalid argument";
    case LR_ERR_CUDA: return "CUDA error";
    case LR_ERR_NOMEM: return "out of host memory";
    case LR_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case LR_ERR_NOT_PD: return "Gram matrix not positive definite";
    case LR_ERR_NONFINITE: return "non-finite value";
    case LR_ERR_TIMEOUT: return "device wait timed out";
    case LR_ERR_STATE: return "call out of order";
    case LR_ERR_UNSUPPORTED: return "configuration not supported";
  }
  return "unknown status";
}

const char* lr_last_error(const lr_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

void lr_destroy(lr_ctx* c) { delete c; }

}  // extern "C"
