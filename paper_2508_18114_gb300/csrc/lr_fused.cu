// FUSED engine, host side: launch planning (variants, team size, cost
// model), workspace layout and launches. The kernel is in lr_fused_kernel.cuh;
// its rotating-frame instantiations are compiled in lr_fused_rwa.cu.
#include <mutex>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "lr_fused_kernel.cuh"

namespace lr {

// ----------------------------------------------------------------- host side

namespace {

struct SmemLayout {
  int o_zs, o_slot, slot_bytes, s_gp, s_tp, s_pop, o_gd, o_w, o_tred, o_trd, o_xs, o_misc, o_tab;
  int o_ta, o_tb, npad, o_gs, total;
};

int al16(int x) { return (x + 15) / 16 * 16; }
int al128(int x) { return (x + 127) / 128 * 128; }

// gs: the two bf16 slice buffers of the tensor-core Gram
SmemLayout layout(int R, int Mp, int zs_smem, size_t es, int tc, int gs) {
  SmemLayout L{};
  int o = 0;
  L.o_zs = o;
  if (zs_smem) o += al16((int)(2 * (size_t)R * (Mp + 1) * es));
  L.s_gp = 0;
  L.s_tp = al16(Mp * Mp * (int)sizeof(double2));
  L.s_pop = L.s_tp + al16(2 * Mp * Mp * (int)es);
  L.slot_bytes = L.s_pop + al16((LR_MAX_NT + 2) * (int)sizeof(double));
  L.o_slot = o;
  o += 2 * L.slot_bytes;
  L.o_gd = o;
  o += al16(Mp * (Mp + 1) * (int)sizeof(double2));
  L.o_w = o;
  o += al16(Mp * (Mp + 1) * (int)sizeof(double2));
  L.o_tred = o;
  o += al16(2 * Mp * Mp * (int)es);
  L.o_trd = o;
  o += al16(Mp * (int)sizeof(double));
  L.o_xs = o;
  o += al16(2 * Mp * Mp * (int)es);
  L.o_misc = o;
  o += al16(168 * (int)sizeof(double));
  L.o_tab = o;
  o += al16(fz::TAB * 7 * (int)(es / 2));
  L.o_ta = L.o_tb = o;
  L.npad = (2 * Mp + 15) / 16 * 16;
  if (tc > 0) {
    const int nbuf = tc == 3 ? 2 : 1;   // big (and small) halves of the TF32 split
    const int K = 4 * Mp;
    o = al128(o);
    L.o_ta = o;
    o += nbuf * fz::TC_ROWS * K * 4;
    L.o_tb = o;
    o += al128(nbuf * L.npad * K * 4);
  }
  L.o_gs = o;
  if (gs) {
    o = al128(o);
    L.o_gs = o;
    o += 2 * GS_BUF;
  }
  L.total = o;
  return L;
}

// tc: tensor-core passes of the projection (0: CUDA cores; 3 or 1: tcgen05,
// L2-resident stage state and FP32 state with the double-word Gram only)
const void* kernel_ptr(lr_precision prec, int zs_smem, int tc, int frame, int gram_mode) {
  if (frame) return fz::rwa_kernel_ptr(prec, zs_smem);
  if (gram_mode == 2) return (const void*)fz::fused_kernel<float2, 2, 0, 0, 0>;
  if (tc == 3) return (const void*)fz::fused_kernel<float2, 1, 0, 3, 0>;
  if (tc == 1) return (const void*)fz::fused_kernel<float2, 1, 0, 1, 0>;
  if (zs_smem) {
    if (prec == LR_PREC_FP64) return (const void*)fz::fused_kernel<double2, 0, 1, 0, 0>;
    if (prec == LR_PREC_FP32) return (const void*)fz::fused_kernel<float2, 0, 1, 0, 0>;
    return (const void*)fz::fused_kernel<float2, 1, 1, 0, 0>;
  }
  if (prec == LR_PREC_FP64) return (const void*)fz::fused_kernel<double2, 0, 0, 0, 0>;
  if (prec == LR_PREC_FP32) return (const void*)fz::fused_kernel<float2, 0, 0, 0, 0>;
  return (const void*)fz::fused_kernel<float2, 1, 0, 0, 0>;
}

// Raise (never lower) a kernel's dynamic shared-memory limit, so that contexts
// planned later cannot shrink it under a context (or a captured graph) that
// needs more.
cudaError_t raise_smem_limit(const void* kern, int bytes) {
  // one lock around the read and the write: two host threads planning at
  // once must not let the smaller request land last
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if (fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int rows_per_cta(const TrajDev& d, int C) {
  return d.Nt * ((d.Nr + C - 1) / C) * d.Nf;
}

}  // namespace

bool fused_plan(const std::vector<TrajDev>& traj, lr_precision prec, int frame, FusedPlan* plan) {
  *plan = FusedPlan{};
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (prop.major < 10) return false;
  const size_t es = prec == LR_PREC_FP64 ? sizeof(double2) : sizeof(float2);
  int Mmax = 0, Nmax = 0, min_nr = 1 << 30;
  bool two = false;
  double max_work = 0.0, tot_work = 0.0;
  for (const TrajDev& d : traj) {
    Mmax = std::max(Mmax, d.M);
    Nmax = std::max(Nmax, d.N);
    if (d.n_modes == 2) two = true;
    min_nr = std::min(min_nr, d.Nr);
    if (d.Nt >= fz::TAB || d.Nr >= fz::TAB || d.Nf >= fz::TAB) return false;
    const double w = (double)d.N * d.M * (d.M + 11.0);
    max_work = std::max(max_work, w);
    tot_work += w;
  }
  const int Mp = (Mmax + 3) / 4 * 4;
  // Variants (stage state placement, tensor-core passes of the projection).
  // Overrides for tuning and tests: LR_FUSED_C = cluster size, LR_FUSED_ZS =
  // "global" keeps the stage state in L2, LR_FUSED_TC = 0 keeps the FP32_G64
  // projection on the CUDA cores (3: only the tensor-core variant).
  int force_c = 0, force_global = 0, force_tc = -1, gram_dw = 0;
  if (const char* e = getenv("LR_FUSED_C")) force_c = atoi(e);
  if (const char* e = getenv("LR_FUSED_GRAM")) gram_dw = strcmp(e, "dw") == 0;
  if (const char* e = getenv("LR_FUSED_ZS")) force_global = strcmp(e, "global") == 0;
  if (const char* e = getenv("LR_FUSED_TC")) force_tc = atoi(e);
  struct Variant {
    int zs_smem, tc, gs;
  };
  std::vector<Variant> vars;
  if (prec == LR_PREC_TF32_G64) {
    if (frame) return false;   // the tensor-core variants are built for the lab frame only
    vars.push_back({0, 1, 0});
  } else {
    if (force_tc != 3) {
      if (!force_global) vars.push_back({1, 0, 0});
      // FP32_G64 in the lab frame at Mp = 20: the Gram matrix on the tensor cores
      // (LR_FUSED_GRAM=dw keeps the double-word CUDA-core sums; 2% slower on the
      // N = 2000, M = 20 batch)
      if (prec == LR_PREC_FP32_G64 && !frame && Mp == 20 && !gram_dw)
        vars.push_back({0, 0, 1});
      else
        vars.push_back({0, 0, 0});
    }
    if (prec == LR_PREC_FP32_G64 && force_tc != 0 && !frame) vars.push_back({0, 3, 0});
  }
  double best = 1e300;
  for (const Variant& v : vars) {
    const int zs_smem = v.zs_smem, tc = v.tc, gs = v.gs;
    const int gmode = gs ? 2 : (prec == LR_PREC_FP32_G64 || prec == LR_PREC_TF32_G64 ? 1 : 0);
    const void* kern = kernel_ptr(prec, zs_smem, tc, frame, gmode);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    const int smem_max = (int)prop.sharedMemPerBlockOptin - (int)fa.sharedSizeBytes;
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int C = 1; C <= 16; ++C) {
      if (two && C > 1) break;
      if (C > min_nr) break;
      if (force_c > 0 && C != force_c) continue;
      int R = 0;
      for (const TrajDev& d : traj) R = std::max(R, rows_per_cta(d, C));
      if (gs && R > GS_MAXR) continue;   // the slice sums stay exact for <= GS_MAXR rows
      const SmemLayout L = layout(R, Mp, zs_smem, es, tc, gs);
      if (L.total > smem_max) continue;
      if (raise_smem_limit(kern, L.total) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(C * 32);
      cfg.blockDim = dim3(fz::threads_for(tc));
      cfg.dynamicSmemBytes = L.total;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl <= 0) {
        cudaGetLastError();
        continue;
      }
      const int n_traj = (int)traj.size();
      // only as many teams as the waves need: the same number of waves, less
      // scratch, and every team runs the same number of trajectories
      const int waves_needed = (n_traj + ncl - 1) / ncl;
      const int used = std::min((n_traj + waves_needed - 1) / waves_needed, n_traj);
      // Cost model, fitted to measurements on GB300 (N = 2000, M = 20 batch):
      // a stage costs ~0.16 us per row per CTA with the stage state in shared
      // memory (x1.3 in L2; x1.7 and x1.55 in L2 with the projection on the
      // tensor cores in 3 and 1 passes: per 128-row tile the operand staging
      // and two block barriers cost more than the FMAs they replace), plus a
      // fixed ~60 us per team (the M x M phase and the cluster barrier, ~M
      // sequential elimination steps) that does not shrink with C; teams run
      // trajectories in waves.
      const double row_cost = zs_smem ? 1.0 : (tc == 3 ? 1.7 : tc == 1 ? 1.55 : gs ? 1.0 : 1.3);
      const double waves = std::ceil((double)n_traj / used);
      double t = 0.0;
      for (const TrajDev& d : traj) {
        const double rows = (double)rows_per_cta(d, C) * row_cost * (d.M * d.M) / 400.0;
        const double fixed = 375.0 * d.M / 20.0 * (C > 1 ? 1.0 : 0.95);
        t += rows + fixed;
      }
      t = waves * t / n_traj;
      if (t < best) {
        best = t;
        plan->ok = 1;
        plan->C = C;
        plan->n_clusters = used;
        plan->threads = fz::threads_for(tc);
        plan->smem = L.total;
        plan->zs_smem = zs_smem;
        plan->tc = tc;
        plan->frame = frame;
        plan->Mp = Mp;
        plan->R = R;
        plan->Nmax = Nmax;
        plan->gram_mode = gmode;
        plan->es = (int)es;
      }
    }
  }
  if (!plan->ok) return false;
  // largest work first, round-robin over the teams
  std::vector<std::pair<double, int>> w;
  for (size_t j = 0; j < traj.size(); ++j)
    w.push_back({-(double)traj[j].N * traj[j].M * (traj[j].M + 11.0), (int)j});
  std::stable_sort(w.begin(), w.end());
  for (auto& x : w) plan->order.push_back(x.second);
  return true;
}

size_t fused_scratch_bytes(const FusedPlan& plan, int n_traj) {
  // order list, then global stage buffers (only without smem residency) and accumulators per team
  size_t b = ((sizeof(int) * n_traj + 255) / 256) * 256;
  const size_t es = plan.es;
  if (!plan.zs_smem)
    b += ((2 * (size_t)plan.R * (plan.Mp + 1) * es * plan.C * plan.n_clusters + 255) / 256) * 256;
  b += (((size_t)plan.Nmax * plan.Mp * es * plan.n_clusters + 255) / 256) * 256;
  return b;
}

cudaError_t fused_prepare(const FusedPlan& plan, lr_precision prec, void* scratch, int n_traj) {
  cudaError_t e = cudaMemcpy(scratch, plan.order.data(), sizeof(int) * n_traj, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  const size_t es = prec == LR_PREC_FP64 ? sizeof(double2) : sizeof(float2);
  const SmemLayout L = layout(plan.R, plan.Mp, plan.zs_smem, es, plan.tc, plan.gram_mode == 2);
  const void* kern = kernel_ptr(prec, plan.zs_smem, plan.tc, plan.frame, plan.gram_mode);
  e = raise_smem_limit(kern, L.total);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t fused_integrate(const FusedPlan& plan, const DevPtrs& p, const RunParams& rp, lr_precision prec,
                            long step0, long n_steps, cudaStream_t s) {
  const size_t es = prec == LR_PREC_FP64 ? sizeof(double2) : sizeof(float2);
  const SmemLayout L = layout(plan.R, plan.Mp, plan.zs_smem, es, plan.tc, plan.gram_mode == 2);
  fz::Args a{};
  a.p = p;
  a.rp = rp;
  a.step0 = step0;
  a.n_steps = n_steps;
  a.C = plan.C;
  a.n_clusters = plan.n_clusters;
  a.Mp = plan.Mp;
  a.R = plan.R;
  a.Nmax = plan.Nmax;
  a.zs_smem = plan.zs_smem;
  a.o_zs = L.o_zs;
  a.o_slot = L.o_slot;
  a.slot_bytes = L.slot_bytes;
  a.s_gp = L.s_gp;
  a.s_tp = L.s_tp;
  a.s_pop = L.s_pop;
  a.o_gd = L.o_gd;
  a.o_w = L.o_w;
  a.o_tred = L.o_tred;
  a.o_trd = L.o_trd;
  a.o_xs = L.o_xs;
  a.o_misc = L.o_misc;
  a.o_tab = L.o_tab;
  a.o_ta = L.o_ta;
  a.o_tb = L.o_tb;
  a.npad = L.npad;
  a.o_gs = L.o_gs;
  char* sc = static_cast<char*>(p.scratch);
  size_t off = ((sizeof(int) * rp.n_traj + 255) / 256) * 256;
  a.order = reinterpret_cast<const int*>(sc);
  if (!plan.zs_smem) {
    a.zs_glob = sc + off;
    off += ((2 * (size_t)plan.R * (plan.Mp + 1) * es * plan.C * plan.n_clusters + 255) / 256) * 256;
  }
  a.acc_glob = sc + off;
  // test hook of the device-wait timeout path (see Args::debug_wait)
  if (const char* e = getenv("LR_DEBUG_WAIT_CYCLES")) a.debug_wait = atoll(e);
  // the trajectory order is in the scratch since fused_prepare; the kernel's
  // attributes are raised here only outside a stream capture
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  if (cap == cudaStreamCaptureStatusNone) {
    const void* kern = kernel_ptr(prec, plan.zs_smem, plan.tc, plan.frame, plan.gram_mode);
    e = raise_smem_limit(kern, L.total);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan.C * plan.n_clusters);
  cfg.blockDim = dim3(plan.threads);
  cfg.dynamicSmemBytes = L.total;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = plan.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (plan.frame) return fz::rwa_launch(cfg, prec, plan.zs_smem, a);
  if (plan.gram_mode == 2) return cudaLaunchKernelEx(&cfg, fz::fused_kernel<float2, 2, 0, 0, 0>, a);
  if (plan.tc == 3) return cudaLaunchKernelEx(&cfg, fz::fused_kernel<float2, 1, 0, 3, 0>, a);
  if (plan.tc == 1) return cudaLaunchKernelEx(&cfg, fz::fused_kernel<float2, 1, 0, 1, 0>, a);
  if (plan.zs_smem) {
    if (prec == LR_PREC_FP64) return cudaLaunchKernelEx(&cfg, fz::fused_kernel<double2, 0, 1, 0, 0>, a);
    if (prec == LR_PREC_FP32) return cudaLaunchKernelEx(&cfg, fz::fused_kernel<float2, 0, 1, 0, 0>, a);
    return cudaLaunchKernelEx(&cfg, fz::fused_kernel<float2, 1, 1, 0, 0>, a);
  }
  if (prec == LR_PREC_FP64) return cudaLaunchKernelEx(&cfg, fz::fused_kernel<double2, 0, 0, 0, 0>, a);
  if (prec == LR_PREC_FP32) return cudaLaunchKernelEx(&cfg, fz::fused_kernel<float2, 0, 0, 0, 0>, a);
  return cudaLaunchKernelEx(&cfg, fz::fused_kernel<float2, 1, 0, 0, 0>, a);
}

}  // namespace lr
