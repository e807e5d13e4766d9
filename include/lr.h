/*
 * lr.h - C ABI of the GB300 low-rank Lindblad readout library.
 *
 * The library time-integrates the low-rank ansatz rho = Z Z^dag (Z complex,
 * N x M, M << N) under the non-stochastic matrix Schroedinger equation of
 * Sec. S1.A (Eq. S5):
 *
 *     dZ/dt = -i H(t) Z + O[Z],
 *     O[Z]  = 1/2 sum_k [ L_k Z (Z^+ L_k Z)^dag - L_k^dag L_k Z ],
 *     Z^+   = (Z^dag Z)^{-1} Z^dag            (Moore-Penrose inverse),
 *
 * for the driven transmon-resonator(-filter) readout model of Eq. 1 / Eq. 2,
 * in the bare-mode Duffing form without the rotating-wave approximation:
 *
 *     H(t) = wq b^dag b + (alpha/2) b^dag b^dag b b + wr a^dag a
 *            + g (b + b^dag)(a + a^dag)
 *            [ + wf f^dag f + J (a + a^dag)(f + f^dag) ]
 *            + Omega(t) cos(w_d t + phi) (r + r^dag),
 *     L_1 = sqrt(kappa) r,   L_2 = sqrt(gamma) b,
 *
 * where r, the readout mode, is the last mode (a with two modes, the filter
 * f with three). Time stepping is classical fixed-step RK4. Observables are
 * the readout signal beta(t) = tr(rho r) (Fig. 2), transmon level
 * populations, the readout-mode photon number tr(rho r^dag r), tr rho, and
 * the assignment error of Sec. S3.A (Eqs. S-SNR, S-separation_error,
 * S-assignment_error):
 *
 *     SNR   = sqrt(2 eta kappa int_0^tau |beta_e - beta_g|^2 dt),
 *     eps_a = 1/2 erfc(SNR/2) + tau gamma / 2.
 *
 * Units: ns, rad/ns, 1/ns.
 *
 * Work is organised in *candidates* (one pulse each). Every candidate c owns
 * two trajectories: 2c starts from the transmon ground state |g,0,0> and
 * 2c+1 from the first excited state |e,0,0> (Eq. S(initial states)).
 *
 * Memory ownership: the context (host) is allocated by lr_create and freed
 * by lr_destroy. The library never allocates device memory: every device
 * buffer lives in one caller-owned workspace (e.g. a torch tensor's storage)
 * bound with lr_bind_workspace, which must stay alive and unmodified while
 * the context uses it. Host buffers passed to the calls are owned by the
 * caller and only read/written during the call.
 *
 * Errors: every call returns an lr_status; nothing crosses the ABI as an
 * exception. lr_last_error() gives a human-readable message for the last
 * failing call on a context. Device-side failures (Cholesky breakdown,
 * non-finite values, a device wait that ran out) set an error word in the
 * workspace; lr_observables and lr_sync read it and return the status.
 *
 * Streams: `stream` arguments are cudaStream_t values passed as void*
 * (NULL = the legacy default stream). Calls marked "async" only enqueue work.
 *
 * Threading: a context is not thread-safe; distinct contexts are independent.
 * Determinism: with the same inputs, seed and options, results are bitwise
 * identical from run to run (all reductions use a fixed order).
 */
#ifndef LR_H
#define LR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LR_ABI_VERSION 1
#define LR_MAX_RANK 32      /* largest supported rank M */
#define LR_MAX_NT 16        /* largest supported transmon truncation N_t */

typedef struct lr_ctx lr_ctx;

typedef enum {
  LR_OK = 0,
  LR_ERR_ARG = 1,         /* invalid argument: null pointer, size or value out of range */
  LR_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
  LR_ERR_NOMEM = 3,       /* host allocation failed */
  LR_ERR_WORKSPACE = 4,   /* no workspace bound, or it is too small or misaligned */
  LR_ERR_NOT_PD = 5,      /* Gram matrix Z^dag Z not positive definite (Cholesky breakdown) */
  LR_ERR_NONFINITE = 6,   /* NaN/Inf reached the state or the readout signal */
  LR_ERR_TIMEOUT = 7,     /* a device-side wait exceeded its iteration budget */
  LR_ERR_STATE = 8,       /* call out of order (e.g. integrate before set_pulse) */
  LR_ERR_UNSUPPORTED = 9  /* configuration not supported by the selected engine */
} lr_status;

/* Arithmetic of the bulk state. FP64: complex128 everywhere.
 * FP32_G64 (FUSED engine): Z, the operator apply, the projections
 * T_k = Z^dag L_k Z, the projection term and the RK4 stages in complex64.
 * The Gram matrix Z^dag Z is accumulated from exact FP32 products in a
 * double-word FP32 sum (hi + lo floats, about 2^-48 relative: FP64-class,
 * not IEEE FP64). Its LDL^dag factorisation, L^-1 and G^-1 run in the same
 * double-word FP32 arithmetic (Dekker products, Knuth sums, a Newton
 * reciprocal; about 2^-48 relative), and so is X_k = G^-1 T_k (from the FP32
 * T_k), which is rounded to FP32 once. The readout signal beta, the populations,
 * photons and trace are summed in FP64 from the FP32 state, and eps_a, T and
 * Lambda are computed in FP64. Where the fused engine keeps the stage state
 * in L2 it may run the projection term (the Y_k X_k^dag product of Eq. S5)
 * on the tensor cores as three TF32 passes of a two-term split (FP32-class
 * products, lr_info.tensor_passes = 3).
 * FP32 (FUSED engine): as FP32_G64 but with the Gram matrix accumulated in
 * plain FP32.
 * TF32_G64 (FUSED engine): as FP32_G64 with the projection term in ONE TF32
 * tensor-core pass (operands rounded to 10-bit mantissas, FP32
 * accumulation): the reduced-precision variant, for measuring its error;
 * only for batches whose operand tiles fit in shared memory (else
 * LR_ERR_UNSUPPORTED).
 * The PLAIN engine runs FP64 only. */
typedef enum { LR_PREC_FP64 = 0, LR_PREC_FP32_G64 = 1, LR_PREC_FP32 = 2, LR_PREC_TF32_G64 = 3 } lr_precision;

/* PLAIN: straightforward HBM-resident kernels, several launches per RK4
 * stage (the reference GPU path). FUSED: one persistent launch per
 * integrate call, state resident on chip. AUTO picks FUSED when supported,
 * except for FP64 contexts whose fused plan needs teams of more than two CTAs
 * per trajectory (batches far smaller than the GPU), which run PLAIN. */
typedef enum { LR_ENGINE_AUTO = 0, LR_ENGINE_PLAIN = 1, LR_ENGINE_FUSED = 2 } lr_engine;

typedef struct {
  int n_modes;        /* 2: transmon x resonator; 3: transmon x resonator x filter */
  int dims[3];        /* N_t (<= LR_MAX_NT), N_r, N_f; dims[2] ignored when n_modes == 2 */
  double wq, alpha;   /* transmon frequency and anharmonicity [rad/ns] */
  double wr, wf;      /* resonator / filter frequency [rad/ns] (wf ignored with 2 modes) */
  double g, J;        /* transmon-resonator / resonator-filter coupling [rad/ns] */
  double kappa;       /* decay rate of the readout (last) mode [1/ns] */
  double gamma;       /* transmon decay rate 1/T1 [1/ns] */
} lr_model;

/* Pulse envelope Omega(t), Sec. S2.C, logistic f(t,t0,s) = 1/(1+exp(-(t-t0)/s)):
 *  kind 0 flat-top:    p = {A, w_d, t_r, phi};  s = t_r/5, t0 = 6 s,
 *                      Omega = A f(t,t0,s) [1 - f(t,tau-t0,s)].
 *  kind 1 two-segment: p = {A1, A2, t_sw, t_rise, t_fall, t_sm, w_d, phi};
 *                      Omega = A1 f(t,6 t_rise/5,t_rise/5)
 *                            + (A2-A1) f(t,t_sw,t_sm/5)
 *                            - A2 f(t,tau-6 t_fall/5,t_fall/5).
 *  The term in H is Omega(t) cos(w_d t + phi) (r + r^dag). */
typedef struct {
  int kind;
  double p[8];
} lr_pulse;

typedef struct {
  lr_precision precision;
  lr_engine engine;
  long max_steps;     /* capacity: largest total number of RK4 steps per pulse run */
  int pop_every;      /* record populations, photons, trace every pop_every steps (>= 1) */
  double eta;         /* measurement efficiency in the SNR (the paper uses 0.6) */
  int record_gram;    /* 1: keep the FP64 Gram matrix Z^dag Z at every record step for
                         lr_diagnostics (the workspace grows by n_traj * n_rec *
                         (max_M^2 * 16 + max_M * 8 + 8) bytes); 0: off */
  int frame;          /* 0: lab frame, H(t) as in lr_pulse (no rotating-wave approximation).
                         1: frame rotating at each candidate's w_d with the rotating-wave
                         approximation (the RWA Hamiltonian of Sec. S2): mode frequencies
                         become detunings w - w_d, the couplings keep g (b^dag a + b a^dag)
                         and J (a^dag f + a f^dag), and the drive is (Omega(t)/2)
                         (e^{i phi} r + e^{-i phi} r^dag). The jump operators are unchanged.
                         beta is then the rotating-frame signal, beta_lab e^{i w_d t}, so
                         |beta_e - beta_g|, eps_a and all populations keep their meaning.
                         A slow Hamiltonian allows a larger dt. lr_backward supports frame 0
                         only. */
} lr_options;

typedef struct {
  int n_cand, n_traj;
  int nt_max;         /* largest N_t in the batch: pops row length */
  long n_rec;         /* recorded points per trajectory: max_steps / pop_every + 1 */
  long max_steps;
  long step;          /* RK4 steps taken since lr_set_initial / lr_set_state */
  lr_engine engine;   /* engine actually used */
  int team_size;      /* CTAs per trajectory (FUSED) */
  int stage_in_smem;  /* FUSED: 1 stage state in shared memory, 0 in L2 */
  int tensor_passes;  /* FUSED: TF32 tensor-core passes of the projection term (0: CUDA cores) */
  int gram_tc;        /* FUSED, FP32_G64: 1 when the Gram matrix is formed on the tensor cores
                         (exact bf16 slices, double-word sums; the default in the lab frame
                         with the rank padded to 20 and <= 1024 rows per CTA), 0 for the
                         double-word CUDA-core sums (LR_FUSED_GRAM=dw at lr_create) */
} lr_info;

/* Create a context for n_cand candidates (2 n_cand trajectories).
 * models[c], ranks[c]: model and rank M (1 <= M <= min(N, LR_MAX_RANK)) of
 * candidate c. Host arrays are copied. No device memory is touched. */
lr_status lr_create(int n_cand, const lr_model* models, const int* ranks,
                    const lr_options* opt, lr_ctx** out);

/* Device bytes the context needs in its workspace. */
lr_status lr_workspace_size(const lr_ctx* ctx, size_t* bytes);

/* Bind caller-owned device memory (>= lr_workspace_size bytes, 256-byte
 * aligned). The library keeps the pointer; it does not free it. */
lr_status lr_bind_workspace(lr_ctx* ctx, void* dev_ptr, size_t bytes);

/* Set the pulse of every candidate (pulses[n_cand], host) and the pulse
 * duration tau [ns] that places the falling edges. Async (copies from a
 * context-owned staging buffer). */
lr_status lr_set_pulse(lr_ctx* ctx, const lr_pulse* pulses, double tau, void* stream);

/* Fixed-rank initial condition of Sec. S1.A on the device:
 * Z(0) = (sqrt(1-(M-1) eps) psi, sqrt(eps) q_2, ..., sqrt(eps) q_M), with
 * psi = |g or e, 0, 0> and q_j the Gram-Schmidt orthonormalisation of
 * (psi, xi_2, ..., xi_M), xi_j complex Gaussian vectors drawn by SplitMix64 +
 * Box-Muller (per-trajectory seed = SplitMix64 output number `traj` of
 * `seed`; pair p = (j-1) N + n uses uniforms 2p and 2p+1, u = ((x>>11)+1)/2^53,
 * xi = sqrt(-2 ln u1) exp(2 pi i u2)). Resets the step counter and the
 * recorded observables. 0 < eps, (M-1) eps < 1. Async. */
lr_status lr_set_initial(lr_ctx* ctx, uint64_t seed, double eps, void* stream);

/* Replace the state of one trajectory with host_Z (complex, row-major
 * [N][M] as interleaved (re, im) doubles) and set the step counter to
 * `step` (for resuming a run; all trajectories share one counter).
 * Synchronous. */
lr_status lr_set_state(lr_ctx* ctx, int traj, const double* host_Z, long step, void* stream);

/* Copy the current state of one trajectory to host_Z (layout as above).
 * Synchronous. */
lr_status lr_get_state(lr_ctx* ctx, int traj, double* host_Z, void* stream);

/* Adaptive rank (Sec. S1.B: the rank is raised when the smallest eigenvalue
 * of rho = Z Z^dag is no longer small against the largest). Continues the pulse
 * run of `src` in `dst`, a context created with the same models, options and
 * workspace kind but ranks M_dst >= M_src per candidate: every trajectory's
 * state becomes Z_dst = [Z_src, sqrt(eps) q_{M_src}, ..., sqrt(eps) q_{M_dst-1}],
 * with q_j the normalised component of a complex Gaussian vector (the
 * generator of lr_set_initial, trajectory seed = output `traj` of `seed`,
 * pair index (j - M_src) N + n) orthogonal to span(Z_src) and to the q before
 * it; rho gains eps (M_dst - M_src) of trace. Copies the pulses, the step
 * counter and the records (beta, populations, photons, trace, eps_a, T,
 * Lambda); Gram snapshots are not copied, and lr_backward of dst is
 * unavailable (no state at step 0). Both contexts must have workspaces bound;
 * src is only read. LR_ERR_ARG when the contexts differ, LR_ERR_NOT_PD when a
 * source Gram matrix is singular. Sync. */
lr_status lr_grow_rank(lr_ctx* dst, const lr_ctx* src, uint64_t seed, double eps, void* stream);

/* Advance every trajectory by n_steps RK4 steps of size dt from the current
 * step counter (t = step * dt), recording beta at every step and the other
 * observables every pop_every steps, then recompute eps_a of every candidate
 * over [0, step*dt]. dt must not change within one pulse run. Async.
 *
 * CUDA graphs (FUSED engine): the call may be captured into a CUDA graph on
 * `stream` (it then issues three kernels: the persistent integrator, the
 * eps_a epilogue and a one-thread step advance, with no copy or host sync).
 * The step counter lives in device memory, so every replay of the graph
 * continues the pulse run by n_steps. A replay that would pass max_steps
 * runs nothing and leaves LR_ERR_STATE for the next synchronising call.
 * Capture does not execute, but it advances the host's copy of the counter:
 * call lr_sync after capturing, and after replays, to bring it back in line
 * with the device. The PLAIN engine refuses capture (LR_ERR_UNSUPPORTED). */
lr_status lr_integrate(lr_ctx* ctx, double dt, long n_steps, void* stream);

/* Copy recorded observables out (any pointer may be NULL to skip it; each
 * may be host or device memory). Layouts, per trajectory j = 0..n_traj-1:
 *   beta  [n_traj][max_steps+1][2]   (re, im) of tr(rho r) at t = n dt
 *   pops  [n_traj][n_rec][nt_max]    transmon level populations (zero padded)
 *   nphot [n_traj][n_rec]            tr(rho r^dag r)
 *   trace [n_traj][n_rec]            tr(rho)
 *   eps_a [n_cand]                   assignment error over [0, step dt]
 * Only entries up to the current step are meaningful. Synchronises the
 * stream and returns the device error word's status. */
lr_status lr_observables(lr_ctx* ctx, double* beta, double* pops, double* nphot,
                         double* trace, double* eps_a, void* stream);

/* Readout loss of Sec. S3.B for every candidate (host or device pointers,
 * either may be NULL), computed with eps_a at the end of lr_integrate:
 *   ionization[c] = T(tau) = (1/tau) sum_{j=g,e} sum_{k>=2} int P_k(t) dt,
 *     the transmon populations of levels k >= 2 integrated by the trapezoid
 *     rule over the recorded grid (every pop_every steps) up to the last
 *     record, tau = step * dt;
 *   loss[c] = log10(eps_a + T).
 * Synchronises the stream and returns the device error word's status. */
lr_status lr_loss(lr_ctx* ctx, double* ionization, double* loss, void* stream);

/* Assignment error from simulated single-shot readout records with seeded
 * Gaussian measurement noise (Sec. S3.A, measurement efficiency eta): the
 * Monte Carlo counterpart of eps_a, over the steps integrated so far.
 * For candidate c (trajectories 2c = |g>, 2c+1 = |e>, readout fields
 * beta_g, beta_e on the step grid, trapezoid weights w_k over steps 0..n) the
 * record is integrated in bins of bin_steps steps: q_b = sum_{k in b} w_k
 * (beta_e - beta_g)_k dt, W_b = sum_{k in b} w_k dt, and a shot of state j has
 * the increments dY_b = sqrt(2 eta kappa) sum_{k in b} w_k beta_j,k dt +
 * sqrt(W_b) xi_b, xi_b complex Gaussian with E|xi|^2 = 1. The matched filter
 * Re sum_b conj(q_b / W_b) dY_b against the midpoint of its two means gives
 * T_j = +-D/2 + N, D = sqrt(2 eta kappa) sum_b |q_b|^2 / W_b,
 * N = sum_b Re(conj(q_b) xi_b) / sqrt(W_b); shot j is misassigned when
 * T_e <= 0 or T_g > 0. Noise: xi_b = (n1 + i n2) / sqrt 2 from Box-Muller on
 * the uniforms u = ((x >> 11) + 1) 2^-53 of outputs 2b and 2b + 1 of the
 * SplitMix64 stream whose seed is output (2c + j) n_shots + s of the stream
 * of `seed` (shot s; the initial-state draws use the same generator).
 * Outputs (host, any may be NULL): eps_shots[c] = (misassigned g + e) /
 * (2 n_shots) + tau gamma / 2; eps_bin[c] = erfc(SNR_b / 2) / 2 + tau gamma / 2,
 * SNR_b^2 = 2 eta kappa sum_b |q_b|^2 / W_b, the value eps_shots converges to
 * (with bin_steps = 1 it is eps_a); errors[c][2] = misassigned g and e shots.
 * LR_ERR_ARG for n_shots outside 1 .. 65535 x 256, bin_steps < 1 or more than 2048 bins;
 * LR_ERR_STATE before the first step. Synchronises the stream. */
lr_status lr_assignment_shots(lr_ctx* ctx, double eta, long n_shots, int bin_steps, unsigned long long seed,
                              double* eps_shots, double* eps_bin, long long* errors, void* stream);

/* Validity diagnostics of the low-rank ansatz (Sec. S1.B, Fig. S1): at every
 * recorded step, the spectrum of rho = Z Z^dag and its purity tr(rho^2).
 * The nonzero eigenvalues of rho are those of the Gram matrix G = Z^dag Z
 * (same nonzero spectrum of A A^dag and A^dag A), and tr(rho^2) = tr(G^2) =
 * sum_ij |G_ij|^2. Needs lr_options.record_gram = 1; the Gram matrices are
 * the FP64 ones the engines form at the record steps (step 0, pop_every, ...).
 * Each (trajectory, record) is diagonalised on the device by cyclic Jacobi
 * rotations (FP64) of the real symmetric embedding [[Re G, -Im G],
 * [Im G, Re G]], whose eigenvalues are those of G, each twice.
 *   purity: host [n_traj][n_rec] doubles, tr(rho^2);
 *   eig:    host [n_traj][n_rec][max_M] doubles, eigenvalues p_1 >= ... >= p_M
 *           of trajectory j (entries beyond its rank M are 0);
 * records after the current step are 0. Either pointer may be NULL. p_M / p_1
 * is the paper's rank-saturation indicator. Synchronises `stream`. Errors:
 * LR_ERR_STATE without record_gram, LR_ERR_CUDA. */
lr_status lr_diagnostics(lr_ctx* ctx, double* purity, double* eig, void* stream);

/* Synchronise the stream, update the host's copy of the step counter from
 * the device (after CUDA graph replays) and return the device error word's
 * status. */
lr_status lr_sync(lr_ctx* ctx, void* stream);

/* Gradient of the assignment errors with respect to the pulse parameters,
 * by the discrete adjoint of the RK4 integration of Eq. S5 (reverse-mode
 * differentiation of Eq. S5, the readout signal beta = tr(rho r) and the
 * assignment error of Sec. S3.A). Differentiates the pulse run made since
 * lr_set_initial (or lr_set_state at step 0): the current step counter S and
 * dt are those of the run; tau stays fixed.
 *
 * d_eps_a (host, [n_cand]): cotangent dL/d eps_a of each candidate.
 * d_theta (host, [n_cand][8], out): dL/d theta; entries past the pulse kind's
 *   parameter count (4 for flat-top) are zero.
 * ckpt_every: states are kept every ckpt_every steps and each segment is
 *   recomputed; memory is (ceil(S/ckpt_every) + ckpt_every + 15) copies of all
 *   states (complex128, or complex64 for an FP32-bulk context) plus small
 *   tables, in the caller's workspace `dev_ws`
 *   (lr_backward_workspace_size bytes, 256-byte aligned).
 * Arithmetic follows the context's precision. FP64 context: FP64 throughout.
 * FP32-bulk context (FP32_G64, FP32, TF32_G64): the checkpoints, stage
 * inputs, cotangents and every per-element product in complex64 / FP32; the
 * Gram matrix summed from exact FP32 products in double-word FP32 (~2^-48,
 * FP64-class); the Cholesky factor, G^-1 and the M x M adjoint factors in
 * FP64; the readout signal and the gradient sums in FP64. The checkpoint
 * segments are recomputed with the PLAIN engine's kernels in that arithmetic
 * (the copies in the workspace are complex64 then: half the memory).
 * Synchronous; returns the device error status. */
lr_status lr_backward_workspace_size(const lr_ctx* ctx, int ckpt_every, size_t* bytes);
lr_status lr_backward(lr_ctx* ctx, void* dev_ws, size_t ws_bytes, const double* d_eps_a, double* d_theta,
                      int ckpt_every, void* stream);

lr_status lr_query(const lr_ctx* ctx, lr_info* info);

/* No-allocation entry point (the paper has no counterpart; this is a
 * deployment convenience).
 *
 * Some callers cannot allocate device memory at all: a plug-in running
 * inside a host application that has already reserved the GPU's memory and
 * forbids further cudaMalloc, code that runs while another library holds the
 * device in a fixed memory budget, or a thin binding with no device
 * allocator of its own. They cannot bind a workspace, so this call runs the
 * PLAIN FP64 engine for ONE trajectory with all of its scratch (stage
 * buffers, RK4 accumulator, partial sums, solved projections, small tables)
 * in a file-scope static device array of about 15.8 MB that every GPU which
 * loads the library keeps until the process exits. It calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *
 * Limits: N = N_t N_r [N_f] <= 4096, M <= 32, N*M <= 65536; larger sizes
 * return LR_ERR_UNSUPPORTED.
 *
 * Arguments: model and rank M as in lr_create; pulse and tau as in
 * lr_set_pulse; Z (device, in/out): the state, complex128 row-major [N][M]
 * as interleaved (re, im) doubles, advanced in place; beta (device, out):
 * n_steps+1 complex values, beta[k] = tr(rho r) at step step0 + k; dt, step0
 * (t = step * dt) and n_steps as in lr_integrate. The call is synchronous
 * and returns the device error status (LR_ERR_NOT_PD, LR_ERR_NONFINITE).
 * Results equal those of lr_integrate with the plain FP64 engine for the
 * same state.
 *
 * Every call made outside stream capture looks up the array's device
 * address (cudaGetSymbolAddress) with the current device, so a device reset
 * that moves the array is picked up by the next call; a call made during
 * capture reuses the address found by the last call outside capture. So the
 * first call on a device must come before any stream capture (a captured
 * first call returns LR_ERR_STATE). All calls share the one array, which keeps the
 * previous call's contents (everything a call reads is rewritten or cleared
 * by that call first); calls that overlap on the GPU (other streams, other
 * host threads) race on it and must be serialised by the caller. */
lr_status lr_integrate_plain_noalloc(const lr_model* model, int M, const lr_pulse* pulse, double tau,
                                     double* Z, double* beta, double dt, long step0, long n_steps,
                                     void* stream);
/* Arithmetic-pipe peak of the current device, measured (the paper has no
 * counterpart: these are the roofline denominators of the kernels above).
 *   kind 0: FP32 FMA (every thread runs 8 independent FFMA chains);
 *   kind 1: FP64 FMA (the same with DFMA);
 *   kind 2: TF32 tensor cores (one thread per CTA issues back-to-back
 *           tcgen05.mma.kind::tf32 128 x 256 x 8 into tensor memory).
 * Grids are a multiple of the SM count; one warm-up launch, then one timed
 * launch with CUDA events on `stream`. flops_per_s (host, out): counted flops
 * (an FMA is 2) per second; seconds (host, out, may be NULL): the timed
 * launch. Synchronous. Uses no workspace (a 4-byte static device word holds
 * the timeout flag). LR_ERR_ARG for an unknown kind, LR_ERR_TIMEOUT when the
 * tensor-core wait ran out of its budget. */
lr_status lr_measure_peak(int kind, double* flops_per_s, double* seconds, void* stream);

const char* lr_status_string(lr_status s);
const char* lr_last_error(const lr_ctx* ctx);
void lr_destroy(lr_ctx* ctx);


/* ======================================================================
 * The paper's own model (Sec. S2.A, S2.D, S2.E) on a sparse-operator engine.
 *
 * Basis |j_l> (x) |j_u> (x) |j_t>: the lower and upper normal modes of the
 * resonator-filter pair and the transmon eigenstates, flat index
 * n = (j_l N_u + j_u) N_t + j_t. The Hamiltonian is the one in the frame of
 * the drive with its counter-rotating e^{+-2i w_d t} terms (Eq.
 * S(hamiltonian_rotated)); the dissipators are kappa D[f] + gamma D[b] (Eq. 2)
 * in the same frame.
 *
 * Every operator X(t) is a sum of time channels,
 *     X(t) = sum_{a,q} Omega(t)^a e^{i q w_d t} X_{a,q},
 *     a in {0, 1}, q in {-2, ..., 2}, channel index 5 a + q + 2,
 * stored as CSR entries (row, column, complex value, channel). Omega(t) is the
 * real pulse envelope of Sec. S2.C (lr_pulse kinds 0 and 1; the pulse phase
 * must be 0 and its w_d must equal the model's).
 * ====================================================================== */

#define LR_SPARSE_MAX_JUMPS 3
#define LR_PAPER_DERIVED 16  /* length of lr_paper_model_build's `derived` output */

/* Physical parameters of the paper's model (Sec. S2.B), rad/ns and 1/ns. */
typedef struct {
  int Nl, Nu, Nt;       /* cutoffs: lower normal mode, upper normal mode, transmon (Nt <= LR_MAX_NT) */
  int n_cut;            /* charge basis |n| <= n_cut of the transmon diagonalisation (>= Nt, <= 64) */
  double Ec, Ej;        /* transmon charging and Josephson energies */
  double wr, wf;        /* bare resonator and filter frequencies */
  double g, J;          /* transmon-resonator and resonator-filter couplings */
  double kappa, gamma;  /* filter and transmon decay rates */
  double wd;            /* drive frequency = frame frequency */
  int frame;            /* 0: the Hamiltonian in the frame of the drive with its counter-rotating
                           e^{+-2i w_d t} terms, Eq. S(hamiltonian_rotated), and L_1(t), r(t) with
                           their e^{2i w_d t} parts; 1: the rotating-wave approximation,
                           Eq. S(hamiltonian_rwa): every explicitly time-dependent term dropped
                           (the channels q != 0 of H), and L_1 = sqrt(kappa) (s23 c_l + s24 c_u),
                           r = s23 c_l + s24 c_u (their slow parts), so that the generator is slow
                           and a larger dt can be used */
} lr_paper_params;

/* Operator set of the sparse engine. K = n_jumps; operator o occupies rows
 * rowptr[o (N+1)] .. rowptr[o (N+1) + N] of the entry arrays:
 *   o = 0        A(t) = -i H_eff(t) = -i H(t) - 1/2 sum_k L_k(t)^dag L_k(t),
 *   o = 1 .. K   the jump operators L_k(t),
 *   o = K + 1    the readout operator r(t), beta(t) = tr(rho r(t)) and the
 *                photon number tr(rho r^dag r).
 * Within a row the entries may come in any order; every row's entries of an
 * operator are contiguous. Arrays are host memory owned by the caller and read
 * only during lr_sparse_create. */
typedef struct {
  int N;                      /* Hilbert-space dimension (1 .. 2^24) */
  int n_jumps;                /* K, 1 .. LR_SPARSE_MAX_JUMPS */
  int n_levels;               /* population bins, 1 .. LR_MAX_NT */
  long nnz;                   /* entries of all operators */
  double wd;                  /* w_d of the time channels [rad/ns] */
  const int* rowptr;          /* [(K + 2) (N + 1)], non-decreasing within each operator, values in [0, nnz] */
  const int* col;             /* [nnz] column in [0, N) */
  const double* val;          /* [2 nnz] complex values (re, im) */
  const unsigned char* chan;  /* [nnz] channel 0 .. 9 */
  const int* level;           /* [N] population bin in [0, n_levels) of each basis state */
} lr_sparse_model;

typedef struct lr_sparse lr_sparse;

/* Sizes of the paper's model for `p`: N = Nl Nu Nt and the total entry count
 * of its four operators (A, L_1 = sqrt(kappa) f in the rotated frame,
 * L_2 = sqrt(gamma) b, r = f). LR_ERR_ARG for cutoffs out of range. Host only. */
lr_status lr_paper_model_size(const lr_paper_params* p, int* N, long* nnz);

/* Builds the operator set of the paper's model into caller-allocated host
 * arrays sized by lr_paper_model_size: rowptr [4 (N+1)], col [nnz],
 * val [2 nnz], chan [nnz], level [N] (the transmon index j_t). Steps:
 *  - transmon: 4 Ec n^2 - Ej cos(phi) in the charge basis (offset charge 0),
 *    cyclic Jacobi eigensolver, lowest Nt levels eps_j, charge matrix elements
 *    n_{j,j+1} > 0 (sign convention); only nearest neighbours are kept
 *    (the approximation of Sec. S2.E);
 *  - normal modes: w_l, w_u in closed form (momentum-coupled oscillators) and
 *    the null vectors of Omega - w (Sec. S2.D), normalised to
 *    alpha^2 + beta^2 - gamma^2 - delta^2 = 1 with beta > 0; then
 *    a = sum_i (alpha_i c_i - gamma_i c_i^dag), f = sum_i (beta_i c_i - delta_i c_i^dag);
 *  - A(t) from Eq. S(hamiltonian_rotated) and
 *    L_1(t) = sqrt(kappa) (s23 c_l + s24 c_u + e^{2i w_d t} (s21 c_u^dag + s22 c_l^dag)),
 *    L_2 = sqrt(gamma) sum_j sqrt(j) |j-1><j|, and the readout r(t) = L_1(t) / sqrt(kappa):
 *    the filter field of Fig. 2, beta_rot(t) = e^{i w_d t} tr(rho_lab f).
 * Products of truncated operators are truncated products (an intermediate
 * state outside the cutoffs contributes zero). Entries with the same row,
 * column and channel are merged; each row is sorted by (column, channel).
 * `derived` (optional, LR_PAPER_DERIVED doubles): w_l, w_u, mu_l, mu_u, nu_l,
 * nu_u, s21, s22, s23, s24, eps_1 - eps_0 (0 when Nt < 2),
 * eps_2 - 2 eps_1 + eps_0 (0 when Nt < 3), then zeros. Host only. */
lr_status lr_paper_model_build(const lr_paper_params* p, int* rowptr, int* col, double* val,
                               unsigned char* chan, int* level, double* derived);

/* Creates a sparse-engine context for n_traj trajectories of rank M
 * (1 <= M <= min(N, LR_MAX_RANK)) on one operator set; trajectory i uses
 * pulses[i]. Copies the operator arrays (they may be freed afterwards).
 * tau places the falling pulse edge; max_steps and pop_every size the
 * recorded observables as for lr_options. Per RK4 stage: an apply kernel
 * (A Z, L_k Z, r Z from the CSR rows, one thread per element of Z), a
 * row-block Gram kernel (Z^dag Z, Z^dag L_k Z and the observables), a
 * per-trajectory solve (Cholesky, X_k = G^-1 Z^dag L_k Z) and an update
 * kernel (F = A Z + 1/2 sum_k (L_k Z) X_k^dag, RK4).
 * precision: LR_PREC_FP64 (complex128 throughout) or LR_PREC_FP32_G64 (state,
 * apply, Z^dag L_k Z, projection term and RK4 in complex64; the Gram matrix
 * accumulated in FP64 from the exact products of the FP32 entries; Cholesky,
 * solves and observables in FP64); others give LR_ERR_UNSUPPORTED. */
lr_status lr_sparse_create(const lr_sparse_model* model, int n_traj, int M, lr_precision precision,
                           const lr_pulse* pulses, double tau, long max_steps, int pop_every, lr_sparse** out);
/* Bytes of device workspace the context needs (256-byte aligned). */
lr_status lr_sparse_workspace_size(const lr_sparse* s, size_t* bytes);
/* Binds a caller-owned device buffer (>= lr_sparse_workspace_size, 256-byte
 * aligned) and uploads the operators and pulses (sync on `stream`). */
lr_status lr_sparse_bind_workspace(lr_sparse* s, void* workspace, size_t bytes, void* stream);
/* Fixed-rank initial state of Sec. S1.A for every trajectory (same recipe and
 * random numbers as lr_set_initial), with the pure state |psi[i]> (a basis
 * index, e.g. |0_l, 0_u, g> = 0 and |0_l, 0_u, e> = 1); step counter reset. Async. */
lr_status lr_sparse_set_initial(lr_sparse* s, const int* psi, uint64_t seed, double eps, void* stream);
/* Host state [n_traj][N][M] complex128 (interleaved re, im) -> device;
 * step counter set to `step` (0 <= step <= max_steps). Sync. */
lr_status lr_sparse_set_state(lr_sparse* s, const double* Z, long step, void* stream);
/* Device state -> host [n_traj][N][M] complex128. Sync. */
lr_status lr_sparse_get_state(const lr_sparse* s, double* Z, void* stream);
/* n_steps RK4 steps of size dt [ns] from the current step; records beta at
 * every step and populations, photons and trace every pop_every steps.
 * LR_ERR_STATE past max_steps; LR_ERR_ARG for a dt other than the one the
 * pulse run has used so far. Async. */
lr_status lr_sparse_integrate(lr_sparse* s, double dt, long n_steps, void* stream);
/* Copies the records to host arrays (any may be NULL): beta [n_traj][max_steps+1]
 * complex128, pops [n_traj][n_rec][n_levels], nphot and trace [n_traj][n_rec]
 * (n_rec = max_steps / pop_every + 1). Syncs `stream` and returns the device
 * error status (LR_ERR_NOT_PD, LR_ERR_NONFINITE). */
lr_status lr_sparse_observables(lr_sparse* s, double* beta, double* pops, double* nphot, double* trace,
                                void* stream);
/* Assignment error and loss of Sec. S3.A / S3.B for candidate c = trajectories
 * (2c, 2c+1), started from |g> and |e>, over the steps integrated so far
 * (tau = step dt): SNR = sqrt(2 eta kappa int |beta_e - beta_g|^2 dt) (trapezoid
 * on the step grid), eps_a = erfc(SNR/2)/2 + tau gamma/2, the ionization penalty
 * T = (1/tau) sum_{g,e} sum_{k>=2} int P_k dt (trapezoid on the record grid, bins
 * k >= 2 of the population levels) and Lambda = log10(eps_a + T). kappa is the
 * decay rate of the read-out mode (the filter for the paper's model), gamma the
 * transmon's. Host outputs of n_traj / 2 doubles each (any may be NULL).
 * LR_ERR_ARG for an odd n_traj; LR_ERR_STATE before the first step. Sync. */
lr_status lr_sparse_loss(lr_sparse* s, double eta, double kappa, double gamma, double* eps_a, double* ion,
                         double* loss, void* stream);
/* Which integrator the context runs (host only): *fused = 1 for the fused
 * persistent kernel (FP32_G64 contexts by default: one launch per
 * lr_sparse_integrate; the stage input, the operator images and the RK4
 * accumulator in a per-team L2-resident region; the Gram matrix in
 * double-word FP32 and its LDL^dag factorisation, L^-1 and G^-1 in
 * double-word FP32), 0 for the four launches per RK4 stage described at
 * lr_sparse_create (FP64 contexts, or FP32_G64 with the environment variable
 * LR_SPARSE_FUSED=0 at lr_sparse_create). *team (may be NULL) = the CTAs
 * (one thread-block cluster) that share each trajectory's rows: 1 when the
 * batch has at least as many trajectories as the GPU has SMs (each CTA then
 * takes an equal span of the batch's trajectory-steps, unless
 * LR_SPARSE_SPLIT=0 at lr_sparse_integrate), else up to 16 (LR_SPARSE_C at
 * lr_sparse_create forces it); 0 for the four-launch path. *gram_tc (may be
 * NULL) = 1 when the fused kernel forms the Gram matrix on the tensor cores
 * (exact bf16 slices, double-word sums, FP64-class; LR_SPARSE_GRAM=tc at
 * lr_sparse_create, rank padded to 20), 0 for the double-word CUDA-core
 * sums (the default). */
lr_status lr_sparse_query(const lr_sparse* s, int* fused, int* team, int* gram_tc);
const char* lr_sparse_last_error(const lr_sparse* s);
void lr_sparse_destroy(lr_sparse* s);

/* ======================================================================
 * The full master equation on the device (FP64), the reference that the
 * low-rank runs of a model are compared with (Fig. 2) and timed against
 * (Table 1): the N x N density matrix under Eq. 2 / Eq. S4,
 *     d rho / dt = A rho + (A rho)^dag + sum_k L_k rho L_k^dag,
 * A = -i H_eff, for one trajectory of an operator set in the lr_sparse_model
 * layout (the paper's model from lr_paper_model_build, either frame), with the
 * classical RK4 scheme of the low-rank engines. Per RK4 stage: the operator
 * values at the stage time, B = A rho and Y_k = L_k rho (CSR row gathers, one
 * thread per element), B^dag and Y_k^dag (tiled transposes), and the update
 * F = B + B^dag + sum_k L_k Y_k^dag with the RK4 stage. Observables at the
 * start of every step: beta = tr(rho r(t)); at recording steps the level
 * populations, the photon number tr(r rho r^dag) and tr rho.
 * Memory: (5 + 2K) N^2 complex128 in the caller's workspace (576 MB at
 * N = 2000, K = 2), N <= 16384.
 * ====================================================================== */
typedef struct lr_full lr_full;
/* Context for one trajectory driven by `pulse` (kinds as lr_pulse, phase 0 and
 * w_d = model->wd as for lr_sparse_create); tau places the falling edge;
 * max_steps and pop_every size the records. Copies the operator arrays. Host only. */
lr_status lr_full_create(const lr_sparse_model* model, const lr_pulse* pulse, double tau, long max_steps,
                         int pop_every, lr_full** out);
lr_status lr_full_workspace_size(const lr_full* f, size_t* bytes);
/* Binds a caller-owned device buffer (>= lr_full_workspace_size, 256-byte
 * aligned) and uploads the operators (sync on `stream`). */
lr_status lr_full_bind_workspace(lr_full* f, void* workspace, size_t bytes, void* stream);
/* rho = |psi><psi| (a basis index), step counter reset. Async. */
lr_status lr_full_set_initial(lr_full* f, int psi, void* stream);
/* Host rho [N][N] complex128 (interleaved re, im) -> device; step counter set.
 * Only the upper triangle is read: rho is made exactly Hermitian from it (the
 * integrator keeps it so). Sync. */
lr_status lr_full_set_state(lr_full* f, const double* rho, long step, void* stream);
/* rho = Z Z^dag from a host low-rank factor Z [N][M] complex128 (e.g. the
 * initial state of a low-rank run, so that both start from the same rho);
 * step counter set. Sync. */
lr_status lr_full_set_state_lowrank(lr_full* f, const double* Z, int M, long step, void* stream);
/* Device rho -> host [N][N] complex128. Sync. */
lr_status lr_full_get_state(const lr_full* f, double* rho, void* stream);
/* n_steps RK4 steps of size dt from the current step, recording beta at every
 * step and the other observables every pop_every steps. LR_ERR_STATE past
 * max_steps; LR_ERR_ARG for a dt other than the run's. Async. */
lr_status lr_full_integrate(lr_full* f, double dt, long n_steps, void* stream);
/* Records to host or device arrays (any may be NULL): beta [max_steps+1]
 * complex128, pops [n_rec][n_levels], nphot and trace [n_rec]. Syncs and
 * returns the device error status (LR_ERR_NONFINITE). */
lr_status lr_full_observables(lr_full* f, double* beta, double* pops, double* nphot, double* trace, void* stream);
const char* lr_full_last_error(const lr_full* f);
void lr_full_destroy(lr_full* f);

#ifdef __cplusplus
}
#endif
#endif /* LR_H */
