#!/usr/bin/env python
"""Benchmark of the low-rank readout integrator on GB300.

Metric: trajectory-steps per second (one RK4 step of one trajectory) and
pulse evaluations per second (the |g> and |e> trajectories of one candidate
over the full pulse, tau / dt RK4 steps each, plus the assignment error).

One bench *step* integrates every trajectory of the batch for `--chunk` RK4
steps of the same pulse run (consecutive slices: warm-up slices first, then
the timed ones) and recomputes eps_a over the integrated interval, i.e. one
pass of the whole hot path. Inputs are seeded synthetic workloads
(lr_inputs) with the shapes of the paper's readout problem.

`--impl reference` times the FP64 CPU oracle on the same workload instead
(bounded samples, host cores).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP32 / FP64 CUDA-core peaks from unit counts: 152 SMs x 128 FP32 FMA/clk
# (2 flops each) and x 2 FP64 FMA/clk, at the sampled SM clock.
SMS = 152
FP32_FMA_PER_CLK = 128
FP64_FMA_PER_CLK = 2


# What each precision computes in (fused engine): the bulk state, operator
# apply, projections and RK4 in FP32; the Gram matrix as a double-word FP32
# sum of exact products, and the M x M factorisation, G^-1 and X_k = G^-1 T_k
# in double-word FP32 (all ~2^-48 relative, FP64-class); the readout signal
# and eps_a in FP64.
DTYPE_LABEL = {
    "fp64": "f64",
    "fp32_g64": "f32 bulk; double-word f32 (~2^-48) Gram, LDL^dag, G^-1 and X_k; f64 signal",
    "fp32": "f32 bulk and Gram; double-word f32 (~2^-48) LDL^dag, G^-1 and X_k; f64 signal",
    "tf32_g64": "f32 bulk, tf32 projection; double-word f32 (~2^-48) Gram, LDL^dag, G^-1 and X_k; f64 signal",
}
# DRAM bytes per trajectory-step of the tensor-core-Gram kernel, from its ncu capture on the
# 76-trajectory, 10-step case (0.578 GB read + 1.713 GB written for 760 trajectory-steps)
TRAFFIC_GRAM_TC = 3.015e6
# FP32_G64 with the Gram matrix on the tensor cores (the default plan of the N=2000, M=20 batch)
DTYPE_GRAM_TC = ("f32 bulk; FP64-class (~2^-48) Gram from exact bf16-slice tcgen05 MMAs (f32 accumulation, "
                 "exact) and double-word sums; double-word f32 LDL^dag, G^-1 and X_k; f64 signal")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--engine", default="auto")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--chunk", type=int, default=None, help="RK4 steps per bench step")
    ap.add_argument("--candidates", type=int, default=None, help="limit the number of candidates")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=None, help="RK4 steps of the oracle sample")
    ap.add_argument("--no-plain-baseline", action="store_true")
    ap.add_argument("--no-full-pulse", action="store_true", help="skip the full-pulse error check against the oracle")
    ap.add_argument("--plain-steps", type=int, default=8, help="RK4 steps timed on the plain FP64 engine")
    ap.add_argument("--no-graph", action="store_true", help="time direct lr_integrate calls instead of graph replays")
    ap.add_argument("--frame", default="lab", choices=["lab", "rwa"],
                    help="rwa: frame rotating at w_d with the rotating-wave approximation")
    ap.add_argument("--dt", type=float, default=None, help="RK4 step [ns] (default: the workload's; 2.5e-3 with rwa)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the gradient (lr_backward) of a pulse slice of --chunk steps instead")
    ap.add_argument("--ckpt", type=int, default=None, help="adjoint checkpoint spacing (default: --chunk)")
    return ap.parse_args()


def load_workload(args, rank=0):
    """The workload of one rank. Batch workloads (c3-c5) are candidate
    populations: rank r takes the next block of candidates of the same seeded
    population (weak scaling, no data-path collective); the single-candidate
    workloads are replicated."""
    import lr_inputs as li
    name = args.workload
    kw = {}
    if name in ("c3", "c4", "c5"):
        n = args.candidates if args.candidates is not None else li.workload(name).n_traj // 2
        kw["n_candidates"] = n
        kw["first"] = rank * n
    wl = li.workload(name, **kw)
    frame = getattr(args, "frame", "lab")
    dt = getattr(args, "dt", None) or (2.5e-3 if frame == "rwa" else None)
    if frame != "lab" or dt:
        import dataclasses
        dt = dt or wl.dt
        wl = dataclasses.replace(wl, name=wl.name + ("-" + frame if frame != "lab" else ""), frame=frame, dt=dt,
                                 n_steps=int(round(wl.tau / dt)))
    return wl


def aggregate(ms_local, units_local, dist=None):
    """Whole-job throughput: units of all ranks / slowest rank's time (max over
    ranks of the device-timed region)."""
    import torch
    ms, units = float(ms_local), float(units_local)
    if dist is not None:
        t = torch.tensor([ms, units], dtype=torch.float64)
        if dist.get_backend() == "nccl":
            t = t.cuda()
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        ms, units = float(mx[0]), float(sm[1])
    return units / (ms * 1e-3), ms, units


def workload_desc(wl, precision):
    c = wl.candidates
    Ns = sorted(set(x.model.N for x in c))
    Ms = sorted(set(x.M for x in c))
    dims = c[0].model.dims
    return {
        "workload": "%s: %d candidates x {g,e} = %d trajectories, N=%s (dims %s), M=%s, dt=%g ns, tau=%g ns, %s"
                    % (wl.name, len(c), 2 * len(c), Ns[0] if len(Ns) == 1 else "%d-%d" % (Ns[0], Ns[-1]),
                       "x".join(map(str, dims)) if len(Ns) == 1 else "uneven",
                       Ms[0] if len(Ms) == 1 else "%d-%d" % (Ms[0], Ms[-1]), wl.dt, wl.tau, precision),
        "trajectories": 2 * len(c),
        "N": Ns if len(Ns) > 1 else Ns[0],
        "M": Ms if len(Ms) > 1 else Ms[0],
        "dt_ns": wl.dt,
        "steps_per_pulse": int(round(wl.tau / wl.dt)),
    }


def flops_per_stage(N, M, K=2, nnz=11):
    """Algorithmic flops of one RK4 stage of one trajectory (complex MAC = 8):
    Gram upper triangle 4 N M^2, projections Z^dag L_k Z 8 K N M^2,
    projection term 8 K N M^2, operator apply ~ 4 nnz N M (real coefficients),
    RK4 update ~ 12 N M."""
    return 4 * N * M * M + 16 * K * N * M * M + 4 * nnz * N * M + 12 * N * M


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


def pipe_peak_measured(kind, stream):
    """FP32/FP64 FMA or TF32 MMA peak from the library's microbenchmark
    (lr_measure_peak), in TFLOP/s, or None."""
    try:
        from paper_2508_18114_gb300 import lr as lrmod
        f, _ = lrmod.measure_peak(kind, stream)
        return f / 1e12
    except Exception:
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return PEAKS_FALLBACK, "fallback"


# ----------------------------------------------------------------- oracle arm
def oracle_sample(wl, n_steps, candidates=(0,)):
    """Oracle traj-steps/s on a bounded sample: `n_steps` RK4 steps of the
    given candidates' g and e trajectories, one process per trajectory."""
    from oracle import parallel
    t0 = time.perf_counter()
    parallel.run_workload(wl, n_steps, max(1, n_steps), candidates=list(candidates),
                          processes=2 * len(candidates))
    dt = time.perf_counter() - t0
    ntraj = 2 * len(candidates)
    return ntraj * n_steps / dt, dt, ntraj


def full_pulse_error(wl, info, dev):
    """Errors of the timed launch plan over the whole pulse against the FP64
    oracle's full-pulse values (tests/golden/full_pulse_c4.txt, written by the
    oracle-only script beside it): the golden candidates of this workload run
    alone in the same plan (the per-trajectory arithmetic of a plan does not
    depend on the other trajectories of the launch) for all tau / dt steps."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from golden import full_pulse
    if not full_pulse.available("c4"):
        return None
    from paper_2508_18114_gb300 import LowRankBatch
    gold = full_pulse.load("c4")
    cands = sorted(gold["cands"])
    sub = [wl.candidates[c] for c in cands]
    saved = {k: os.environ.get(k) for k in ("LR_FUSED_C", "LR_FUSED_ZS", "LR_FUSED_TC", "LR_FUSED_GRAM")}
    os.environ.update({"LR_FUSED_C": str(info.team_size), "LR_FUSED_ZS": "smem" if info.stage_in_smem else "global",
                       "LR_FUSED_TC": str(info.tensor_passes), "LR_FUSED_GRAM": "tc" if info.gram_tc else "dw"})
    try:
        b = LowRankBatch([c.model for c in sub], [c.M for c in sub], precision="fp32_g64", engine="fused",
                         max_steps=wl.n_steps, pop_every=gold["rec_every"], eta=wl.eta, device=dev)
        q = b.query()
        b.set_pulse([(c.pulse.kind, c.pulse.p) for c in sub], wl.tau)
        b.set_initial(wl.init_seed, wl.eps)
        t0 = time.perf_counter()
        b.integrate(wl.dt, wl.n_steps)
        obs = b.observables()
        ion, _ = b.loss()
        sec = time.perf_counter() - t0
        b.close()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    obs["pop_every"] = gold["rec_every"]
    e = full_pulse.errors(gold, obs, cands, eps_a=obs["eps_a"], ion=ion)
    e.update({"sample": "candidates %s of this workload, g and e, all %d RK4 steps (tau = %g ns), plan: team %d, "
                        "stage state %s, tensor passes %d (%.1f s)"
                        % (cands, wl.n_steps, wl.tau, q.team_size, "shared memory" if q.stage_in_smem else "L2",
                           q.tensor_passes, sec),
              "eps_a": [float(x) for x in obs["eps_a"]],
              "eps_a_oracle": [gold["cands"][c]["eps_a"] for c in cands]})
    return e


def default_cpu_steps(wl):
    N = max(c.model.N for c in wl.candidates)
    M = max(c.M for c in wl.candidates)
    # ~1-2e-3 s per RK4 step at N=2000, M=20 on one core (numpy/scipy)
    return int(max(20, min(4000, 3e5 / (N * M / 40.0 + 50))))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "paper":
        return run_reference_paper(args)
    wl = load_workload(args)
    prec = args.precision or getattr(wl, "precision", "fp64")
    ns = args.cpu_steps or default_cpu_steps(wl)
    for _ in range(args.warmup):
        oracle_sample(wl, max(2, ns // 10))
    vals, tt = [], 0.0
    for _ in range(args.steps):
        v, dt, ntraj = oracle_sample(wl, ns)
        vals.append(v)
        tt += dt
    value = ntraj * ns * args.steps / tt
    desc = workload_desc(wl, prec)
    line = {
        "impl": "reference", "metric": "traj_steps_per_s", "value": value, "unit": "traj*steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(desc, parallelism="cpu oracle, one process per trajectory"),
        "pulse_evals_per_s": value / (2 * desc["steps_per_pulse"]),
        "cpu_baseline": {"value": value, "unit": "traj*steps/s", "cores": ntraj, "kind": "oracle",
                         "sample": "%d RK4 steps of the g and e trajectories of candidate 0 per step" % ns},
        "e2e": {"value": value, "unit": "traj*steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_reference_paper(args):
    import lr_inputs as li
    from oracle import paper_model as pm
    wl = li.paper(args.candidates if args.candidates is not None else 256)
    frame = "rwa" if args.frame == "rwa" else "rot"
    dt = args.dt or (2.5e-3 if frame == "rwa" else wl.dt)
    model_o = pm.PaperModel(*wl.dims, frame=frame, **wl.params)
    ns = args.cpu_steps or 400
    for _ in range(args.warmup):
        paper_oracle_sample(wl, model_o, max(2, ns // 10), dt=dt)
    tt = 0.0
    for _ in range(args.steps):
        tt += paper_oracle_sample(wl, model_o, ns, dt=dt)[1]
    value = ns * args.steps / tt
    line = {
        "impl": "reference", "metric": "traj_steps_per_s", "value": value, "unit": "traj*steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "paper: normal-mode model of Sec. S2 (%s), N=%d, M=%d, dt=%g ns"
                               % ("RWA, Eq. S(hamiltonian_rwa)" if frame == "rwa" else "frame of the drive",
                                  model_o.N, wl.M, dt), "parallelism": "cpu oracle, one trajectory"},
        "cpu_baseline": {"value": value, "unit": "traj*steps/s", "cores": 1, "kind": "oracle",
                         "sample": "%d RK4 steps of trajectory 0 per step" % ns},
        "e2e": {"value": value, "unit": "traj*steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2508_18114_gb300 import LowRankBatch
    from paper_2508_18114_gb300 import lr as lrmod

    wl = load_workload(args, rank)
    prec = args.precision or getattr(wl, "precision", "fp64")
    spp = int(round(wl.tau / wl.dt))
    # default slice: ~4 s of integration per bench step on this workload
    chunk = args.chunk or max(1, min(spp // 20, int(7e10 / sum(c.model.N * c.M * c.M for c in wl.candidates))))
    total_steps = chunk * (args.warmup + args.steps)
    if total_steps > spp:
        raise SystemExit("warmup + steps slices exceed one pulse (%d steps)" % spp)
    # weak scaling: every rank integrates the whole batch (independent replicas
    # of the candidate population, no data-path collective)
    cands = wl.candidates
    b = LowRankBatch([c.model for c in cands], [c.M for c in cands], precision=prec, engine=args.engine,
                     max_steps=spp, pop_every=max(1, chunk), eta=wl.eta, device=dev, frame=wl.frame)
    b.set_pulse([(c.pulse.kind, c.pulse.p) for c in cands], wl.tau)
    b.set_initial(wl.init_seed + 7919 * rank, wl.eps)   # replicas of single-candidate workloads differ by seed
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        b.integrate(wl.dt, chunk)
    b.sync()
    # the fused engine's integrate is timed as a captured CUDA graph, replayed
    # once per bench step (each replay continues the pulse run)
    graph = b.capture_integrate(wl.dt, chunk) if b.engine == "fused" and not args.no_graph else None
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()                       # L2 flush between timed iterations (not timed)
        ev[k][0].record(stream)
        if graph is not None:
            graph.replay()
        else:
            b.integrate(wl.dt, chunk)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    b.sync()
    ms_local = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    ntraj = b.n_traj
    value, ms, _ = aggregate(ms_local, ntraj * chunk * args.steps, dist)
    info = b.query()
    engine = lrmod.ENGINE_NAME[info.engine]

    # algorithmic work and roofline of the integrate kernel(s)
    # operator nonzeros per row: diagonal + g (4, or 2 with the RWA) [+ J (4 or 2)] + drive (2)
    nnz = lambda c: 1 + (2 if wl.frame == "rwa" else 4) * (2 if c.model.n_modes == 3 else 1) + 2  # noqa: E731
    fl = sum(2 * flops_per_stage(c.model.N, c.M, nnz=nnz(c)) for c in cands) * 4 * chunk   # per bench step
    peaks, peak_src = measured_peaks()
    mhz = clocks.get("sm_mhz") or 2070.0
    if prec == "fp64":
        peak = SMS * FP64_FMA_PER_CLK * 2 * mhz * 1e6 / 1e12
        pipe = "FP64 FMA"
    else:
        peak = SMS * FP32_FMA_PER_CLK * 2 * mhz * 1e6 / 1e12
        pipe = "FP32 FMA"
    achieved = fl / (ms * 1e-3 / args.steps) / 1e12
    # DRAM bytes per launch from one ncu capture of this kernel on a 76-trajectory, 10-step case
    # of the same workload, per trajectory-step at the same number of resident teams, scaled by
    # the trajectory-steps of one launch; only for the kernels those captures measured:
    # double-word Gram 0.338 GB read + 1.586 GB written for 760 trajectory-steps (2.532 MB),
    # tensor-core Gram 3.015 MB (TRAFFIC_GRAM_TC)
    # Those captures predate the 32-byte stage-state accesses of the current kernel, so the
    # line's traffic is null and the last capture's figure is reported beside it.
    traffic, traffic_last = None, None
    if (wl.name == "c4" and prec == "fp32_g64" and engine == "fused" and info.team_size == 2
            and not info.stage_in_smem and info.tensor_passes == 0):
        per = TRAFFIC_GRAM_TC if info.gram_tc else 2.532e6
        traffic_last = per * ntraj * chunk if per else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_last_capture": traffic_last,
                "kernel": "integrate (%s engine)" % engine,
                "peak_source": "%s pipe: 152 SMs x %d FMA/clk x 2 x %.0f MHz sampled SM clock (unit counts)"
                               % (pipe, FP64_FMA_PER_CLK if prec == "fp64" else FP32_FMA_PER_CLK, mhz),
                "flops_per_step": fl}
    pm = pipe_peak_measured("fp64_fma" if prec == "fp64" else "fp32_fma", stream)
    roofline["peak_measured"] = pm
    roofline["frac_of_measured"] = achieved / pm if pm else None
    roofline["peak_measured_source"] = ("lr_measure_peak: %s chains, 8 CTAs x 256 threads per SM, CUDA events, "
                                        "after the timed region" % ("DFMA" if prec == "fp64" else "FFMA"))
    # kernels per bench step: the integrator's (plain: 3 per RK4 stage pair and
    # records; fused: one persistent launch), the eps_a epilogue and the step advance
    if engine == "plain":
        launches = (12 * chunk + 2) + 2
    else:
        launches = 3
    launches *= args.steps

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        N0 = [int(np.prod(c.model.dims)) for c in cands]
        host_Z = [np.asarray(b.get_state(j)) for j in range(ntraj)]
        out = {"beta": np.empty((ntraj, spp + 1, 2)), "pops": np.empty((ntraj, info.n_rec, info.nt_max)),
               "nphot": np.empty((ntraj, info.n_rec)), "trace": np.empty((ntraj, info.n_rec)),
               "eps_a": np.empty(len(cands))}
        h2d = sum(z.nbytes for z in host_Z)
        d2h = sum(v.nbytes for v in out.values())
        step0 = info.step
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        reps = max(1, min(args.steps, 2))
        for r in range(reps):
            for j in range(ntraj):
                b.set_state(j, host_Z[j], step=step0)
            b.integrate(wl.dt, chunk)
            b.observables(out=out)
        te = time.perf_counter() - t0
        e2e = {"value": world * ntraj * chunk * reps / te, "unit": "traj*steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # plain FP64 engine (the reference GPU path) on the same batch
    plain = None
    if not args.no_plain_baseline and engine != "plain":
        bp = LowRankBatch([c.model for c in cands], [c.M for c in cands], precision="fp64", engine="plain",
                          max_steps=args.plain_steps + 1, pop_every=args.plain_steps, eta=wl.eta, device=dev,
                          frame=wl.frame)
        bp.set_pulse([(c.pulse.kind, c.pulse.p) for c in cands], wl.tau)
        bp.set_initial(wl.init_seed, wl.eps)
        bp.integrate(wl.dt, 1)
        bp.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bp.integrate(wl.dt, args.plain_steps)
        e1.record(stream)
        bp.sync()
        pms = e0.elapsed_time(e1)
        pv = world * bp.n_traj * args.plain_steps / (pms * 1e-3)
        plain = {"value": pv, "unit": "traj*steps/s", "engine": "plain", "dtype": "f64",
                 "steps_timed": args.plain_steps, "speedup": value / pv,
                 "workload": "the same batch on the plain FP64 kernels (three launches per stage, state in HBM)",
                 "accuracy": {"plain_fp64": "1e-10 relative against the FP64 oracle (parity tests)",
                              "this_line": "error_vs_oracle_full_pulse (FP32 bulk over the whole pulse)"}}
        bp.close()

    cpu = None
    err = None
    full = None
    if rank == 0 and not args.no_full_pulse and wl.name == "c4" and prec == "fp32_g64" and engine == "fused":
        full = full_pulse_error(wl, info, dev)
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import parallel
        ns = args.cpu_steps or default_cpu_steps(wl)
        t0 = time.perf_counter()
        ora = parallel.run_workload(wl, ns, max(1, ns), candidates=[0], processes=2)
        dt_cpu = time.perf_counter() - t0
        cpu = {"value": 2 * ns / dt_cpu, "unit": "traj*steps/s", "cores": 2, "kind": "oracle",
               "sample": "%d RK4 steps of the g and e trajectories of candidate 0 (%.1f s)" % (ns, dt_cpu)}
        # accuracy of this path on the same sample, against the FP64 oracle
        bq = LowRankBatch([cands[0].model], [cands[0].M], precision=prec, engine=args.engine, max_steps=ns,
                          pop_every=ns, eta=wl.eta, device=dev, frame=wl.frame)
        bq.set_pulse([(cands[0].pulse.kind, cands[0].pulse.p)], wl.tau)
        bq.set_initial(wl.init_seed, wl.eps)
        bq.integrate(wl.dt, ns)
        og = bq.observables()
        qinfo = bq.query()
        bq.close()
        bo = ora["beta"]
        err = {"sample": "candidate 0, g and e, %d RK4 steps (team %d, tensor passes %d, gram on tensor cores %d)"
                         % (ns, qinfo.team_size, qinfo.tensor_passes, qinfo.gram_tc),
               "beta_rel": float(np.abs(og["beta"] - bo).max() / np.abs(bo).max()),
               "pops_abs": float(max(np.abs(og["pops"][j][:, :ora["pops"][j].shape[1]] - ora["pops"][j]).max()
                                     for j in range(2))),
               "eps_a_rel": float(abs(og["eps_a"][0] - ora["eps_a"][0]) / abs(ora["eps_a"][0]))}

    if rank == 0:
        desc = workload_desc(wl, prec)
        desc.update({"parallelism": "dp%d (independent replicas)" % world, "engine": engine,
                     "team_size": info.team_size, "stage_state": "shared memory" if info.stage_in_smem else "L2",
                     "projection": ("tcgen05 TF32 x%d" % info.tensor_passes) if info.tensor_passes else "CUDA cores",
                     "gram": ("tcgen05 bf16 slices (exact), double-word sums" if info.gram_tc else
                              "double-word FP32 on the CUDA cores" if prec in ("fp32_g64", "tf32_g64") else prec),
                     "chunk_rk4_steps": chunk,
                     "launch": "CUDA graph replay" if graph is not None else "direct lr_integrate",
                     "l2": "flushed (256 MiB write) between timed steps"})
        line = {
            "metric": "traj_steps_per_s", "value": value, "unit": "traj*steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_GRAM_TC if info.gram_tc else DTYPE_LABEL[prec],
            "data": "synthetic (seeded pulses and initial states)", "config": desc,
            "pulse_evals_per_s": value / (2 * spp),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "peaks_source": peak_src,
            "plain_fp64_baseline": plain, "error_vs_oracle": err, "error_vs_oracle_full_pulse": full,
        }
        print(json.dumps(line))
    b.close()
    if dist:
        dist.destroy_process_group()


def run_adjoint(args):
    """Gradient evaluations: forward slice of `chunk` RK4 steps from step 0,
    then lr_backward (discrete adjoint, FP64) for dL/dtheta of every candidate.
    Metric: trajectory-steps of the differentiated slice per second of backward."""
    import numpy as np
    import torch
    from paper_2508_18114_gb300 import LowRankBatch, lr as lrmod
    wl = load_workload(args)
    prec = args.precision or getattr(wl, "precision", "fp64")
    chunk = args.chunk or 20
    cands = wl.candidates
    b = LowRankBatch([c.model for c in cands], [c.M for c in cands], precision=prec, engine=args.engine,
                     max_steps=chunk, pop_every=chunk, eta=wl.eta)
    b.set_pulse([(c.pulse.kind, c.pulse.p) for c in cands], wl.tau)
    times = []
    for k in range(args.warmup + args.steps):
        b.set_initial(wl.init_seed, wl.eps)
        b.integrate(wl.dt, chunk)
        b.sync()
        t0 = time.perf_counter()
        g = b.backward(np.ones(len(cands)), args.ckpt or chunk)
        torch.cuda.synchronize()
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    tt = sum(times)
    value = b.n_traj * chunk * args.steps / tt
    desc = workload_desc(wl, prec)
    ck = args.ckpt or chunk
    desc.update({"chunk_rk4_steps": chunk, "engine_forward": lrmod.ENGINE_NAME[b.query().engine],
                 "adjoint": "lr_backward, plain-kernel recomputation per checkpoint segment (%d steps), %s"
                            % (ck, "FP64" if prec == "fp64" else
                               "FP32 bulk with the Gram matrix summed from exact products in double-word FP32, FP64 "
                               "Cholesky/G^-1/solves, FP64 signal and gradient sums")})
    print(json.dumps({"metric": "adjoint_traj_steps_per_s", "value": value, "unit": "traj*steps/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
                      "higher_is_better": True, "dtype": "f64" if prec == "fp64" else "f32 bulk (f64 Gram/solves)",
                      "config": desc,
                      "grad_evals_per_s": value / (2 * desc["steps_per_pulse"]),
                      "grad_norm": float(np.abs(g).max())}))
    b.close()


# ------------------------------------------------- the paper's own model
def paper_flops_per_stage(model, M):
    """Algorithmic flops of one RK4 stage of one trajectory on the sparse engine
    (complex MAC = 8): one MAC per operator entry and column for A Z and L_k Z,
    the Gram upper triangle and Z^dag L_k Z per row, the projection term
    Y_k X_k^dag per element, the RK4 update ~ 12 N M."""
    N, K = model["N"], model["n_jumps"]
    rp = model["rowptr"]
    entries = sum(int(rp[o * (N + 1) + N] - rp[o * (N + 1)]) for o in range(K + 1))
    return 8 * entries * M + 8 * N * (M * (M + 1) // 2 + K * M * M) + 8 * K * N * M * M + 12 * N * M


def paper_oracle_sample(wl, model_o, n_steps, traj=0, dt=None):
    """FP64 oracle on one trajectory of the paper's model: (traj-steps/s, seconds, result)."""
    dt = dt or wl.dt
    from oracle import init_state
    from oracle import paper_model as pm
    from oracle import pulse as opulse
    kind, p = wl.pulses[traj // 2]
    env = lambda t: opulse.envelope(kind, p, t, wl.tau)  # noqa: E731
    m0 = init_state.initial_state(model_o.N, wl.M, traj % 2, wl.eps, wl.init_seed, traj)
    t0 = time.perf_counter()
    out = pm.integrate(m0, model_o, env, dt, n_steps, pop_every=n_steps, low_rank=True)
    sec = time.perf_counter() - t0
    return n_steps / sec, sec, out


def run_paper(args):
    """Sparse-operator engine on the paper's normal-mode model (FP64)."""
    import numpy as np
    import torch
    import lr_inputs as li
    from paper_2508_18114_gb300 import sparse

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.candidates if args.candidates is not None else 256
    wl = li.paper(n, first=rank * n)
    frame = "rwa" if args.frame == "rwa" else "rot"
    dt = args.dt or (2.5e-3 if frame == "rwa" else wl.dt)
    model = sparse.paper_model(*wl.dims, frame=frame, **wl.params)
    T = 2 * n
    pulses = [q for q in wl.pulses for _ in (0, 1)]
    spp = int(round(wl.tau / dt))
    chunk = args.chunk or 40
    total = chunk * (args.warmup + args.steps)
    prec = args.precision or "fp32_g64"
    b = sparse.SparseBatch(model, wl.M, pulses, wl.tau, spp, pop_every=chunk, device=dev, precision=prec)
    psi = [i % 2 for i in range(T)]
    b.set_initial(psi, wl.init_seed + 7919 * rank, wl.eps)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        b.integrate(dt, chunk)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kap, gam = wl.params["kappa"], wl.params["gamma"]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        b.integrate(dt, chunk)
        b.loss(kap, gam)                    # eps_a, T, Lambda over the run so far (syncs)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms_local = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    value, ms, _ = aggregate(ms_local, T * chunk * args.steps, dist)
    mhz = clocks.get("sm_mhz") or 2070.0
    fl = paper_flops_per_stage(model, wl.M) * 4 * chunk * T
    fma_clk = FP64_FMA_PER_CLK if prec == "fp64" else FP32_FMA_PER_CLK
    peak = SMS * fma_clk * 2 * mhz * 1e6 / 1e12
    achieved = fl / (ms * 1e-3 / args.steps) / 1e12
    team = b.team
    split = b.fused and team == 1 and T > torch.cuda.get_device_properties(dev).multi_processor_count \
        and os.environ.get("LR_SPARSE_SPLIT", "1") != "0"
    kname = (("sf_kernel (fused persistent sparse kernel, one launch per integrate; %s)"
              % ("equal spans of trajectory-steps per CTA" if split else "%d CTA(s) per trajectory" % team))
             if b.fused else "integrate (sparse engine, 4 launches per RK4 stage)")
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": kname,
                "peak_source": "%s FMA pipe: 152 SMs x %d FMA/clk x 2 x %.0f MHz sampled SM clock (unit counts)"
                               % ("FP64" if prec == "fp64" else "FP32", fma_clk, mhz), "flops_per_step": fl}
    pm = pipe_peak_measured("fp64_fma" if prec == "fp64" else "fp32_fma", stream)
    roofline["peak_measured"] = pm
    roofline["frac_of_measured"] = achieved / pm if pm else None
    # fused: one integrate launch and sp_loss per bench step; four-launch path: per RK4
    # step sp_chi + 4 x (apply, gram, solve, update), the closing observation pass
    # sp_chi, apply, gram, solve, then sp_loss
    launches = (2 if b.fused else 17 * chunk + 4 + 1) * args.steps

    e2e = None
    if not args.no_e2e:
        Zh = b.get_state()
        step0 = b.max_steps - chunk      # any slice inside the pulse run
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        reps = max(1, min(args.steps, 2))
        obs = None
        for _ in range(reps):
            b.set_state(Zh, step=step0)
            b.integrate(dt, chunk)
            obs = b.observables()
            obs.update(b.loss(kap, gam))
        te = time.perf_counter() - t0
        e2e = {"value": world * T * chunk * reps / te, "unit": "traj*steps/s", "h2d_bytes_per_step": int(Zh.nbytes),
               "d2h_bytes_per_step": int(sum(v.nbytes for v in obs.values()))}

    cpu = err = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import paper_model as pm
        model_o = pm.PaperModel(*wl.dims, frame=frame, **wl.params)
        ns = args.cpu_steps or 400
        v, dt_cpu, ora = paper_oracle_sample(wl, model_o, ns, traj=1, dt=dt)
        cpu = {"value": v, "unit": "traj*steps/s", "cores": 1, "kind": "oracle",
               "sample": "%d RK4 steps of trajectory 1 (candidate 0, |e>) (%.1f s)" % (ns, dt_cpu)}
        bq = sparse.SparseBatch(model, wl.M, pulses[:2], wl.tau, ns, pop_every=ns, device=dev, precision=prec)
        bq.set_initial([0, 1], wl.init_seed, wl.eps)
        bq.integrate(dt, ns)
        og = bq.observables()
        bo = ora["beta"]
        err = {"sample": "candidate 0, |e>, %d RK4 steps" % ns,
               "beta_rel": float(np.abs(og["beta"][1] - bo).max() / np.abs(bo).max()),
               "pops_abs": float(np.abs(og["pops"][1] - ora["pops"]).max())}
        del bq

    if rank == 0:
        line = {
            "metric": "traj_steps_per_s", "value": value, "unit": "traj*steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else (DTYPE_GRAM_TC if b.fused and b.gram_tc else
                                                   ("f32 bulk; double-word f32 (~2^-48) Gram, LDL^dag, G^-1 "
                                                    "and X_k; f64 signal") if b.fused else
                                                   "f32 bulk; double-word f32 (~2^-48) Gram; f64 Cholesky, "
                                                   "solves and signal"),
            "data": "synthetic (seeded flat-top pulses, seeded initial states)",
            "config": {"workload": "paper: %d candidates x {g,e} = %d trajectories, normal-mode model of Sec. S2 "
                                   "(%s), N=%d (%s), M=%d, dt=%g ns, tau=%g ns, %s"
                                   % (n, T, "rotating-wave approximation, Eq. S(hamiltonian_rwa)" if frame == "rwa"
                                      else "frame of the drive, counter-rotating terms kept", model["N"],
                                      "x".join(map(str, wl.dims)), wl.M, dt, wl.tau, prec),
                       "trajectories": T, "N": model["N"], "M": wl.M, "nnz": int(model["nnz"]),
                       "engine": "sparse (fused persistent kernel)" if b.fused else "sparse (four launches per stage)",
                       "gram": ("tcgen05 bf16 slices (exact), double-word sums" if b.fused and b.gram_tc else
                                "double-word FP32 on the CUDA cores" if prec != "fp64" else "f64"),
                       "schedule": (("equal spans of the batch's trajectory-steps, one per CTA" if split else
                                     "teams of %d CTA(s), one trajectory at a time" % team) if b.fused else None),
                       "chunk_rk4_steps": chunk,
                       "parallelism": "dp%d (independent replicas)" % world,
                       "l2": "flushed (256 MiB write) between timed steps"},
            "pulse_evals_per_s": value / (2 * spp),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "error_vs_oracle": err,
        }
        print(json.dumps(line))
    del b
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.workload == "paper" and args.impl != "reference":
        run_paper(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.adjoint:
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
