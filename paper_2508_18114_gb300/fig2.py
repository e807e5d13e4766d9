"""The readout of Fig. 2 and the timing of Table 1 on this GPU: the paper's
normal-mode model (Sec. S2, N = N_l N_u N_t = 100 x 4 x 5 = 2000) driven by the
square pulse of the paper's figure (|Omega_d| / 2 pi = 150 MHz, logistic edges
with sigma = 0.5 ns, tau = 40 ns), from |g> and |e>, integrated

* by the full master equation (lr_full_*, FP64, the N x N density matrix), and
* by the low-rank ansatz of rank M (lr_sparse_*, FP64 on the four-launch
  path, and FP32 bulk with the FP64-class Gram matrix on the fused kernel),
* each also with the RWA of Eq. S(hamiltonian_rwa) at its longer step (the RWA
  columns of Table 1),

with RK4 at dt = 0.5 ps, both from the same initial density matrix (the
low-rank initial state of Sec. S1.A, rho(0) = Z(0) Z(0)^dag). Output (JSON): the readout signals beta_g(t), beta_e(t)
and photon numbers n(t) of both methods every `--every` steps, the relative
deviation delta = |y_full - y| / |y_full| of beta and n of every other run
from the full master equation in the frame of the drive, the assignment error
of each method (Sec. S3.A), and the wall time of each run (the low-rank runs
with g and e in one batch, and each alone).

    python -m paper_2508_18114_gb300.fig2 --out fig2.json [--steps 80000]

Argument marshalling and bookkeeping only: every step runs in liblr.so.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

TWO_PI = 2.0 * math.pi


def paper_params():
    """Sec. S2.B (rad/ns, 1/ns)."""
    Ec = TWO_PI * 0.315
    return dict(Ec=Ec, Ej=51.0 * Ec, wr=TWO_PI * 7.2, wf=TWO_PI * 7.21, g=TWO_PI * 0.15, J=TWO_PI * 0.03,
                kappa=TWO_PI * 0.03, gamma=TWO_PI * 8e-6, wd=TWO_PI * 7.18)


def assignment_error(beta_g, beta_e, dt, kappa, gamma, eta=0.6):
    """Sec. S3.A: SNR = sqrt(2 eta kappa int |beta_e - beta_g|^2), trapezoid on the step grid."""
    d2 = np.abs(np.asarray(beta_e) - np.asarray(beta_g)) ** 2
    s = dt * (0.5 * d2[0] + d2[1:-1].sum() + 0.5 * d2[-1])
    snr = math.sqrt(2.0 * eta * kappa * s)
    return 0.5 * math.erfc(0.5 * snr) + 0.5 * (len(d2) - 1) * dt * gamma


def _deviation(full, lra, every_full, every_lra):
    """delta = |y_full - y_LRA| / |y_full| of beta and n at the common record
    times where |y_full| is at least 1% of its maximum (before the drive has
    filled the mode both are ~0 and the ratio says nothing), at the end of the
    pulse, and max |y_full - y_LRA| / max |y_full|."""
    bf = np.asarray(full["beta"])[::every_full]
    bl = np.asarray(lra["beta"])[::every_lra]
    nf, nl = np.asarray(full["nphot"]), np.asarray(lra["nphot"])
    k = min(len(bf), len(bl))
    kn = min(len(nf), len(nl))
    bf, bl, nf, nl = bf[:k], bl[:k], nf[:kn], nl[:kn]
    mb = np.abs(bf) >= 0.01 * np.abs(bf).max()
    mn = np.abs(nf) >= 0.01 * np.abs(nf).max()
    return {"delta_beta_max": float(np.max(np.abs(bf - bl)[mb] / np.abs(bf)[mb])),
            "delta_beta_end": float(abs(bf[-1] - bl[-1]) / abs(bf[-1])),
            "delta_n_max": float(np.max(np.abs(nf - nl)[mn] / np.abs(nf)[mn])),
            "delta_n_end": float(abs(nf[-1] - nl[-1]) / abs(nf[-1])),
            "beta_abs_dev_over_max": float(np.abs(bf - bl).max() / np.abs(bf).max()),
            "n_abs_dev_over_max": float(np.abs(nf - nl).max() / np.abs(nf).max())}


def run(steps=80000, dt=5e-4, M=20, every=100, amp_mhz=150.0, dims=(100, 4, 5), eps=1e-5, seed=1008,
        fp32=True, rwa_dt=2.5e-3, rwa=True, device="cuda:0"):
    import torch
    from . import sparse
    P = paper_params()
    tau = steps * dt
    pulse = (0, [TWO_PI * amp_mhz * 1e-3, P["wd"], 2.5, 0.0])
    frames = [("rot", dt)] + ([("rwa", rwa_dt)] if rwa else [])
    out = {"model": "paper's normal-mode model, %s (N=%d), frame of the drive" % ("x".join(map(str, dims)),
                                                                                  int(np.prod(dims))),
           "pulse": "flat-top %.0f MHz, sigma 0.5 ns, tau %.3g ns" % (amp_mhz, tau),
           "dt_ns": dt, "steps": steps, "M": M, "every": every, "runs": {}}
    if rwa:
        out["rwa"] = {"dt_ns": rwa_dt, "steps": int(round(tau / rwa_dt)),
                      "model": "Eq. S(hamiltonian_rwa): the counter-rotating channels dropped"}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    curves = {}
    results = {}
    for frame, h in frames:
        model = sparse.paper_model(*dims, frame=frame, **P)
        n = int(round(tau / h))
        ev = max(1, int(round(every * dt / h)))
        sfx = "" if frame == "rot" else "_rwa"
        # the low-rank initial states (Sec. S1.A: |g> or |e> plus padding of weight
        # eps); the full master equation starts from the same rho(0) = Z(0) Z(0)^dag,
        # so that the deviation is the rank truncation alone
        b0 = sparse.SparseBatch(model, M, [pulse, pulse], tau, 1, precision="fp64", device=device)
        b0.set_initial([0, 1], seed, eps)
        z0 = b0.get_state()
        del b0
        full = {}
        for lv, tag in ((0, "g"), (1, "e")):
            f = sparse.FullME(model, pulse, tau, n, pop_every=ev, device=device)
            f.set_state_lowrank(z0[lv])
            _, sec = timed(lambda: f.integrate(h, n))
            full[tag] = dict(f.observables(), seconds=sec)
            del f
        out["runs"]["full_fp64" + sfx] = {
            "seconds_per_trajectory": [full["g"]["seconds"], full["e"]["seconds"]],
            "eps_a": assignment_error(full["g"]["beta"], full["e"]["beta"], h, P["kappa"], P["gamma"])}
        results["full" + sfx] = (full, ev)
        precs = ["fp64"] + (["fp32_g64"] if fp32 else [])
        for prec in precs:
            runs = {}
            # g and e together (one batch), and each alone (the single-trajectory time of Table 1)
            for name, lvs in (("together", [0, 1]), ("g", [0]), ("e", [1])) if prec != "fp64" else (("together", [0, 1]),):
                b = sparse.SparseBatch(model, M, [pulse] * len(lvs), tau, n, pop_every=ev, precision=prec,
                                       device=device)
                b.set_initial(lvs, seed, eps)
                _, sec = timed(lambda: b.integrate(h, n))
                runs[name] = (b.observables(), sec, b.team if b.fused else 0)
                del b
            o, sec, team = runs["together"]
            key = "lra_%s%s" % (prec, sfx)
            out["runs"][key] = {
                "engine": ("fused, %d CTA(s) per trajectory" % team) if team else "four launches per stage",
                "seconds_g_and_e_together": sec,
                "seconds_per_trajectory_alone": [runs["g"][1], runs["e"][1]] if "g" in runs else None,
                "eps_a": assignment_error(o["beta"][0], o["beta"][1], h, P["kappa"], P["gamma"])}
            results[key] = (o, ev)
    # deviations from the full master equation of the frame of the drive (Fig. 2)
    full, evf = results["full"]
    ef = out["runs"]["full_fp64"]["eps_a"]
    for key, (res, ev) in results.items():
        if key == "full":
            continue
        r = out["runs"][key if not key.startswith("full") else "full_fp64_rwa"]
        r["eps_a_rel_dev"] = abs(r["eps_a"] - ef) / ef
        dev = {}
        for j, tag in ((0, "g"), (1, "e")):
            other = res[tag] if key.startswith("full") else {"beta": res["beta"][j], "nphot": res["nphot"][j]}
            dev[tag] = _deviation(full[tag], other, evf, ev)
        r["deviation_from_full"] = dev
    curves["t_ns"] = (np.arange(0, steps + 1, every) * dt).tolist()
    for key, (res, ev) in results.items():
        for j, tag in ((0, "g"), (1, "e")):
            o = res[tag] if key.startswith("full") else {"beta": res["beta"][j], "nphot": res["nphot"][j]}
            curves["%s_beta_%s" % (key, tag)] = [[float(z.real), float(z.imag)] for z in np.asarray(o["beta"])[::ev]]
            curves["%s_n_%s" % (key, tag)] = np.asarray(o["nphot"]).tolist()
    out["curves"] = curves
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--steps", type=int, default=80000)
    ap.add_argument("--dt", type=float, default=5e-4)
    ap.add_argument("--M", type=int, default=20)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-rwa", action="store_true", help="skip the RWA runs (Table 1's RWA columns)")
    ap.add_argument("--rwa-dt", type=float, default=2.5e-3)
    a = ap.parse_args()
    res = run(steps=a.steps, dt=a.dt, M=a.M, every=a.every, fp32=not a.no_fp32, rwa=not a.no_rwa, rwa_dt=a.rwa_dt)
    with open(a.out, "w") as fh:
        json.dump(res, fh)
    summary = {k: v for k, v in res.items() if k != "curves"}
    print(json.dumps(summary, indent=1))


if __name__ == "__main__":
    main()
