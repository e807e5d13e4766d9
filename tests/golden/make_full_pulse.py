#!/usr/bin/env python
"""Writes the full-pulse expected values of the readout workloads.

Calls only the FP64 oracle (``oracle/``) and the seeded input recipes
(``lr_inputs``); nothing here touches the CUDA library. Each trajectory is
integrated over the whole readout pulse (tau = 40 ns, dt = 0.5 ps, 80,000
RK4 steps), one process per trajectory:

* ``full_pulse_c4.txt``: the bare-mode three-mode model at N = 2000
  (transmon 10 x resonator 20 x filter 10), M = 20, candidates 0-2 of the
  seeded two-segment pulse population, |g> and |e> (Eq. S5, Sec. S3.A);
* ``full_pulse_paper.txt``: the paper's normal-mode model in the frame of the
  drive (Sec. S2, N = 100 x 4 x 5 = 2000, M = 20), candidate 0 of the seeded
  flat-top population, |g> and |e>.

Stored per trajectory: beta(t) = tr(rho r) every 100 steps, and the transmon
populations, readout photon number and tr rho every 1000 steps. Stored per
candidate: eps_a (Sec. S3.A, from beta at every step) and the ionization
penalty T (Sec. S3.B, from the populations every 1000 steps).

Run from the repository root:  python tests/golden/make_full_pulse.py
(about 25 minutes on 8 cores).
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

# one BLAS thread per worker process (set before numpy loads in each process)
os.environ["OPENBLAS_NUM_THREADS"] = "1"
os.environ["OMP_NUM_THREADS"] = "1"

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))

BETA_EVERY = 100
REC_EVERY = 1000
C4_CANDIDATES = (0, 1, 2)
PAPER_CANDIDATES = (0,)


def _task(args):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import lr_inputs as li
    from oracle import init_state, lowrank, pulse
    from oracle import paper_model as pm
    from oracle.model import Model
    kind, cand, level = args
    t0 = time.time()
    if kind == "c4":
        wl = li.c4(n_candidates=cand + 1)
        c = wl.candidates[cand]
        mdl = Model.from_params(c.model)
        coef = pulse.coefficient(c.pulse.kind, c.pulse.p, wl.tau)
        psi = mdl.basis_index((level, 0, 0))
        m0 = init_state.initial_state(mdl.N, c.M, psi, wl.eps, wl.init_seed, 2 * cand + level)
        out = lowrank.integrate(m0, mdl, coef, wl.dt, wl.n_steps, pop_every=REC_EVERY)
    else:
        wl = li.paper(cand + 1)
        mdl = pm.PaperModel(*wl.dims, frame="rot", **wl.params)
        pk, pp = wl.pulses[cand]
        env = lambda t: pulse.envelope(pk, pp, t, wl.tau)  # noqa: E731
        m0 = init_state.initial_state(mdl.N, wl.M, level, wl.eps, wl.init_seed, 2 * cand + level)
        n_steps = int(round(wl.tau / wl.dt))
        out = pm.integrate(m0, mdl, env, wl.dt, n_steps, pop_every=REC_EVERY, low_rank=True)
    out["seconds"] = time.time() - t0
    return (kind, cand, level), out


def _write(path, header, rows_by_key):
    with open(path, "w") as fh:
        for h in header:
            fh.write("# " + h + "\n")
        for key, lines in rows_by_key:
            fh.write("[%s]\n" % key)
            for ln in lines:
                fh.write(ln + "\n")


def _fmt(x):
    return "%.17e" % x


def main():
    sys.path.insert(0, ROOT)
    import lr_inputs as li
    from oracle import signal
    tasks = [("c4", c, lv) for c in C4_CANDIDATES for lv in (0, 1)]
    tasks += [("paper", c, lv) for c in PAPER_CANDIDATES for lv in (0, 1)]
    with mp.get_context("spawn").Pool(min(len(tasks), os.cpu_count() or 1)) as pool:
        res = dict(pool.map(_task, tasks, chunksize=1))
    for kind, cands in (("c4", C4_CANDIDATES), ("paper", PAPER_CANDIDATES)):
        if kind == "c4":
            wl = li.c4(n_candidates=max(cands) + 1)
            dt, tau, eta = wl.dt, wl.tau, wl.eta
            kap = [wl.candidates[c].model.kappa for c in cands]
            gam = [wl.candidates[c].model.gamma for c in cands]
            desc = ("bare-mode model 10x20x10 (N=2000), M=20, two-segment pulses, seed 1004, "
                    "eps 1e-5, lab frame")
        else:
            wl = li.paper(max(cands) + 1)
            dt, tau, eta = wl.dt, wl.tau, 0.6
            kap = [wl.params["kappa"]] * len(cands)
            gam = [wl.params["gamma"]] * len(cands)
            desc = ("paper's normal-mode model 100x4x5 (N=2000), M=20, flat-top pulses, seed 1008, "
                    "eps 1e-5, frame of the drive")
        n_steps = int(round(tau / dt))
        blocks = []
        for i, c in enumerate(cands):
            rg, re = res[(kind, c, 0)], res[(kind, c, 1)]
            eps_a = signal.assignment_error(rg["beta"], re["beta"], dt, kap[i], gam[i], eta)
            T = signal.ionization(rg["pops"], re["pops"], REC_EVERY * dt, tau)
            blocks.append(("candidate %d" % c, ["eps_a " + _fmt(eps_a), "T " + _fmt(T),
                                                "seconds %.1f %.1f" % (rg["seconds"], re["seconds"])]))
            for lv, r in ((0, rg), (1, re)):
                b = r["beta"][::BETA_EVERY]
                blocks.append(("beta %d %d" % (c, lv), ["%s %s" % (_fmt(z.real), _fmt(z.imag)) for z in b]))
                lines = []
                for k in range(r["pops"].shape[0]):
                    lines.append(" ".join(_fmt(x) for x in
                                          list(r["pops"][k]) + [r["nr"][k], r["trace"][k]]))
                blocks.append(("records %d %d" % (c, lv), lines))
        header = ["Full-pulse FP64 oracle values, written by tests/golden/make_full_pulse.py (oracle only).",
                  desc, "dt %g ns, %d RK4 steps, tau %g ns, eta %g" % (dt, n_steps, tau, eta),
                  "beta every %d steps: Re Im; records every %d steps: pops[0..N_t-1] nphot trace"
                  % (BETA_EVERY, REC_EVERY),
                  "candidates " + " ".join(str(c) for c in cands)]
        _write(os.path.join(HERE, "full_pulse_%s.txt" % kind), header, blocks)
        print("wrote", kind, flush=True)


if __name__ == "__main__":
    main()
