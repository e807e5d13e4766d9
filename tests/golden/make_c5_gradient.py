#!/usr/bin/env python
"""Writes the FP64 oracle's finite-difference gradient for the adjoint test at
the differentiation workload's size.

Calls only the FP64 oracle (``oracle/``) and the seeded input recipes
(``lr_inputs``). Workload: transmon 10 x resonator 40 x filter 20 (N = 8000),
rank M = 32, a two-segment pulse whose edges and switch lie inside the
differentiated window (``workload()``), 400 RK4 steps of dt = 0.5 ps (tau =
0.2 ns), |g> and |e> (Eq. S5; the assignment error of Sec. S3.A). The
gradient is ``oracle.gradient.fd_gradient``: the central difference of eps_a
with respect to each of the 8 pulse parameters, step h_i = 1e-4 |theta_i|;
its 16 runs go to parallel worker processes.

Output: ``c5_gradient.txt`` (theta, eps_a, gradient).
Run from the repository root:  python tests/golden/make_c5_gradient.py
(about 6 minutes on 8 cores).
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

os.environ["OPENBLAS_NUM_THREADS"] = "1"
os.environ["OMP_NUM_THREADS"] = "1"

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))

N_STEPS = 400
CAND = 0
REL = 1e-4


def workload():
    """The N = 8000, M = 32 model of the differentiation workload with a pulse
    that is on within the differentiated window: the two-segment form with both
    edges and the switch inside the first 0.2 ns (candidate 0's drive frequency
    and phase), tau = 0.2 ns."""
    import dataclasses
    import lr_inputs as li
    base = li.c5(n_candidates=CAND + 1, n_steps=N_STEPS)
    c = base.candidates[CAND]
    p = c.pulse.p
    theta = (li.TWO_PI * 0.3, li.TWO_PI * 0.2, 0.1, 0.02, 0.02, 0.02, p[6], p[7])
    cand = dataclasses.replace(c, pulse=li.PulseParams(1, theta))
    return dataclasses.replace(base, candidates=[cand] * (CAND + 1))


def main():
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import gradient
    wl = workload()
    theta = np.array(wl.candidates[CAND].pulse.p, dtype=float)
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        grad = gradient.fd_gradient(wl, CAND, N_STEPS, rel=REL, pool_map=lambda f, xs: pool.map(f, xs, chunksize=1))
        eps = pool.map(gradient._eps_at, [(wl, CAND, N_STEPS, tuple(theta))])[0]
    with open(os.path.join(HERE, "c5_gradient.txt"), "w") as fh:
        fh.write("# FP64 oracle central-difference gradient of eps_a (oracle.gradient.fd_gradient), "
                 "written by tests/golden/make_c5_gradient.py\n")
        fh.write("# transmon 10 x resonator 40 x filter 20 (N=8000), M=32, trajectories 2c, 2c+1 = %d, %d, %d RK4 steps "
                 "of %g ns, tau %g ns, seed %d, eps %g, h_i = %g |theta_i|\n"
                 % (2 * CAND, 2 * CAND + 1, N_STEPS, wl.dt, wl.tau, wl.init_seed, wl.eps, REL))
        fh.write("n_steps %d\n" % N_STEPS)
        fh.write("candidate %d\n" % CAND)
        fh.write("tau %.17e\n" % wl.tau)
        fh.write("eps_a %.17e\n" % eps)
        fh.write("theta " + " ".join("%.17e" % x for x in theta) + "\n")
        fh.write("grad " + " ".join("%.17e" % x for x in grad) + "\n")
    print("wrote c5_gradient.txt", flush=True)


if __name__ == "__main__":
    main()
