"""Rank sweep (the M-convergence method of Fig. S4) against the oracle.

Each rank of the batch is checked against the oracle's low-rank run at that
rank (FP64, 1e-10). At M = N the low-rank result is the master equation: its
eps_a must match the oracle's full master equation from the same rho(0) to
within the RK4 gap between integrating Z and integrating rho (pinned on the
CPU to shrink 16x per halving of dt; below 1e-4 relative here).
"""

import numpy as np
import pytest

import lr_inputs as li
from oracle import init_state, lindblad, lowrank, pulse, signal
from oracle.model import Model
from paper_2508_18114_gb300 import msweep

pytestmark = pytest.mark.gpu


def test_rank_sweep_matches_oracle_and_master_equation():
    p = li.ModelParams(dims=(2, 4, 3), wq=li.TWO_PI * 6.0, alpha=-li.TWO_PI * 0.3, wr=li.TWO_PI * 7.5,
                       g=li.TWO_PI * 0.15, kappa=li.TWO_PI * 0.05, gamma=1.0 / 50.0, wf=li.TWO_PI * 7.51,
                       J=li.TWO_PI * 0.1)
    pl = li.pulse_two_segment(77, li.TWO_PI * 7.5)
    N, ranks, dt, n, tau, seed, eps = p.N, [1, 3, 8, p.N], 1e-3, 2000, 2.0, 5, 1e-3
    out = msweep.rank_sweep(p, ranks, (pl.kind, pl.p), tau, dt, n, seed, eps=eps, precision="fp64",
                            engine="plain", pop_every=500)
    mdl = Model.from_params(p)
    coef = pulse.coefficient(pl.kind, pl.p, tau)
    for k, m in enumerate(ranks):
        betas = []
        for lv in (0, 1):
            psi = mdl.basis_index((lv, 0, 0))
            z0 = init_state.initial_state(N, m, psi, eps, seed, 2 * k + lv)
            ora = lowrank.integrate(z0, mdl, coef, dt, n, pop_every=500)
            scale = np.abs(ora["beta"]).max()
            assert np.abs(out["beta"][k, lv] - ora["beta"]).max() <= 1e-10 * scale
            betas.append(ora["beta"])
            if m == N:   # the master equation from the same rho(0)
                me = lindblad.integrate(z0 @ z0.conj().T, mdl, coef, dt, n, pop_every=500)
                assert np.abs(me["beta"] - ora["beta"]).max() <= 1e-4 * scale
                betas[-1] = me["beta"]
        want = signal.assignment_error(betas[0], betas[1], dt, p.kappa, p.gamma)
        rel = abs(out["eps_a"][k] - want) / want
        print("M=%d eps_a %.6e rel %.2e pM/p1 %s" % (m, out["eps_a"][k], rel, out["pM_over_p1"][k]))
        assert rel <= (1e-4 if m == N else 1e-10)
    # rank 1 is a pure state (purity 1 up to the trace loss of the projection)
    assert np.all(out["pM_over_p1"][0] == 1.0)
