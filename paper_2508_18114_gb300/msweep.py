"""Rank sweep: one pulse candidate at several ranks M in one batched launch.

The paper judges the low-rank ansatz by how eps_a converges with M (Fig. S4:
the relative error of eps_a at tau = 40 ns falls from 5% at M = 20 to 1.5% at
M = 80) and by the rank-saturation indicator p_M / p_1 (Sec. S1.B). The
library integrates batches of uneven rank, so a sweep is a batch that holds
the same model and pulse once per rank: one launch integrates every rank,
lr_observables gives eps_a(M), and lr_diagnostics gives the spectrum of rho
at the record steps. At M = N the ansatz is the full master equation (up to
the RK4 discretisation of Z instead of rho).
"""
from __future__ import annotations

import numpy as np

from .lr import LowRankBatch


def rank_sweep(model, ranks, pulse, tau, dt, n_steps, seed, eps=1e-5, eta=0.6, precision="fp64",
               engine="auto", pop_every=None, device="cuda:0"):
    """Integrate `pulse` = (kind, params) on `model` at every rank in `ranks`.

    Returns a dict with, per rank: eps_a, beta [2, n_steps + 1] (g, e), the
    indicator p_M / p_1 and the purity tr(rho^2) of both trajectories at the
    last record step. Batch entry k uses initial-state trajectories 2k, 2k + 1
    of `seed`."""
    ranks = [int(m) for m in ranks]
    pe = pop_every or n_steps
    b = LowRankBatch([model] * len(ranks), ranks, precision=precision, engine=engine, max_steps=n_steps,
                     pop_every=pe, eta=eta, device=device, record_gram=True)
    try:
        b.set_pulse([pulse] * len(ranks), tau)
        b.set_initial(seed, eps)
        b.integrate(dt, n_steps)
        obs = b.observables()
        pur, eig = b.diagnostics()
    finally:
        b.close()
    last = n_steps // pe
    ratio = np.array([[eig[2 * k + lv, last, m - 1] / eig[2 * k + lv, last, 0] for lv in (0, 1)]
                      for k, m in enumerate(ranks)])
    return {"M": np.array(ranks), "eps_a": np.asarray(obs["eps_a"]),
            "beta": np.asarray(obs["beta"]).reshape(len(ranks), 2, -1),
            "pM_over_p1": ratio, "purity": pur[:, last].reshape(len(ranks), 2)}
