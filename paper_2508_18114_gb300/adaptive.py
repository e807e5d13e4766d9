"""Adaptive rank control (Sec. S1.B; the paper points to adaptive low-rank
schemes as the alternative to checking convergence in M by hand).

The run is split into segments of `segment` RK4 steps. After each segment the
spectrum p_1 >= ... >= p_M of rho = Z Z^dag comes from lr_diagnostics, and a
candidate whose ratio p_M / p_1 (the larger of its |g> and |e> trajectories)
exceeds `tol` gets `d_rank` more columns, up to `max_rank`, through
lr_grow_rank: the state keeps its columns and gains orthonormal padding columns
of weight `eps`, as the fixed-rank initial condition pads a pure state. The
continuing run records the observables of the grown state at the growth step.
Every step runs in the library's kernels; this module only orchestrates the
calls.
"""
from __future__ import annotations

import numpy as np

from .lr import LowRankBatch


def adaptive_run(models, pulses, tau: float, dt: float, n_steps: int, rank0: int, max_rank: int,
                 d_rank: int = 2, tol: float = 1e-3, segment: int = 100, seed: int = 0, eps: float = 1e-5,
                 grow_seed: int = 1, precision: str = "fp64", engine: str = "auto", device="cuda:0",
                 frame: str = "lab"):
    """Integrate n_steps with rank control. Returns (batch, history): the final
    LowRankBatch (its records cover the whole run) and, per segment end, the
    step, the ratios p_M/p_1 per candidate and the ranks after the decision.
    The k-th growth draws its padding columns from seed grow_seed + k."""
    n = len(models)
    ranks = [int(rank0)] * n
    b = LowRankBatch(models, ranks, precision=precision, engine=engine, max_steps=n_steps, pop_every=segment,
                     record_gram=True, device=device, frame=frame)
    b.set_pulse(pulses, tau)
    b.set_initial(seed, eps)
    history, done, grows = [], 0, 0
    while done < n_steps:
        k = min(segment, n_steps - done)
        b.integrate(dt, k)
        done += k
        if done % segment:
            break                                  # no record at a partial segment's end
        _, eig = b.diagnostics()
        rec = done // segment
        ratio = np.zeros(n)
        for c in range(n):
            M = ranks[c]
            for tj in (2 * c, 2 * c + 1):
                p = eig[tj, rec, :M]
                ratio[c] = max(ratio[c], p[M - 1] / p[0])
        new = [min(max_rank, r + d_rank) if (q > tol and r < max_rank) else r for r, q in zip(ranks, ratio)]
        history.append({"step": done, "ratio": ratio.copy(), "ranks": list(new)})
        if new != ranks and done < n_steps:
            b = b.grown(new, grow_seed + grows, eps)
            grows += 1
            ranks = new
    return b, history
