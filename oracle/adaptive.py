"""Adaptive rank control (oracle; test infrastructure only).

The same scheme as the library's controller, on the FP64 oracle integrator:
segments of `segment` RK4 steps; after each, the spectrum of rho = m m^dag
(the eigenvalues of the Gram matrix m^dag m, Sec. S1.B); a candidate whose
p_M / p_1 (larger of its g and e trajectories) exceeds `tol` gains `d_rank`
columns up to `max_rank`:

    m -> [m, sqrt(eps) q_1, ..., sqrt(eps) q_dM],

q_j the orthonormalisation of complex Gaussian vectors (the generator of the
fixed-rank initial condition, pair index (j-1) N + n, trajectory seed = output
`traj` of the growth seed) against span(m) and each other, here by two
Householder QRs (numpy), equal to the library's Gram-Schmidt up to a phase per
column (rho does not see it).

At a growth step the observables recorded are those of the grown state (the
run continues from it).

Parity: pinned by orthogonality of the new columns to span(m), rho gaining
exactly eps Q Q^dag, and the unchanged old columns (tests).
"""
from __future__ import annotations

import numpy as np

from . import init_state, lowrank


def grow(m: np.ndarray, M_new: int, eps: float, seed: int, traj: int) -> np.ndarray:
    N, Ms = m.shape
    if M_new <= Ms:
        return m.copy()
    xi = init_state.gaussian_columns(init_state.trajectory_seed(seed, traj), N, M_new - Ms)
    q0, _ = np.linalg.qr(m)
    q, _ = np.linalg.qr(np.column_stack([q0, xi]))
    return np.column_stack([m, np.sqrt(eps) * q[:, Ms:]])


def ratio(m: np.ndarray) -> float:
    """p_M / p_1 of rho = m m^dag (eigenvalues of m^dag m)."""
    p = np.linalg.eigvalsh(m.conj().T @ m)
    return float(p[0] / p[-1])


def adaptive_run(model_pairs, coefs, dt, n_steps, rank0, max_rank, d_rank, tol, segment, m0s,
                 eps, grow_seed=1):
    """model_pairs[c] = oracle Model of candidate c; coefs[c] its pulse coefficient;
    m0s[2c], m0s[2c+1] the initial states of its g and e trajectories (rank rank0).
    Returns (beta per trajectory [n_steps+1], pops per trajectory at the segment
    ends (with step 0), history as the library's)."""
    n = len(model_pairs)
    ms = [np.array(x, dtype=complex) for x in m0s]
    ranks = [int(rank0)] * n
    betas = [[] for _ in ms]
    pops = [[] for _ in ms]
    history, done, grows = [], 0, 0
    for tj, m in enumerate(ms):
        b, p, _, _ = lowrank.observables(m, model_pairs[tj // 2])
        betas[tj].append(b)
        pops[tj].append(p)
    while done < n_steps:
        k = min(segment, n_steps - done)
        for tj in range(len(ms)):
            c = tj // 2
            out = lowrank.integrate(ms[tj], model_pairs[c], coefs[c], dt, k, pop_every=k, t0=done * dt,
                                    return_state=True)
            ms[tj] = out["m"]
            betas[tj].extend(out["beta"][1:])
            pops[tj].append(out["pops"][-1])
        done += k
        if done % segment:
            break
        rat = np.array([max(ratio(ms[2 * c]), ratio(ms[2 * c + 1])) for c in range(n)])
        new = [min(max_rank, r + d_rank) if (q > tol and r < max_rank) else r for r, q in zip(ranks, rat)]
        history.append({"step": done, "ratio": rat, "ranks": list(new)})
        if new != ranks and done < n_steps:
            for tj in range(len(ms)):
                ms[tj] = grow(ms[tj], new[tj // 2], eps, grow_seed + grows, tj)
                # the run continues from the grown state: its observables are the ones
                # recorded at this step
                b, p, _, _ = lowrank.observables(ms[tj], model_pairs[tj // 2])
                betas[tj][-1] = b
                pops[tj][-1] = p
            grows += 1
            ranks = new
    return [np.array(b) for b in betas], [np.array(p) for p in pops], history
