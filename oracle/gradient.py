"""Workload runner and finite-difference gradient (oracle; test infrastructure).

``run_candidate`` integrates one pulse candidate from |g> and from |e> with
the low-rank oracle (Eq. S5) and returns the readout signals, populations and
the assignment error (Sec. S3.A). Trajectory 2c is |g>, 2c+1 is |e>; the
initial state of trajectory j uses ``init_state.initial_state(..., traj=j)``.

``fd_gradient`` is the central finite difference of the assignment error with
respect to the pulse parameters, step h_i = rel * |theta_i| (rel = 1e-4).
"""
from __future__ import annotations

import numpy as np

from . import init_state, lowrank, pulse, signal
from .model import Model


def run_candidate(wl, cand_index: int, n_steps=None, pop_every=1, theta=None,
                  model=None):
    cand = wl.candidates[cand_index]
    p = cand.model
    mdl = model if model is not None else Model.from_params(p)
    n_steps = wl.n_steps if n_steps is None else n_steps
    tau = wl.tau
    th = cand.pulse.p if theta is None else tuple(theta)
    coef = pulse.coefficient(cand.pulse.kind, th, tau)
    res = {}
    for lvl, tag in ((0, "g"), (1, "e")):
        traj = 2 * cand_index + lvl
        psi_index = mdl.basis_index((lvl,) + (0,) * (len(p.dims) - 1))
        m0 = init_state.initial_state(mdl.N, cand.M, psi_index, wl.eps,
                                      wl.init_seed, traj)
        res[tag] = lowrank.integrate(m0, mdl, coef, wl.dt, n_steps, pop_every)
    res["eps_a"] = signal.assignment_error(res["g"]["beta"], res["e"]["beta"],
                                           wl.dt, p.kappa, p.gamma, wl.eta)
    return res


def _eps_at(args):
    wl, cand_index, n_steps, theta = args
    return run_candidate(wl, cand_index, n_steps, theta=theta)["eps_a"]


def fd_gradient(wl, cand_index: int, n_steps=None, rel=1e-4, pool_map=None):
    """Central differences (eps_a(theta + h_i e_i) - eps_a(theta - h_i e_i)) / (2 h_i).
    pool_map (optional, e.g. a process pool's map) evaluates the 2 n runs; by
    default they run here, one after the other."""
    cand = wl.candidates[cand_index]
    theta = np.array(cand.pulse.p, dtype=float)
    grad = np.zeros_like(theta)
    hs, points = [], []
    for i in range(theta.size):
        h = rel * abs(theta[i]) if theta[i] != 0.0 else rel
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        hs.append(h)
        points += [tp, tm]
    if pool_map is None:
        mdl = Model.from_params(cand.model)
        vals = [run_candidate(wl, cand_index, n_steps, theta=t, model=mdl)["eps_a"] for t in points]
    else:
        vals = list(pool_map(_eps_at, [(wl, cand_index, n_steps, tuple(t)) for t in points]))
    for i in range(theta.size):
        grad[i] = (vals[2 * i] - vals[2 * i + 1]) / (2.0 * hs[i])
    return grad
