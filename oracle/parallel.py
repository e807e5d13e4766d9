"""Run oracle trajectories in parallel worker processes (test infrastructure).

Workers are started with the ``spawn`` method (safe next to a CUDA context)
and run single-threaded BLAS. Each task integrates one trajectory of one
candidate with ``oracle.lowrank``; the assignment error is formed in the
parent with ``oracle.signal``.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _traj_task(args):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from . import init_state, lowrank, pulse
    from .model import Model
    cand, traj, level, n_steps, pop_every, dt, tau, seed, eps, gram, frame = args
    p = cand.model
    if frame == "rwa":
        mdl = Model.from_params(p, rwa=pulse.drive_frequency_phase(cand.pulse.kind, cand.pulse.p))
        coef = pulse.rwa_coefficient(cand.pulse.kind, cand.pulse.p, tau)
    else:
        mdl = Model.from_params(p)
        coef = pulse.coefficient(cand.pulse.kind, cand.pulse.p, tau)
    psi = mdl.basis_index((level,) + (0,) * (len(p.dims) - 1))
    m0 = init_state.initial_state(mdl.N, cand.M, psi, eps, seed, traj)
    return lowrank.integrate(m0, mdl, coef, dt, n_steps, pop_every, gram=gram)


def _tasks(wl, n_steps, pop_every, candidates, traj_base, gram=False):
    idx = list(range(len(wl.candidates))) if candidates is None else list(candidates)
    ns = wl.n_steps if n_steps is None else n_steps
    tasks = []
    for k, ci in enumerate(idx):
        base = 2 * k if traj_base is None else traj_base[k]
        for lvl in (0, 1):
            tasks.append((wl.candidates[ci], base + lvl, lvl, ns, pop_every, wl.dt, wl.tau, wl.init_seed, wl.eps,
                          gram, getattr(wl, "frame", "lab")))
    return idx, tasks


def _collect(wl, idx, res):
    from . import signal
    out = {"beta": np.array([r["beta"] for r in res]),
           "pops": [r["pops"] for r in res], "nphot": [r["nr"] for r in res],
           "trace": [r["trace"] for r in res], "eps_a": []}
    if "gram" in res[0]:
        out["gram"] = [r["gram"] for r in res]
    for k, ci in enumerate(idx):
        p = wl.candidates[ci].model
        out["eps_a"].append(signal.assignment_error(res[2 * k]["beta"], res[2 * k + 1]["beta"],
                                                    wl.dt, p.kappa, p.gamma, wl.eta))
    out["eps_a"] = np.array(out["eps_a"])
    return out


class OracleJob:
    """Oracle run in a spawn pool, started now and collected with result().

    Trajectory 2k (|g>) and 2k+1 (|e>) of candidate position k use initial-state
    trajectory index traj_base[k] + level (default 2k), matching the CUDA batch
    built from the same candidate list.
    """

    def __init__(self, wl, n_steps=None, pop_every=1, candidates=None, processes=None, traj_base=None, gram=False):
        self.wl = wl
        self.idx, tasks = _tasks(wl, n_steps, pop_every, candidates, traj_base, gram)
        procs = processes or min(len(tasks), os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(procs)
        self.async_res = self.pool.map_async(_traj_task, tasks, chunksize=1)

    def result(self, timeout=None):
        try:
            res = self.async_res.get(timeout)
        finally:
            self.pool.close()
            self.pool.join()
        return _collect(self.wl, self.idx, res)


def run_workload(wl, n_steps=None, pop_every=1, candidates=None, processes=None, traj_base=None, gram=False):
    """Oracle observables for candidates of a workload (blocking); gram=True
    adds the Gram matrices at the record steps."""
    idx, tasks = _tasks(wl, n_steps, pop_every, candidates, traj_base, gram)
    procs = processes or min(len(tasks), os.cpu_count() or 1)
    if procs <= 1:
        res = [_traj_task(t) for t in tasks]
    else:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_traj_task, tasks, chunksize=1)
    return _collect(wl, idx, res)
