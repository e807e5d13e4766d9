"""Full Lindblad master equation (oracle; test infrastructure only).

Eq. 2 of the paper (Eq. S4 in the supplement):

    drho/dt = -i [H, rho] + sum_k D[L_k] rho,
    D[L] rho = L rho L^dag - 1/2 {L^dag L, rho},

with rho a dense N x N complex128 matrix, integrated with the same classical
RK4 as the low-rank oracle. Observables as in ``oracle.lowrank`` but read
off rho directly: beta = tr(rho r), P_j = sum of diag(rho) over transmon
level j, n_r = tr(rho r^dag r), trace = tr rho.

Parity: pinned by trace preservation, Hermiticity and positivity of rho, the
coherent-state closed form and exponential decay (tests).
"""
from __future__ import annotations

import numpy as np

from .lowrank import rk4_step


def _dag(x):
    return x.conj().T


def lindblad_rhs(rho: np.ndarray, t: float, model, coef) -> np.ndarray:
    c = coef(t)
    H_rho = model.apply_hamiltonian(c, rho)
    rho_H = _dag(model.apply_hamiltonian(c, _dag(rho)))
    out = -1j * (H_rho - rho_H)                        # -i [H, rho]
    for L, Ldag in zip(model.jumps, model.jumps_dag):
        L_rho = L @ rho
        out += _dag(L @ _dag(L_rho))                   # L rho L^dag
        LdL_rho = Ldag @ L_rho                         # L^dag L rho
        out -= 0.5 * (LdL_rho + _dag(LdL_rho))         # {L^dag L, rho}/2 (rho Hermitian)
    return out


def observables(rho: np.ndarray, model):
    beta = np.trace(model.r @ rho)
    nr = np.trace(model.n_r @ rho).real
    d = np.real(np.diag(rho))
    pops = np.bincount(model.level, weights=d, minlength=model.dims[0])
    return beta, pops, nr, float(np.sum(d))


def integrate(rho0, model, coef, dt, n_steps, pop_every=1, t0=0.0,
              return_state=False):
    rhs = lambda y, t: lindblad_rhs(y, t, model, coef)  # noqa: E731
    rho = np.array(rho0, dtype=complex)
    beta = np.zeros(n_steps + 1, dtype=complex)
    pops, nrs, traces = [], [], []
    for n in range(n_steps + 1):
        if n > 0:
            rho = rk4_step(rhs, rho, t0 + (n - 1) * dt, dt)
        if n % pop_every == 0:
            b, p, nr, tr = observables(rho, model)
            pops.append(p)
            nrs.append(nr)
            traces.append(tr)
            beta[n] = b
        else:
            beta[n] = np.trace(model.r @ rho)
    out = {"beta": beta, "pops": np.array(pops), "nr": np.array(nrs),
           "trace": np.array(traces)}
    if return_state:
        out["rho"] = rho
    return out
