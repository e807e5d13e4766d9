"""Low-rank integrator (oracle; test infrastructure only).

Sec. S1.A of the paper. The density matrix is rho = m m^dag (Eq. S3) with m
an N x M complex matrix, evolved by the non-stochastic matrix Schroedinger
equation (Eq. S5)

    dm/dt = -i H m + O[m],
    O[m]  = 1/2 sum_k [ L_k m (m^+ L_k m)^dag - L_k^dag L_k m ],

where m^+ = (m^dag m)^{-1} m^dag is the Moore-Penrose inverse. The reading
that the 1/2 multiplies both terms is the only one for which
O m^dag + m O^dag equals sum_k D[L_k] m m^dag at M = N (tested).

The Gram matrix m^dag m is factorised by Cholesky (scipy); the integrator
is classical fixed-step RK4 (weights 1/6, 1/3, 1/3, 1/6, stage times
t, t + dt/2, t + dt/2, t + dt).

Observables (no renormalisation by tr rho):
  beta(t)   = tr(rho r) = tr(m^dag r m)        (Fig. 2 caption)
  P_j(t)    = sum over basis states with transmon level j of diag(rho)
  n_r(t)    = tr(m^dag r^dag r m)
  trace(t)  = tr(m^dag m)

Parity: pinned against the full master equation at M = N (Eq. S4), the
Schroedinger equation without jumps, the coherent-state closed form of a
driven damped resonator, exponential level decay, the trace-loss law of the
projected equation, gauge covariance and RK4's fourth-order convergence.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _dag(x):
    return x.conj().T


def nosse_rhs(m: np.ndarray, t: float, model, coef) -> np.ndarray:
    """Right-hand side of Eq. S5 at time t (coef(t) is the pulse coefficient)."""
    gram = _dag(m) @ m
    chol = sla.cho_factor(gram, lower=False)
    O = np.zeros_like(m)
    for L, Ldag in zip(model.jumps, model.jumps_dag):
        Lm = L @ m
        pinv_Lm = sla.cho_solve(chol, _dag(m) @ Lm)    # m^+ L_k m
        O += 0.5 * (Lm @ _dag(pinv_Lm) - Ldag @ Lm)
    return -1j * model.apply_hamiltonian(coef(t), m) + O


def rk4_step(rhs, y, t, dt):
    k1 = rhs(y, t)
    k2 = rhs(y + 0.5 * dt * k1, t + 0.5 * dt)
    k3 = rhs(y + 0.5 * dt * k2, t + 0.5 * dt)
    k4 = rhs(y + dt * k3, t + dt)
    return y + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def observables(m: np.ndarray, model):
    rm = model.r @ m
    beta = np.trace(_dag(m) @ rm)
    nr = np.vdot(rm, rm).real
    w = np.sum(np.abs(m) ** 2, axis=1)
    pops = np.bincount(model.level, weights=w, minlength=model.dims[0])
    trace = float(np.sum(w))
    return beta, pops, nr, trace


def integrate(m0, model, coef, dt, n_steps, pop_every=1, t0=0.0,
              return_state=False, gram=False):
    """RK4-integrate Eq. S5 for n_steps steps.

    Returns a dict with beta[n_steps+1] (complex), and pops[n_rec, N_t],
    nr[n_rec], trace[n_rec] at steps 0, pop_every, 2 pop_every, ...; with
    gram=True also gram[n_rec, M, M], the Gram matrix m^dag m at those steps.
    """
    rhs = lambda y, t: nosse_rhs(y, t, model, coef)  # noqa: E731
    m = np.array(m0, dtype=complex)
    beta = np.zeros(n_steps + 1, dtype=complex)
    pops, nrs, traces, grams = [], [], [], []
    for n in range(n_steps + 1):
        if n > 0:
            m = rk4_step(rhs, m, t0 + (n - 1) * dt, dt)
        if n % pop_every == 0:
            b, p, nr, tr = observables(m, model)
            pops.append(p)
            nrs.append(nr)
            traces.append(tr)
            if gram:
                grams.append(_dag(m) @ m)
            beta[n] = b
        else:
            beta[n] = np.trace(_dag(m) @ (model.r @ m))
    out = {"beta": beta, "pops": np.array(pops), "nr": np.array(nrs),
           "trace": np.array(traces)}
    if gram:
        out["gram"] = np.array(grams)
    if return_state:
        out["m"] = m
    return out
