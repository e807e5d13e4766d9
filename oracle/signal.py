"""Assignment error of the dispersive readout (oracle; test infrastructure).

Sec. S3.A of the paper:

    SNR(tau)     = sqrt(2 eta kappa int_0^tau |beta_e(t) - beta_g(t)|^2 dt)
    eps_sep(tau) = 1/2 erfc(SNR / 2)
    eps_decay    = tau gamma / 2
    eps_a        = eps_sep + eps_decay

kappa is the decay rate of the readout mode (Eq. 2), eta = 0.6. The time
integral is the composite trapezoid rule on the RK4 step grid (the paper's
adaptive solver output is not available; the readout signal is sampled at
every step t_n = n dt).

Parity: pinned by the constant-difference closed form
SNR = sqrt(2 eta kappa tau) |Delta| and by erfc(1) (tests).
"""
from __future__ import annotations

import math

import numpy as np


def integrated_separation(beta_g, beta_e, dt: float) -> float:
    d2 = np.abs(np.asarray(beta_e) - np.asarray(beta_g)) ** 2
    if d2.size < 2:
        return 0.0
    return float(dt * (0.5 * d2[0] + np.sum(d2[1:-1]) + 0.5 * d2[-1]))


def snr(beta_g, beta_e, dt: float, kappa: float, eta: float = 0.6) -> float:
    return math.sqrt(2.0 * eta * kappa * integrated_separation(beta_g, beta_e, dt))


def assignment_error(beta_g, beta_e, dt: float, kappa: float, gamma: float,
                     eta: float = 0.6) -> float:
    tau = (len(beta_g) - 1) * dt
    s = snr(beta_g, beta_e, dt, kappa, eta)
    return 0.5 * math.erfc(0.5 * s) + 0.5 * tau * gamma


def ionization(pops_g, pops_e, dt_rec: float, tau: float) -> float:
    """Ionization penalty of Sec. S3.B,
        T(tau) = (1/tau) sum_{j=g,e} sum_{k>=2} int_0^tau tr(|k_t><k_t| rho_j(t)) dt,
    with the transmon populations P_k(t) sampled every dt_rec (pops arrays
    [n_rec, N_t]) and the integral taken by the trapezoid rule over the
    recorded grid [0, (n_rec - 1) dt_rec]."""
    total = 0.0
    for p in (np.asarray(pops_g), np.asarray(pops_e)):
        hi = p[:, 2:].sum(axis=1) if p.shape[1] > 2 else np.zeros(p.shape[0])
        if hi.size >= 2:
            total += dt_rec * (0.5 * hi[0] + hi[1:-1].sum() + 0.5 * hi[-1])
    return total / tau


def loss(eps_a: float, T: float) -> float:
    """Loss of Sec. S3.B: Lambda = log10(eps_a + T)."""
    return math.log10(eps_a + T)
