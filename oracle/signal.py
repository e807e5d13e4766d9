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

assignment_shots simulates the measurement behind that formula: seeded
single-shot heterodyne records of the readout mode, a matched filter and a
midpoint threshold; its misassignment rate converges to the formula's eps_sep
(binomial bound) and its binned SNR reduces to the trapezoid SNR for bins of
one step (tests).
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


def assignment_shots(beta_g, beta_e, dt: float, kappa: float, gamma: float, eta: float, n_shots: int,
                     bin_steps: int, seed: int, cand: int) -> dict:
    """Seeded single-shot readout of candidate `cand` (Sec. S3.A's measurement).

    Steps 0..n with trapezoid weights w_k (dt, halved at both ends), bins of
    bin_steps steps: q_b = sum_{k in b} w_k (beta_e - beta_g)_k, W_b = sum w_k.
    A shot of state j has record increments dY_b = sqrt(2 eta kappa) sum w_k
    beta_j,k + sqrt(W_b) xi_b (xi_b complex Gaussian, E|xi|^2 = 1); the matched
    filter Re sum_b conj(q_b / W_b) dY_b minus the midpoint of its two means is
    T_j = +-D/2 + N, D = sqrt(2 eta kappa) sum_b |q_b|^2 / W_b,
    N = sum_b Re(conj(q_b) xi_b) / sqrt(W_b). State e is misassigned when
    T_e <= 0, state g when T_g > 0.

    Noise: xi_b = (n1 + i n2) / sqrt(2), Box-Muller on the uniforms of outputs
    2b, 2b + 1 of the SplitMix64 stream seeded with output (2 cand + j) n_shots
    + s of the stream of `seed` (shot s), the generator of the initial states.
    Sums over steps and over bins are sequential, in FP64.
    Returns eps_shots, eps_bin = erfc(SNR_b / 2) / 2 + tau gamma / 2 with
    SNR_b^2 = 2 eta kappa sum_b |q_b|^2 / W_b, errors (g, e), D and the
    statistics T_g, T_e of every shot."""
    from .init_state import GOLDEN, mix64, splitmix64
    bg = np.asarray(beta_g, dtype=np.complex128)
    be = np.asarray(beta_e, dtype=np.complex128)
    n = len(bg) - 1
    if n < 1:
        raise ValueError("need at least one step")
    w = np.full(n + 1, float(dt))
    w[0] = w[n] = 0.5 * dt
    nb = (n + bin_steps) // bin_steps
    q = np.zeros(nb, np.complex128)
    W = np.zeros(nb)
    diff = be - bg
    for b in range(nb):
        k0, k1 = b * bin_steps, min((b + 1) * bin_steps, n + 1)
        qr = qi = wt = 0.0
        for k in range(k0, k1):                       # sequential, as the definition reads
            qr += w[k] * diff[k].real
            qi += w[k] * diff[k].imag
            wt += w[k]
        q[b] = complex(qr, qi)
        W[b] = wt
    s2 = float(np.sum(np.abs(q) ** 2 / W))
    D = math.sqrt(2.0 * eta * kappa) * s2
    snr_b = math.sqrt(2.0 * eta * kappa * s2)
    a = np.conj(q) / np.sqrt(W)
    k = np.arange(nb, dtype=np.uint64)
    out_T = []
    errors = []
    for j in (0, 1):
        keys = splitmix64(seed, np.uint64((2 * cand + j) * n_shots) + np.arange(n_shots, dtype=np.uint64))
        with np.errstate(over="ignore"):
            x1 = mix64(keys[:, None] + (2 * k[None, :] + np.uint64(1)) * GOLDEN)
            x2 = mix64(keys[:, None] + (2 * k[None, :] + np.uint64(2)) * GOLDEN)
        u1 = ((x1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = ((x2 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        r = np.sqrt(-2.0 * np.log(u1))
        n1, n2 = r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)
        terms = (a.real[None, :] * n1 - a.imag[None, :] * n2) / math.sqrt(2.0)
        N = np.cumsum(terms, axis=1)[:, -1]           # sequential over the bins
        T = (0.5 * D if j == 1 else -0.5 * D) + N
        out_T.append(T)
        errors.append(int(np.sum(T <= 0.0)) if j == 1 else int(np.sum(T > 0.0)))
    tau = n * dt
    dec = 0.5 * tau * gamma
    return {"eps_shots": (errors[0] + errors[1]) / (2.0 * n_shots) + dec,
            "eps_bin": 0.5 * math.erfc(0.5 * snr_b) + dec, "snr_bin": snr_b, "errors": tuple(errors), "D": D,
            "T_g": out_T[0], "T_e": out_T[1]}
