"""SPSA pulse optimisation (oracle; test infrastructure only).

Sec. S3.C of the paper: simultaneous-perturbation stochastic approximation
(Spall 1992) over the pulse parameters; each epoch evaluates the loss at
theta + c_k Delta_k and theta - c_k Delta_k (two loss calls, each the |g>
and |e> trajectories) and steps along the finite-difference directional
derivative in the random direction Delta_k:

    g_k = (L(theta + c_k Delta) - L(theta - c_k Delta)) / (2 c_k) * Delta^-1,
    theta <- Proj(theta - a_k g_k),
    a_k = a / (k + 1 + A)^0.602,  c_k = c / (k + 1)^0.101,

with Delta_k in {-1, +1}^p (Spall's standard gain exponents). The
perturbations are inputs (drawn by the caller). Proj clips the amplitudes
to the bound |Omega| <= Omega_max of Sec. S3.B (2 pi 400 MHz) and keeps the
widths positive. Parameters are scaled per component by `scale` (the
perturbation is c_k * scale_i * Delta_i).
"""
from __future__ import annotations

import numpy as np

OMEGA_MAX = 2.0 * np.pi * 0.4


def project(kind: int, theta):
    th = np.array(theta, dtype=float)
    amps = [0] if kind == 0 else [0, 1]
    widths = [2] if kind == 0 else [3, 4, 5]
    for i in amps:
        th[i] = min(max(th[i], 0.0), OMEGA_MAX)
    for i in widths:
        th[i] = max(th[i], 0.05)
    return th


def gains(k: int, a: float, c: float, A: float):
    return a / (k + 1 + A) ** 0.602, c / (k + 1) ** 0.101


def spsa(loss_pair, kind, theta0, deltas, scale, a=0.1, c=0.1, A=10.0):
    """Run len(deltas) epochs; loss_pair(theta_plus, theta_minus) -> (L+, L-).
    Returns the parameter history [epochs + 1, p] and the loss pairs."""
    th = project(kind, theta0)
    hist, losses = [th.copy()], []
    scale = np.asarray(scale, dtype=float)
    for k, dl in enumerate(deltas):
        ak, ck = gains(k, a, c, A)
        dl = np.asarray(dl, dtype=float)
        tp = project(kind, th + ck * scale * dl)
        tm = project(kind, th - ck * scale * dl)
        lp, lm = loss_pair(tp, tm)
        g = (lp - lm) / (2.0 * ck) / dl
        th = project(kind, th - ak * scale * g)
        hist.append(th.copy())
        losses.append((lp, lm))
    return np.array(hist), losses
