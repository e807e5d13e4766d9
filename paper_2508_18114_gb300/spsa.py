"""SPSA outer loop over the CUDA integrator (Sec. S3.C of the paper).

Many independent SPSA chains run at once: every epoch evaluates, for each
chain, the loss Lambda = log10(eps_a + T) (Sec. S3.B, computed on the device
by lr_integrate / lr_loss) at theta + c_k Delta and theta - c_k Delta: two
candidates per chain in one batched launch. The update (host arithmetic on a
few parameters per chain) is

    g = (L+ - L-) / (2 c_k) / Delta,   theta <- Proj(theta - a_k g),
    a_k = a / (k + 1 + A)^0.602,  c_k = c / (k + 1)^0.101  (Spall 1992),

with perturbations Delta in {-1, +1}^p supplied by the caller, per-parameter
scales, amplitudes clipped to |Omega| <= 2 pi 400 MHz and widths kept
positive (Sec. S3.B/S3.C).
"""
from __future__ import annotations

import numpy as np

from .lr import LowRankBatch

OMEGA_MAX = 2.0 * np.pi * 0.4


def project(kind: int, theta: np.ndarray) -> np.ndarray:
    th = np.array(theta, dtype=float)
    amp = [0] if kind == 0 else [0, 1]
    wid = [2] if kind == 0 else [3, 4, 5]
    th[..., amp] = np.clip(th[..., amp], 0.0, OMEGA_MAX)
    th[..., wid] = np.maximum(th[..., wid], 0.05)
    return th


class SPSA:
    """n_chains SPSA chains on the same model (one batched launch per epoch)."""

    def __init__(self, model, M, kind, theta0, scale, tau, dt, seed, eps=1e-5, eta=0.6, precision="fp64",
                 engine="auto", pop_every=1, a=0.1, c=0.1, A=10.0, device="cuda:0"):
        self.kind = int(kind)
        self.theta = project(self.kind, np.atleast_2d(np.asarray(theta0, dtype=float)))
        self.n = self.theta.shape[0]
        self.p = 4 if self.kind == 0 else 8
        self.scale = np.asarray(scale, dtype=float)
        self.tau, self.dt, self.seed, self.eps = tau, dt, seed, eps
        self.n_steps = int(round(tau / dt))
        self.a, self.c, self.A = a, c, A
        self.k = 0
        self.batch = LowRankBatch([model] * (2 * self.n), [M] * (2 * self.n), precision=precision, engine=engine,
                                  max_steps=self.n_steps, pop_every=pop_every, eta=eta, device=device)

    def losses(self, thetas: np.ndarray) -> np.ndarray:
        """Device loss Lambda of each parameter row (one batched launch)."""
        b = self.batch
        rows = list(thetas)
        pulses = [(self.kind, r[: self.p]) for r in rows]
        if len(pulses) != len(b.models):
            raise ValueError("expected %d parameter rows" % len(b.models))
        b.set_pulse(pulses, self.tau)
        b.set_initial(self.seed, self.eps)
        b.integrate(self.dt, self.n_steps)
        return b.loss()[1]

    def step(self, delta: np.ndarray):
        """One epoch for every chain; delta [n_chains, p] with entries +-1."""
        ak = self.a / (self.k + 1 + self.A) ** 0.602
        ck = self.c / (self.k + 1) ** 0.101
        dl = np.asarray(delta, dtype=float).reshape(self.n, self.p)
        tp = project(self.kind, self.theta + ck * self.scale * dl)
        tm = project(self.kind, self.theta - ck * self.scale * dl)
        L = self.losses(np.concatenate([tp, tm], axis=0))
        lp, lm = L[: self.n], L[self.n:]
        g = ((lp - lm) / (2.0 * ck))[:, None] / dl
        self.theta = project(self.kind, self.theta - ak * self.scale * g)
        self.k += 1
        return lp, lm

    def close(self):
        self.batch.close()
