"""torch.autograd.Function around the CUDA integrator and its adjoint.

``assignment_error(theta, batch, ...)`` returns eps_a of every candidate
(forward: lr_set_pulse, lr_set_initial, lr_integrate, lr_observables); its
backward calls lr_backward (discrete adjoint of the RK4 integration of
Eq. S5, checkpointed). theta is a float64 CPU tensor [n_cand, 8] (flat-top
pulses use the first 4 columns). Argument marshalling only: the arithmetic
runs in liblr.so.
"""
from __future__ import annotations

import numpy as np
import torch


class AssignmentError(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, batch, kinds, tau, dt, n_steps, seed, eps, ckpt_every):
        th = theta.detach().cpu().double().numpy()
        pulses = [(int(k), th[c, : (4 if int(k) == 0 else 8)]) for c, k in enumerate(kinds)]
        batch.set_pulse(pulses, tau)
        batch.set_initial(seed, eps)
        batch.integrate(dt, n_steps)
        out = batch.observables()
        ctx.batch = batch
        ctx.ckpt = ckpt_every
        ctx.kinds = list(kinds)
        return torch.from_numpy(np.array(out["eps_a"], dtype=np.float64))

    @staticmethod
    def backward(ctx, grad_eps):
        g = grad_eps.detach().cpu().double().numpy()
        dth = ctx.batch.backward(g, ctx.ckpt)
        return (torch.from_numpy(dth),) + (None,) * 8


def assignment_error(theta, batch, kinds, tau, dt, n_steps, seed, eps=1e-5, ckpt_every=200):
    return AssignmentError.apply(theta, batch, kinds, tau, dt, n_steps, seed, eps, ckpt_every)
