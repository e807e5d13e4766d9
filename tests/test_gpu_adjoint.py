"""Adjoint gradient of the assignment error with respect to the pulse
parameters (lr_backward / torch.autograd) against central finite differences
of the FP64 oracle and of the CUDA forward, plus structural checks."""
import math

import numpy as np
import pytest

import lr_inputs as li
from oracle import gradient
from paper_2508_18114_gb300 import autograd, runner

pytestmark = pytest.mark.gpu


def _flat_top_tiny(n_steps=1500, dt=2e-3):
    m = li.ModelParams(dims=(3, 6), wq=2.0, alpha=-0.4, wr=3.0, g=0.5, kappa=2.0, gamma=0.05)
    pul = li.PulseParams(0, (1.2, 3.05, 1.0, 0.3))
    return li.Workload("tiny", [li.Candidate(m, 3, pul)], dt, n_steps, n_steps * dt, init_seed=11, eps=1e-3)


def _two_segment_tiny(n_steps=1200, dt=2e-3):
    m = li.ModelParams(dims=(3, 4, 3), wq=2.0, alpha=-0.4, wr=3.0, g=0.5, kappa=1.5, gamma=0.05, wf=3.1, J=0.4)
    pul = li.PulseParams(1, (1.0, 0.6, 1.1, 0.5, 0.4, 0.3, 3.05, 0.7))
    return li.Workload("tiny3", [li.Candidate(m, 4, pul)], dt, n_steps, n_steps * dt, init_seed=12, eps=1e-3)


def _adjoint(wl, engine="plain", precision="fp64", ckpt=200, d_eps=1.0):
    b = runner.make_batch(wl, precision=precision, engine=engine)
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    eps_a = b.observables()["eps_a"]
    g = b.backward(np.full(len(wl.candidates), d_eps), ckpt)
    b.close()
    return eps_a, g


@pytest.mark.parametrize("make", [_flat_top_tiny, _two_segment_tiny])
def test_adjoint_matches_oracle_finite_differences(make):
    wl = make()
    n = wl.candidates[0].pulse.n_params
    fd = gradient.fd_gradient(wl, 0, rel=1e-4)[:n]
    _, g = _adjoint(wl)
    got = g[0, :n]
    assert np.all(g[0, n:] == 0.0)
    scale = np.abs(fd).max()
    err = np.abs(got - fd) / scale
    print("adjoint vs oracle FD:", got, fd, err)
    assert err.max() < 1e-5


def test_adjoint_independent_of_checkpoint_spacing():
    wl = _two_segment_tiny(400)
    _, g1 = _adjoint(wl, ckpt=7)
    _, g2 = _adjoint(wl, ckpt=400)
    assert np.array_equal(g1, g2)


def test_adjoint_linear_in_cotangent_and_engine_independent():
    wl = _flat_top_tiny(600)
    _, g1 = _adjoint(wl, d_eps=1.0)
    _, g2 = _adjoint(wl, d_eps=-2.0)   # a power of two scales every rounding exactly
    assert np.array_equal(g2, -2.0 * g1)
    e_f, gf = _adjoint(wl, engine="fused")
    assert np.allclose(gf, g1, rtol=1e-12, atol=1e-14 * np.abs(g1).max())


def test_autograd_function_matches_gpu_finite_differences():
    import torch
    wl = _two_segment_tiny(800)
    cand = wl.candidates[0]
    b = runner.make_batch(wl, engine="fused", precision="fp64")
    theta = torch.tensor([list(cand.pulse.p)], dtype=torch.float64, requires_grad=True)
    eps = autograd.assignment_error(theta, b, [1], wl.tau, wl.dt, wl.n_steps, wl.init_seed, wl.eps, 100)
    eps.sum().backward()
    grad = theta.grad.numpy()[0]
    fd = np.zeros(8)
    for i in range(8):
        h = 1e-4 * abs(cand.pulse.p[i])
        vals = []
        for sgn in (1, -1):
            th = theta.detach().clone()
            th[0, i] += sgn * h
            vals.append(float(autograd.assignment_error(th, b, [1], wl.tau, wl.dt, wl.n_steps, wl.init_seed,
                                                        wl.eps, 100)[0]))
        fd[i] = (vals[0] - vals[1]) / (2 * h)
    b.close()
    assert np.abs(grad - fd).max() / np.abs(fd).max() < 1e-5


def test_adjoint_of_fp32_context_is_fp64():
    wl = _flat_top_tiny(300)
    _, g64 = _adjoint(wl, engine="fused", precision="fp64")
    _, g32 = _adjoint(wl, engine="fused", precision="fp32_g64")
    # the FP32 context keeps its initial state in FP32: only that rounding differs
    assert np.allclose(g32, g64, rtol=1e-4, atol=1e-6 * np.abs(g64).max())
    assert math.isfinite(g32.sum())
