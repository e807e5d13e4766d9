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


# FP32-bulk adjoint (an FP32 context): states, cotangents and per-element
# products carry FP32 rounding (u = 2^-24 = 6e-8 relative) that grows like a
# random walk over the S forward and S backward steps, ~sqrt(2 S) u; with
# S <= 1500 that is 3e-6, and the gradient, a sum over all stages, carries the
# same relative error. The finite differences at h = 1e-4 |theta_i| add
# O(h^2) truncation. Bound: 1e-4 of the largest gradient component.
FP32_GRAD_TOL = 1e-4


@pytest.mark.parametrize("make", [_flat_top_tiny, _two_segment_tiny])
def test_fp32_adjoint_matches_oracle_finite_differences(make):
    wl = make()
    n = wl.candidates[0].pulse.n_params
    fd = gradient.fd_gradient(wl, 0, rel=1e-4)[:n]
    _, g = _adjoint(wl, engine="fused", precision="fp32_g64")
    got = g[0, :n]
    assert np.all(g[0, n:] == 0.0)
    err = np.abs(got - fd) / np.abs(fd).max()
    print("fp32 adjoint vs oracle FD:", err)
    assert err.max() < FP32_GRAD_TOL
    assert math.isfinite(got.sum())


def test_fp32_adjoint_close_to_fp64_adjoint():
    wl = _two_segment_tiny(600)
    _, g64 = _adjoint(wl, engine="fused", precision="fp64")
    _, g32 = _adjoint(wl, engine="fused", precision="fp32_g64")
    err = np.abs(g32 - g64).max() / np.abs(g64).max()
    print("fp32 vs fp64 adjoint:", err)
    assert 0.0 < err < FP32_GRAD_TOL      # different arithmetic, the same gradient


@pytest.mark.parametrize("precision", ["fp64", "fp32_g64"])
def test_adjoint_dot_product(precision):
    """<J v, w> = <v, J^T w> for the Jacobian J = d eps_a / d theta of a batch
    of three candidates: J^T w from lr_backward with cotangent w, J v as the
    central difference of the GPU forward (FP64 fused engine) along a seeded
    direction v (scaled by |theta|). The FD error is O(h^2) = 1e-8 relative."""
    base = _two_segment_tiny(600)
    c0 = base.candidates[0]
    rng = np.random.default_rng(7)
    cands = []
    for k in range(3):
        th = np.array(c0.pulse.p) * (1.0 + 0.05 * k)
        cands.append(li.Candidate(c0.model, c0.M, li.PulseParams(1, tuple(th))))
    wl = li.Workload("tiny3x", cands, base.dt, base.n_steps, base.tau, init_seed=base.init_seed, eps=base.eps)
    w = rng.standard_normal(3)
    v = rng.standard_normal((3, 8)) * np.abs(np.array([c.pulse.p for c in cands]))
    b = runner.make_batch(wl, precision=precision, engine="fused")
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    jtw = b.backward(w, 200)
    b.close()
    h = 1e-4

    def eps_at(sign):
        cs = [li.Candidate(c.model, c.M, li.PulseParams(1, tuple(np.array(c.pulse.p) + sign * h * v[k])))
              for k, c in enumerate(cands)]
        wl2 = li.Workload("tiny3x", cs, wl.dt, wl.n_steps, wl.tau, init_seed=wl.init_seed, eps=wl.eps)
        bb = runner.make_batch(wl2, precision="fp64", engine="fused")
        bb.set_initial(wl2.init_seed, wl2.eps)
        bb.integrate(wl2.dt, wl2.n_steps)
        e = bb.observables()["eps_a"]
        bb.close()
        return e

    jv = (eps_at(1.0) - eps_at(-1.0)) / (2.0 * h)
    lhs = float(w @ jv)
    rhs = float(np.sum(v * jtw))
    # both sides are sums of terms of either sign: the error scale is the sum of
    # the magnitudes of the terms of <v, J^T w>
    scale = float(np.sum(np.abs(v * jtw)))
    print(precision, "dot test", lhs, rhs, "scale", scale)
    tol = 1e-6 if precision == "fp64" else FP32_GRAD_TOL
    assert abs(lhs - rhs) <= tol * scale


def _c5_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "c5_gradient.txt")
    if not os.path.exists(path):
        return None
    out = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            out[k] = [float(x) for x in v]
    return out


@pytest.mark.skipif(_c5_golden() is None, reason="c5 oracle gradient not generated")
def test_c5_adjoint_against_oracle_fd():
    """Transmon 10 x resonator 40 x filter 20 (N = 8000), M = 32, checkpoints
    every 200 steps, 400 RK4 steps of a pulse whose edges lie inside the window
    (tests/golden/c5_gradient.txt). Within 0.2 ns the g / e signals barely
    separate (eps_a = 0.5 - 8e-8 + tau gamma / 2): the gradient is ~1e-9 and the
    oracle's central differences (h = 1e-4 |theta_i|) carry an FP64 cancellation
    noise of ~1e-16 / h against eps_a ~ 0.5, up to a few percent of the smaller
    components; the FP64 adjoint must agree within that (5e-2 of the largest
    component). eps_a of both precisions' forwards against the oracle's."""
    import dataclasses
    g = _c5_golden()
    n, c = int(g["n_steps"][0]), int(g["candidate"][0])
    base = li.c5(n_candidates=c + 1, n_steps=n)
    assert abs(base.tau - g["tau"][0]) < 1e-12
    cand = dataclasses.replace(base.candidates[c], pulse=li.PulseParams(1, tuple(g["theta"])))
    wl = dataclasses.replace(base, candidates=[cand] * (c + 1))
    eps = {}
    for prec in ("fp64", "fp32_g64"):
        b = runner.make_batch(wl, precision=prec, engine="fused", max_steps=n, pop_every=n, candidates=[c])
        b.set_initial(wl.init_seed, wl.eps)
        b.integrate(wl.dt, n)
        eps[prec] = b.observables()["eps_a"][0]
        if prec == "fp64":
            grad = b.backward(np.ones(1), 200)[0]
        b.close()
    fd = np.array(g["grad"])
    err = np.abs(grad - fd).max() / np.abs(fd).max()
    print("c5 eps_a", eps, g["eps_a"][0], "fp64 adjoint", grad, "fd", fd, "err", err)
    assert abs(eps["fp64"] - g["eps_a"][0]) <= 1e-13
    assert abs(eps["fp32_g64"] - g["eps_a"][0]) <= 1e-9
    assert err < 5e-2


def test_c5_fp32_adjoint_against_fp64_adjoint():
    """The FP32-bulk adjoint against the FP64 adjoint at N = 8000, M = 32
    (checkpoints every 200 steps) over 2000 RK4 steps (1 ns) of a pulse with
    both edges and the switch inside the window. The gradient of eps_a is the
    difference of the |g> and |e> responses; where the signals have barely
    separated the two nearly cancel, and the FP32 rounding of each (~1e-6
    relative) is amplified by that cancellation (at 0.2 ns the FP32 gradient is
    off by ~30%). At 1 ns the separation is ~25 times larger; bound 5e-2 of the
    largest component."""
    import dataclasses
    n = 2000
    base = li.c5(n_candidates=1, n_steps=n)
    p = base.candidates[0].pulse.p
    theta = (li.TWO_PI * 0.3, li.TWO_PI * 0.2, 0.5, 0.02, 0.02, 0.02, p[6], p[7])
    cand = dataclasses.replace(base.candidates[0], pulse=li.PulseParams(1, theta))
    wl = dataclasses.replace(base, candidates=[cand])
    grads, eps = {}, {}
    for prec in ("fp64", "fp32_g64"):
        b = runner.make_batch(wl, precision=prec, engine="fused", max_steps=n, pop_every=n)
        b.set_initial(wl.init_seed, wl.eps)
        b.integrate(wl.dt, n)
        eps[prec] = b.observables()["eps_a"][0]
        grads[prec] = b.backward(np.ones(1), 200)[0]
        b.close()
    d = np.abs(grads["fp32_g64"] - grads["fp64"]).max() / np.abs(grads["fp64"]).max()
    print("c5 1 ns: eps_a", eps, "fp32", grads["fp32_g64"], "fp64", grads["fp64"], "rel", d)
    assert d < 5e-2
