"""Readout loss (Sec. S3.B) and the SPSA outer loop (Sec. S3.C) on the GPU
against the FP64 oracle."""
import numpy as np
import pytest

import lr_inputs as li
from oracle import gradient, signal, spsa as ospsa
from paper_2508_18114_gb300 import runner, spsa

pytestmark = pytest.mark.gpu


def _model():
    return li.ModelParams(dims=(5, 4, 3), wq=2.0, alpha=-0.4, wr=3.0, g=0.5, kappa=1.5, gamma=0.05, wf=3.1, J=0.4)


def test_loss_matches_oracle():
    m = _model()
    cands = [li.Candidate(m, 4, li.PulseParams(1, (0.9, 0.5, 1.0, 0.5, 0.4, 0.3, 3.05, 0.7))),
             li.Candidate(m, 6, li.PulseParams(1, (1.3, 0.2, 0.8, 0.3, 0.6, 0.2, 2.95, 1.9)))]
    wl = li.Workload("loss", cands, 2e-3, 1000, 2.0, init_seed=21, eps=1e-3)
    pe = 10
    for engine in ("plain", "fused"):
        b = runner.make_batch(wl, precision="fp64", engine=engine, pop_every=pe)
        b.set_initial(wl.init_seed, wl.eps)
        b.integrate(wl.dt, wl.n_steps)
        ion, loss = b.loss()
        b.close()
        for k in range(2):
            r = gradient.run_candidate(wl, k, pop_every=pe)
            T = signal.ionization(r["g"]["pops"], r["e"]["pops"], pe * wl.dt, wl.tau)
            assert T > 0
            assert ion[k] == pytest.approx(T, rel=1e-10)
            assert loss[k] == pytest.approx(signal.loss(r["eps_a"], T), rel=1e-10)


def test_spsa_chains_follow_the_oracle():
    m = _model()
    th0 = np.array([[0.9, 0.5, 1.0, 0.5, 0.4, 0.3, 3.05, 0.7],
                    [1.2, 0.3, 0.9, 0.4, 0.5, 0.25, 3.0, 1.2]])
    scale = np.array([0.2, 0.2, 0.1, 0.05, 0.05, 0.05, 0.02, 0.3])
    tau, dt, seed, eps, pe = 1.2, 2e-3, 5, 1e-3, 10
    rng = np.random.default_rng(7)
    deltas = rng.choice([-1.0, 1.0], size=(3, 2, 8))
    opt = spsa.SPSA(m, 4, 1, th0, scale, tau, dt, seed, eps=eps, precision="fp64", engine="fused",
                    pop_every=pe, a=0.2, c=0.1, A=2.0)
    gpu_hist = [opt.theta.copy()]
    for k in range(3):
        opt.step(deltas[k])
        gpu_hist.append(opt.theta.copy())
    opt.close()
    # oracle: the same chains; candidate j of the batch uses initial-state
    # trajectories 2j, 2j+1 (plus-candidates first, then minus-candidates)
    n = th0.shape[0]
    for ch in range(n):
        def pair(tp, tm, ch=ch):
            out = []
            for slot, th in ((ch, tp), (n + ch, tm)):
                cand = li.Candidate(m, 4, li.PulseParams(1, tuple(th)))
                wl = li.Workload("spsa", [cand] * (2 * n), dt, int(round(tau / dt)), tau, init_seed=seed, eps=eps)
                r = gradient.run_candidate(wl, slot, pop_every=pe)
                T = signal.ionization(r["g"]["pops"], r["e"]["pops"], pe * dt, tau)
                out.append(signal.loss(r["eps_a"], T))
            return tuple(out)
        hist, _ = ospsa.spsa(pair, 1, th0[ch], deltas[:, ch], scale, a=0.2, c=0.1, A=2.0)
        for k in range(4):
            assert np.allclose(gpu_hist[k][ch], hist[k], rtol=1e-9, atol=1e-12), (ch, k)
