"""Seeded single-shot readout (lr_assignment_shots) against the oracle's
definition (oracle.signal.assignment_shots), each on its own integration of
the same three-candidate batch (FP64, 12,000 steps): the misassigned shots per
candidate and state are equal (the decisions are FP64 on both sides; a shot
would differ only if its statistic sat within rounding of the threshold), and
the empirical error lies within four binomial standard deviations of the
binned closed form it converges to."""
import math

import numpy as np
import pytest

import lr_inputs as li
from oracle import parallel
from oracle import signal
from paper_2508_18114_gb300 import LrError, runner

pytestmark = pytest.mark.gpu


def _batch(n_steps=12000):
    """Transmon x resonator (4 x 25), g/2pi = 300 MHz, kappa/2pi = 50 MHz, a
    strong resonant drive (120 MHz, 1 ns rise) over 12 ns: the g and e fields
    separate (eps_a 0.23-0.30), so the shot counts test the decisions."""
    TP = li.TWO_PI
    m = li.ModelParams(dims=(4, 25), wq=TP * 6.0, alpha=-TP * 0.3, wr=TP * 7.0, g=TP * 0.3, kappa=TP * 0.05,
                       gamma=1.0 / 50000.0)
    cands = [li.Candidate(m, 4, li.PulseParams(0, (TP * 0.12, TP * 7.0 + d, 1.0, 0.3)))
             for d in (0.0, -TP * 0.02, TP * 0.015)]
    return li.Workload("shots", cands, 1e-3, n_steps, n_steps * 1e-3, init_seed=97, eps=1e-5)


@pytest.mark.parametrize("bin_steps", [6, 20])
def test_shots_match_the_oracle(bin_steps):
    wl = _batch()
    job = parallel.OracleJob(wl, None, 1000)
    b = runner.make_batch(wl, precision="fp64", pop_every=1000)
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    eta, ns, seed = 0.6, 3000, 424242
    got = b.assignment_shots(ns, seed, bin_steps=bin_steps, eta=eta)
    b.close()
    ora = job.result()
    for c, cand in enumerate(wl.candidates):
        m = cand.model
        want = signal.assignment_shots(ora["beta"][2 * c], ora["beta"][2 * c + 1], wl.dt, m.kappa, m.gamma, eta, ns,
                                       bin_steps, seed, c)
        print(c, "errors gpu", got["errors"][c], "oracle", want["errors"], "eps_bin", got["eps_bin"][c],
              want["eps_bin"])
        assert want["eps_bin"] < 0.35                 # the states do separate
        assert tuple(int(x) for x in got["errors"][c]) == want["errors"]
        assert got["eps_bin"][c] == pytest.approx(want["eps_bin"], rel=1e-9)
        assert got["eps_shots"][c] == pytest.approx(want["eps_shots"], rel=1e-12)


def test_shots_converge_on_the_device():
    """200,000 shots per state on the device: within four binomial standard
    deviations of erfc(SNR_b / 2) / 2 (+ tau gamma / 2)."""
    wl = _batch()
    b = runner.make_batch(wl, precision="fp64", pop_every=1000)
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    ns = 200000
    r = b.assignment_shots(ns, 99, bin_steps=10)
    tau = wl.n_steps * wl.dt
    for c, cand in enumerate(wl.candidates):
        dec = 0.5 * tau * cand.model.gamma
        p = r["eps_bin"][c] - dec
        got = r["eps_shots"][c] - dec
        sig = math.sqrt(max(p * (1 - p), 1e-12) / (2 * ns))
        print(c, got, p, sig)
        assert abs(got - p) <= 4 * sig + 1e-12
    # argument checks
    with pytest.raises(LrError):
        b.assignment_shots(0, 1)
    with pytest.raises(LrError):
        b.assignment_shots(10, 1, bin_steps=0)
    b.close()


def test_shots_need_a_step():
    wl = _batch(100)
    b = runner.make_batch(wl, precision="fp64", pop_every=100)
    b.set_initial(wl.init_seed, wl.eps)
    with pytest.raises(LrError) as ei:
        b.assignment_shots(10, 1)
    assert ei.value.status == 8   # LR_ERR_STATE
    b.close()
