"""Seeded single-shot readout (lr_assignment_shots) against the oracle's
definition (oracle.signal.assignment_shots), each on its own integration of
the same three-candidate batch (FP64, 300 steps): the misassigned shots per
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


def _batch(n_steps=300):
    f = lambda nt, nr, nf: li.ModelParams(  # noqa: E731
        dims=(nt, nr, nf), wq=li.TWO_PI * 6.0, alpha=-li.TWO_PI * 0.3, wr=li.TWO_PI * 7.5, g=li.TWO_PI * 0.15,
        kappa=li.TWO_PI * 0.05, gamma=1.0 / 50000.0, wf=li.TWO_PI * 7.51, J=li.TWO_PI * 0.1)
    cands = [li.Candidate(f(3, 7, 5), 7, li.pulse_two_segment(61, li.TWO_PI * 7.5)),
             li.Candidate(f(4, 9, 6), 12, li.pulse_two_segment(62, li.TWO_PI * 7.5)),
             li.Candidate(f(2, 5, 4), 3, li.pulse_two_segment(63, li.TWO_PI * 7.5))]
    return li.Workload("shots", cands, 5e-4, n_steps, 2.0, init_seed=95, eps=1e-5)


@pytest.mark.parametrize("bin_steps", [1, 20])
def test_shots_match_the_oracle(bin_steps):
    wl = _batch()
    job = parallel.OracleJob(wl, None, 100)
    b = runner.make_batch(wl, precision="fp64", pop_every=100)
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
        assert tuple(int(x) for x in got["errors"][c]) == want["errors"]
        assert got["eps_bin"][c] == pytest.approx(want["eps_bin"], rel=1e-9)
        assert got["eps_shots"][c] == pytest.approx(want["eps_shots"], rel=1e-12)


def test_shots_converge_on_the_device():
    """200,000 shots per state on the device: within four binomial standard
    deviations of erfc(SNR_b / 2) / 2 (+ tau gamma / 2)."""
    wl = _batch()
    b = runner.make_batch(wl, precision="fp64", pop_every=100)
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    ns = 200000
    r = b.assignment_shots(ns, 99, bin_steps=5)
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
    wl = _batch()
    b = runner.make_batch(wl, precision="fp64", pop_every=100)
    b.set_initial(wl.init_seed, wl.eps)
    with pytest.raises(LrError) as ei:
        b.assignment_shots(10, 1)
    assert ei.value.status == 8   # LR_ERR_STATE
    b.close()
