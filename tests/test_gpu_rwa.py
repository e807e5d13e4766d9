"""Rotating frame with the rotating-wave approximation (RWA Hamiltonian of
Sec. S2) against the oracle's rotating-frame model.

Both sides integrate H = sum (w - w_d) n + (alpha/2) b^dag b^dag b b
+ g (b^dag a + b a^dag) [+ J (a^dag f + a f^dag)] + (Omega/2)(e^{i phi} r
+ e^{-i phi} r^dag) with the same jumps. The slow Hamiltonian allows a step
of 2.5-5 ps. Tolerances as for the lab frame: 1e-10 for the FP64 engines,
5e-5 for FP32_G64 (FP32 state rounding, u32 sqrt(4 n_steps)).
"""
import dataclasses

import pytest

import lr_inputs as li
from oracle import parallel
from paper_2508_18114_gb300 import LrError, runner

from _compare import compare_observables

pytestmark = pytest.mark.gpu


def _nts(wl):
    return [c.model.dims[0] for c in wl.candidates for _ in (0, 1)]


def _ragged(n_steps=400, dt=5e-3):
    f = lambda nt, nr, nf: li.ModelParams(  # noqa: E731
        dims=(nt, nr, nf), wq=li.TWO_PI * 6.0, alpha=-li.TWO_PI * 0.3, wr=li.TWO_PI * 7.5, g=li.TWO_PI * 0.15,
        kappa=li.TWO_PI * 0.05, gamma=1.0 / 50000.0, wf=li.TWO_PI * 7.51, J=li.TWO_PI * 0.1)
    cands = [li.Candidate(f(3, 7, 5), 7, li.pulse_two_segment(61, li.TWO_PI * 7.5)),
             li.Candidate(f(5, 6, 3), 12, li.pulse_two_segment(62, li.TWO_PI * 7.5)),
             li.Candidate(f(4, 9, 6), 20, li.pulse_two_segment(63, li.TWO_PI * 7.5))]
    return li.Workload("ragged_rwa", cands, dt, n_steps, n_steps * dt, init_seed=94, eps=1e-5, frame="rwa")


@pytest.mark.parametrize("engine,precision,tol", [("plain", "fp64", 1e-10), ("fused", "fp64", 1e-10),
                                                  ("fused", "fp32_g64", 5e-5)])
def test_rwa_three_modes_match_oracle(engine, precision, tol):
    wl = _ragged()
    job = parallel.OracleJob(wl, None, 50)   # spawn workers before any GPU work
    g = runner.run(wl, precision=precision, engine=engine, pop_every=50)
    ora = job.result()
    assert g["engine"] == engine
    print(compare_observables(g, ora, 2 * len(wl.candidates), _nts(wl), tol, tol, "rwa %s %s" % (engine, precision)))


@pytest.mark.parametrize("engine", ["plain", "fused"])
def test_rwa_two_modes_full_pulse(engine):
    """c1 model (drive on the resonator) over its 40 ns pulse at dt = 5 ps
    (8000 steps instead of the lab frame's 40000)."""
    wl = dataclasses.replace(li.c1(), dt=5e-3, n_steps=8000, frame="rwa")
    job = parallel.OracleJob(wl, None, 400)
    g = runner.run(wl, precision="fp64", engine=engine, pop_every=400)
    ora = job.result()
    print(compare_observables(g, ora, 2, _nts(wl), 1e-10, 1e-10, "c1 rwa " + engine))


def test_rwa_backward_is_unsupported():
    wl = _ragged(20)
    b = runner.make_batch(wl, precision="fp64", engine="plain", pop_every=10)
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, 20)
    with pytest.raises(LrError) as ei:
        b.backward([1.0] * len(wl.candidates), ckpt_every=10)
    assert ei.value.status == 9   # LR_ERR_UNSUPPORTED
    b.close()
