"""Validity diagnostics (Sec. S1.B, Fig. S1) against the oracle.

The library records the FP64 Gram matrix at the record steps and
diagonalises it on the device (lr_diagnostics); the oracle records m^dag m
and takes numpy's eigvalsh. Spectra are compared eigenvalue by eigenvalue,
each relative to itself (the smallest are ~eps = 1e-5 of the largest).
FP64 engines: 1e-9 relative (the Jacobi sweeps stop at 1e-14 relative
off-diagonal norm, which moves the eps-sized eigenvalues by up to ~1e-9 of
themselves) and 1e-10 for the purity. FP32_G64: the state carries FP32
rounding (a random walk of u32 sqrt(4 n_steps)), so 5e-5, as the other
observables.
"""
import numpy as np
import pytest

import lr_inputs as li
from oracle import diagnostics, parallel
from paper_2508_18114_gb300 import LrError, runner

pytestmark = pytest.mark.gpu


def _batch(n_steps=300):
    f = lambda nt, nr, nf: li.ModelParams(  # noqa: E731
        dims=(nt, nr, nf), wq=li.TWO_PI * 6.0, alpha=-li.TWO_PI * 0.3, wr=li.TWO_PI * 7.5, g=li.TWO_PI * 0.15,
        kappa=li.TWO_PI * 0.05, gamma=1.0 / 50000.0, wf=li.TWO_PI * 7.51, J=li.TWO_PI * 0.1)
    cands = [li.Candidate(f(3, 7, 5), 7, li.pulse_two_segment(51, li.TWO_PI * 7.5)),
             li.Candidate(f(4, 9, 6), 20, li.pulse_two_segment(52, li.TWO_PI * 7.5)),
             li.Candidate(f(2, 5, 4), 1, li.pulse_two_segment(53, li.TWO_PI * 7.5))]
    return li.Workload("diag", cands, 5e-4, n_steps, 2.0, init_seed=93, eps=1e-5)


def _compare(pur, eig, ora, wl, tol_eig, tol_pur, what):
    worst_e, worst_p = 0.0, 0.0
    for j, G_list in enumerate(ora["gram"]):
        M = wl.candidates[j // 2].M
        for r, G in enumerate(G_list):
            want = diagnostics.gram_spectrum(G)
            got = eig[j, r, :M]
            worst_e = max(worst_e, float(np.max(np.abs(got - want) / np.abs(want))))
            assert np.all(eig[j, r, M:] == 0.0)
            p = diagnostics.gram_purity(G)
            worst_p = max(worst_p, abs(pur[j, r] - p) / p)
    msg = "%s: eigenvalues %.3g purity %.3g" % (what, worst_e, worst_p)
    assert worst_e <= tol_eig, msg
    assert worst_p <= tol_pur, msg
    return msg


@pytest.mark.parametrize("engine,precision,tol", [("plain", "fp64", 1e-9), ("fused", "fp64", 1e-9),
                                                  ("fused", "fp32_g64", 5e-5)])
def test_spectrum_and_purity_match_oracle(engine, precision, tol):
    wl = _batch()
    pe = 50
    job = parallel.OracleJob(wl, None, pe, gram=True)   # spawn workers before any GPU work
    b = runner.make_batch(wl, precision=precision, engine=engine, pop_every=pe, record_gram=True)
    assert b.engine == engine
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    pur, eig = b.diagnostics()
    b.close()
    ora = job.result()
    print(_compare(pur, eig, ora, wl, tol, tol if precision == "fp32_g64" else 1e-10, engine + " " + precision))


@pytest.mark.parametrize("engine", ["plain", "fused"])
def test_initial_state_closed_forms_on_device(engine):
    """Step 0: eigenvalues 1 - (M-1) eps and eps, purity (1-(M-1)eps)^2 + (M-1) eps^2,
    rank indicator p_M / p_1 = eps / (1 - (M-1) eps); records after the step are zero."""
    wl = _batch(10)
    b = runner.make_batch(wl, precision="fp64", engine=engine, pop_every=5, record_gram=True)
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, 0)
    pur, eig = b.diagnostics()
    b.close()
    eps = wl.eps
    for j in range(2 * len(wl.candidates)):
        M = wl.candidates[j // 2].M
        p0 = 1.0 - (M - 1) * eps
        want = np.array([p0] + [eps] * (M - 1))
        assert np.allclose(eig[j, 0, :M], want, rtol=1e-9, atol=0), (j, eig[j, 0, :M])
        assert abs(pur[j, 0] - (p0 ** 2 + (M - 1) * eps ** 2)) < 1e-12
        if M > 1:
            assert abs(eig[j, 0, M - 1] / eig[j, 0, 0] - eps / p0) < 1e-9 * eps / p0
        assert np.all(eig[j, 1:] == 0.0) and np.all(pur[j, 1:] == 0.0)


def test_diagnostics_need_recorded_gram():
    wl = _batch(10)
    b = runner.make_batch(wl, precision="fp64", engine="plain", pop_every=5)
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, 5)
    with pytest.raises(LrError) as ei:
        b.diagnostics()
    assert ei.value.status == 8   # LR_ERR_STATE
    b.close()
