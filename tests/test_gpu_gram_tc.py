"""The Gram matrix on the tensor cores (FP32_G64, fused engine, Mp = 20): exact
bf16 slices of the scaled columns, bf16 MMAs with FP32 accumulation that is
exact for at most 1024 rows, slice pairs added in double-word. It must be
FP64-class like the double-word CUDA-core sums it replaces: on the same FP32
state, the spectrum of rho = Z Z^dag (from the recorded FP64 Gram matrix)
agrees with the double-word Gram's to ~1e-10 relative even for the eigenvalues
eps = 1e-5, which an FP32-accurate Gram matrix (2^-24 of the largest entry)
would miss by ~1e-2. Whole runs against the oracle: the fused and full-pulse
tests at N = 2000, whose plan uses this Gram by default, and the test below."""
import numpy as np
import pytest

import lr_inputs as li
from paper_2508_18114_gb300 import runner

pytestmark = pytest.mark.gpu

PLAN = {"LR_FUSED_C": "2", "LR_FUSED_ZS": "global", "LR_FUSED_TC": "0"}


def _spectrum(monkeypatch, gram, n_steps):
    for k, v in PLAN.items():
        monkeypatch.setenv(k, v)
    if gram:
        monkeypatch.delenv("LR_FUSED_GRAM", raising=False)   # the default of this plan
    else:
        monkeypatch.setenv("LR_FUSED_GRAM", "dw")
    wl = li.c4(n_candidates=3)
    b = runner.make_batch(wl, precision="fp32_g64", engine="fused", pop_every=10, max_steps=max(n_steps, 10),
                          record_gram=True)
    info = b.query()
    assert info.gram_tc == (1 if gram else 0)
    assert info.team_size == 2
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, n_steps)
    pur, eig = b.diagnostics()
    z = b.get_state(0)
    b.close()
    return pur, eig, z


def test_gram_tc_spectrum_of_the_initial_state(monkeypatch):
    pur_t, eig_t, _ = _spectrum(monkeypatch, True, 0)
    pur_d, eig_d, _ = _spectrum(monkeypatch, False, 0)
    e_t, e_d = eig_t[:, 0, :20], eig_d[:, 0, :20]
    assert np.all(e_d[:, -1] > 5e-6)          # the eps eigenvalues are there
    rel = np.abs(e_t - e_d) / np.abs(e_d)
    print("initial spectrum: max relative difference", rel.max())
    assert rel.max() < 1e-9
    assert np.abs(pur_t[:, 0] - pur_d[:, 0]).max() < 1e-13


def test_gram_tc_spectrum_after_steps(monkeypatch):
    """After 40 steps both runs carry their own FP32 rounding of the state
    (~1e-7 relative per entry): the spectra agree at that level."""
    pur_t, eig_t, zt = _spectrum(monkeypatch, True, 40)
    pur_d, eig_d, zd = _spectrum(monkeypatch, False, 40)
    r = 4   # record at step 40
    rel = np.abs(eig_t[:, r, :20] - eig_d[:, r, :20]) / np.abs(eig_d[:, r, :20])
    print("spectrum after 40 steps: max relative difference", rel.max())
    assert rel.max() < 1e-3
    assert np.abs(zt - zd).max() < 1e-5 * np.abs(zd).max()


def test_gram_tc_parity_with_oracle(monkeypatch):
    """Three candidates of the N = 2000, M = 20 batch, 120 steps, against the
    FP64 oracle at the FP32_G64 bounds, with the Gram on the tensor cores."""
    from oracle import parallel
    from _compare import compare_observables
    for k, v in PLAN.items():
        monkeypatch.setenv(k, v)
    monkeypatch.delenv("LR_FUSED_GRAM", raising=False)
    wl = li.c4(n_candidates=3, n_steps=120)
    job = parallel.OracleJob(wl, None, 40)
    b = runner.make_batch(wl, precision="fp32_g64", engine="fused", pop_every=40)
    assert b.query().gram_tc == 1
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    got = b.observables()
    b.close()
    ora = job.result()
    nts = [c.model.dims[0] for c in wl.candidates for _ in (0, 1)]
    print(compare_observables(got, ora, 6, nts, 5e-5, 5e-5, "gram on tensor cores"))
