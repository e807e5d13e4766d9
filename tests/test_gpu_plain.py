"""PLAIN engine (complex128, state in HBM) against the FP64 oracle.

Tolerance for FP64 paths: 1e-10 relative (max norm over the record) for the
readout signal, photon number and assignment error; 1e-10 absolute for the
level populations and tr(rho), which are O(1).
"""
import math

import numpy as np
import pytest

import lr_inputs as li
from oracle import init_state, lindblad, lowrank, parallel, pulse
from oracle.model import Model
from paper_2508_18114_gb300 import LowRankBatch, LrError, runner

from _compare import compare_observables

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _nts(wl):
    return [c.model.dims[0] for c in wl.candidates for _ in (0, 1)]


def _small_filter(nt, nr, nf):
    return li.ModelParams(dims=(nt, nr, nf), wq=li.TWO_PI * 6.0, alpha=-li.TWO_PI * 0.3,
                          wr=li.TWO_PI * 7.5, g=li.TWO_PI * 0.15, kappa=li.TWO_PI * 0.05,
                          gamma=1.0 / 50000.0, wf=li.TWO_PI * 7.51, J=li.TWO_PI * 0.1)


def _ragged_workload(n_steps=400):
    """Uneven N and M spanning several 16-row tiles with ragged tails, both
    model families, maximum rank 32 and maximum transmon truncation 16."""
    c1m = li.c1().candidates[0].model
    cands = [
        li.Candidate(_small_filter(3, 5, 7), 7, li.pulse_two_segment(21, li.TWO_PI * 7.5)),
        li.Candidate(c1m, 5, li.pulse_flat_top(22, c1m.wr)),
        li.Candidate(_small_filter(5, 4, 3), 12, li.pulse_two_segment(23, li.TWO_PI * 7.5)),
        li.Candidate(_small_filter(16, 4, 3), 32, li.pulse_two_segment(24, li.TWO_PI * 7.5)),
    ]
    dt = 5e-4
    # pulse tau = 2 ns so that the short run sees rising and falling edges
    return li.Workload("ragged", cands, dt, n_steps, 2.0, init_seed=77, eps=1e-5)


def test_c1_full_pulse_parity():
    wl = li.c1()
    pe = 100
    job = parallel.OracleJob(wl, None, pe)       # spawn workers before any GPU work
    gpu = runner.run(wl, precision="fp64", engine="plain", pop_every=pe)
    ora = job.result()
    w = compare_observables(gpu, ora, 2, _nts(wl), TOL, TOL, "c1 plain fp64")
    print("c1 full pulse plain fp64:", w)
    assert gpu["engine"] == "plain"


def test_c2_full_size_parity():
    wl = li.c2(n_steps=300)
    gpu = runner.run(wl, precision="fp64", engine="plain", pop_every=50)
    ora = parallel.run_workload(wl, None, 50)
    w = compare_observables(gpu, ora, 2, _nts(wl), TOL, TOL, "c2 plain fp64 (300 steps)")
    print("c2 N=2000 M=20 plain fp64:", w)


def test_ragged_batch_parity():
    wl = _ragged_workload()
    gpu = runner.run(wl, precision="fp64", engine="plain", pop_every=40)
    ora = parallel.run_workload(wl, None, 40)
    compare_observables(gpu, ora, 2 * len(wl.candidates), _nts(wl), TOL, TOL, "ragged plain fp64")


def test_initial_state_matches_oracle():
    wl = _ragged_workload()
    b = runner.make_batch(wl, engine="plain", max_steps=10)
    b.set_initial(wl.init_seed, wl.eps)
    for k, c in enumerate(wl.candidates):
        mdl = Model.from_params(c.model)
        for lvl in (0, 1):
            j = 2 * k + lvl
            z = b.get_state(j)
            psi = mdl.basis_index((lvl,) + (0,) * (len(c.model.dims) - 1))
            zo = init_state.initial_state(mdl.N, c.M, psi, wl.eps, wl.init_seed, j)
            rg, ro = z @ z.conj().T, zo @ zo.conj().T
            assert np.abs(rg - ro).max() < 1e-13
            assert abs(np.trace(rg).real - 1) < 1e-13
    b.close()


def test_full_rank_matches_oracle_and_lindblad():
    """M = N: the CUDA path equals the low-rank oracle and follows the full
    master equation up to RK4's gap, which shrinks ~16x when dt halves."""
    m = _small_filter(2, 3, 2)
    cand = li.Candidate(m, 12, li.PulseParams(1, (0.3, 0.1, 0.3, 0.1, 0.1, 0.1, li.TWO_PI * 7.45, 0.4)))
    mdl = Model.from_params(m)
    gaps = []
    for dt, n in ((1e-3, 500), (5e-4, 1000)):
        wl = li.Workload("fullrank", [cand], dt, n, n * dt, init_seed=5, eps=1e-3)
        gpu = runner.run(wl, precision="fp64", engine="plain", pop_every=n)
        ora = parallel.run_workload(wl, None, n, processes=1)
        compare_observables(gpu, ora, 2, _nts(wl), TOL, TOL, "full rank")
        coef = pulse.coefficient(1, cand.pulse.p, wl.tau)
        z0 = init_state.initial_state(12, 12, mdl.basis_index((1, 0, 0)), wl.eps, wl.init_seed, 1)
        full = lindblad.integrate(z0 @ z0.conj().T, mdl, coef, dt, n, pop_every=n)
        gaps.append(np.abs(gpu["beta"][1] - full["beta"]).max())
    assert gaps[1] < 1e-5
    assert 10 < gaps[0] / gaps[1] < 22


def test_resume_is_bitwise():
    wl = _ragged_workload(200)
    a = runner.make_batch(wl, engine="plain", max_steps=200, pop_every=20)
    a.set_initial(wl.init_seed, wl.eps)
    a.integrate(wl.dt, 200)
    oa = a.observables()
    b = runner.make_batch(wl, engine="plain", max_steps=200, pop_every=20)
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, 120)
    zs = [b.get_state(j) for j in range(b.n_traj)]
    b.integrate(wl.dt, 80)
    ob = b.observables()
    for k in ("beta", "pops", "nphot", "trace", "eps_a"):
        assert np.array_equal(oa[k], ob[k]), k
    # checkpoint / restore into a fresh context continues identically
    c = runner.make_batch(wl, engine="plain", max_steps=200, pop_every=20)
    c.set_initial(wl.init_seed, wl.eps)
    c.integrate(wl.dt, 120)
    for j, z in enumerate(zs):
        c.set_state(j, z, step=120)
    c.integrate(wl.dt, 80)
    oc = c.observables()
    assert np.array_equal(oa["beta"], oc["beta"])
    for j in range(a.n_traj):
        assert np.array_equal(a.get_state(j), c.get_state(j))
    for x in (a, b, c):
        x.close()


def test_state_roundtrip_and_determinism():
    wl = _ragged_workload(50)
    a = runner.make_batch(wl, engine="plain", max_steps=50)
    rng = np.random.default_rng(0)
    N, M = 105, 7
    z = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    a.set_state(0, z)
    assert np.array_equal(a.get_state(0), z)
    r1 = runner.run(wl, engine="plain", pop_every=10)
    r2 = runner.run(wl, engine="plain", pop_every=10)
    for k in ("beta", "pops", "eps_a"):
        assert np.array_equal(r1[k], r2[k])
    a.close()


def test_not_positive_definite_is_reported():
    """A rank-deficient state (two equal columns) is caught by the Cholesky
    pivot check and reported as LR_ERR_NOT_PD; the GPU keeps running."""
    wl = _ragged_workload(20)
    b = runner.make_batch(wl, engine="plain", max_steps=20)
    b.set_initial(wl.init_seed, wl.eps)
    z = b.get_state(0)
    z[:, 1] = z[:, 2]
    b.set_state(0, z)
    b.integrate(wl.dt, 5)
    with pytest.raises(LrError) as ei:
        b.observables()
    assert ei.value.status == 5
    b.close()


def test_call_order_and_capacity_errors():
    wl = _ragged_workload(20)
    b = LowRankBatch([c.model for c in wl.candidates], [c.M for c in wl.candidates], engine="plain",
                     max_steps=20)
    with pytest.raises(LrError) as ei:
        b.integrate(wl.dt, 5)
    assert ei.value.status == 8
    b.set_pulse([(c.pulse.kind, c.pulse.p) for c in wl.candidates], wl.tau)
    b.set_initial(1, 1e-5)
    with pytest.raises(LrError) as ei:
        b.integrate(wl.dt, 21)
    assert ei.value.status == 1
    b.integrate(wl.dt, 5)
    with pytest.raises(LrError) as ei:
        b.integrate(2 * wl.dt, 5)
    assert ei.value.status == 8
    with pytest.raises(LrError):
        b.set_pulse([(1, (math.nan,) * 8)] * len(wl.candidates), wl.tau)
    b.close()
