"""The full master equation on the device (lr_full_*, FP64) against the
oracle's full master equation (Eq. S4 with the time-dependent operators of the
paper's model), through the C ABI."""
import numpy as np
import pytest

from oracle import paper_model as pm
from oracle import pulse as opulse

pytestmark = pytest.mark.gpu

TP = 2.0 * np.pi


def _params(**over):
    P = dict(Ec=TP * 0.315, Ej=51 * TP * 0.315, wr=TP * 7.2, wf=TP * 7.21, g=TP * 0.15, J=TP * 0.03,
             kappa=TP * 0.03, gamma=TP * 8e-6, wd=TP * 7.18)
    P.update(over)
    return P


@pytest.mark.parametrize("frame", ["rot", "rwa"])
@pytest.mark.parametrize("psi", [0, 1])
def test_full_me_matches_oracle(frame, psi):
    """N = 72 (6 x 3 x 4), strong short drive, 800 steps: beta at every step,
    populations, photons and trace every 100 steps, the final rho; FP64
    rounding only (1e-10)."""
    from paper_2508_18114_gb300 import sparse
    P = _params(g=TP * 0.3, kappa=1.0, gamma=0.05)
    dims, dt, n, pe, tau = (6, 3, 4), 5e-4, 800, 100, 0.4
    pulse = (0, [TP * 1.0, P["wd"], 0.05, 0.0])
    model = sparse.paper_model(*dims, frame=frame, **P)
    f = sparse.FullME(model, pulse, tau, n, pop_every=pe)
    f.set_initial(psi)
    f.integrate(dt, 300)
    f.integrate(dt, n - 300)
    got = f.observables()
    rho = f.get_state()
    ora = pm.PaperModel(*dims, frame=frame, **P)
    env = lambda t: opulse.envelope(pulse[0], pulse[1], t, tau)  # noqa: E731
    r0 = np.zeros((ora.N, ora.N), complex)
    r0[psi, psi] = 1.0
    want = pm.integrate(r0, ora, env, dt, n, pop_every=pe, low_rank=False, return_state=True)
    bs = np.abs(want["beta"]).max()
    assert bs > 1e-2
    assert np.abs(got["beta"] - want["beta"]).max() <= 1e-10 * bs
    assert np.abs(got["pops"] - want["pops"]).max() <= 1e-10
    assert np.abs(got["nphot"] - want["nr"]).max() <= 1e-10 * max(want["nr"].max(), 1.0)
    assert np.abs(got["trace"] - want["trace"]).max() <= 1e-11
    assert np.abs(rho - want["state"]).max() <= 1e-10


def test_full_me_paper_size_first_steps():
    """The paper's N = 2000 (100 x 4 x 5) from |e>: 3 steps against the oracle
    (every element of rho)."""
    from paper_2508_18114_gb300 import sparse
    P = _params()
    dims, dt, n, tau = (100, 4, 5), 5e-4, 3, 40.0
    pulse = (0, [TP * 0.15, P["wd"], 2.5, 0.0])
    model = sparse.paper_model(*dims, **P)
    f = sparse.FullME(model, pulse, tau, n, pop_every=1)
    f.set_initial(1)
    f.integrate(dt, n)
    got = f.observables()
    rho = f.get_state()
    ora = pm.PaperModel(*dims, frame="rot", **P)
    env = lambda t: opulse.envelope(pulse[0], pulse[1], t, tau)  # noqa: E731
    r0 = np.zeros((ora.N, ora.N), complex)
    r0[1, 1] = 1.0
    want = pm.integrate(r0, ora, env, dt, n, pop_every=1, low_rank=False, return_state=True)
    assert np.abs(rho - want["state"]).max() <= 1e-12
    assert np.abs(got["pops"] - want["pops"]).max() <= 1e-12
    assert np.abs(got["beta"] - want["beta"]).max() <= 1e-12


def test_full_me_from_a_low_rank_factor_equals_the_low_rank_run_at_full_rank():
    """rho(0) = Z Z^dag on the device (lr_full_set_state_lowrank); with M = N the
    low-rank equation is the master equation (Eq. S5 vs Eq. S4), so the two GPU
    engines agree to the RK4 discretisation gap (O(dt^4) per unit time)."""
    from paper_2508_18114_gb300 import sparse
    P = _params(g=TP * 0.3, kappa=1.0, gamma=0.05)
    dims, dt, n, tau = (3, 2, 3), 5e-4, 400, 0.2
    pulse = (0, [TP * 1.0, P["wd"], 0.03, 0.0])
    model = sparse.paper_model(*dims, **P)
    N = model["N"]
    b = sparse.SparseBatch(model, N, [pulse], tau, n, pop_every=100, precision="fp64")
    b.set_initial([1], 5, 1e-3)
    z0 = b.get_state()[0]
    f = sparse.FullME(model, pulse, tau, n, pop_every=100)
    f.set_state_lowrank(z0)
    assert np.abs(f.get_state() - z0 @ z0.conj().T).max() < 1e-15
    b.integrate(dt, n)
    f.integrate(dt, n)
    lo, fo = b.observables(), f.observables()
    assert np.abs(lo["beta"][0] - fo["beta"]).max() < 1e-8 * max(np.abs(fo["beta"]).max(), 1.0)
    assert np.abs(lo["pops"][0] - fo["pops"]).max() < 1e-8
