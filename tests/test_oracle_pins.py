"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, published constants, identities between two different equations of
the paper (Eq. S5 vs Eq. S4), or convergence orders.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import init_state, lindblad, lowrank, pulse, signal, gradient, diagnostics
from oracle.model import Model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def small_model(dims=(3, 4), **kw):
    p = dict(wq=2.0, alpha=-0.4, wr=3.0, g=0.3, kappa=0.5, gamma=0.2,
             wf=3.2, J=0.25)
    p.update(kw)
    return Model(dims, **p, dense=True)


def random_state(N, M, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))


# ---------------------------------------------------------------- RNG / init

def test_splitmix64_published_outputs():
    want = [int(r[0], 16) for r in _read_golden("splitmix64_seed0.txt")]
    got = init_state.splitmix64(0, np.arange(len(want)))
    assert [int(x) for x in got] == want


def test_box_muller_moments():
    xi = init_state.gaussian_columns(12345, 200000, 1)[:, 0]
    assert abs(xi.real.mean()) < 0.01 and abs(xi.imag.mean()) < 0.01
    assert abs(np.mean(np.abs(xi) ** 2) - 2.0) < 0.02
    assert abs(np.mean(xi ** 2)) < 0.02          # circular symmetry
    assert abs(np.mean(xi.real ** 4) - 3.0) < 0.1  # Gaussian kurtosis


def test_uniforms_in_open_unit_interval():
    u = init_state.uniforms(7, np.arange(100000))
    assert u.min() > 0.0 and u.max() <= 1.0
    assert abs(u.mean() - 0.5) < 0.005


@pytest.mark.parametrize("N,M", [(40, 4), (12, 12), (30, 1)])
def test_initial_state_structure(N, M):
    eps = 1e-5
    m = init_state.initial_state(N, M, 5, eps, seed=3, traj=2)
    G = m.conj().T @ m
    want = np.diag([1.0 - (M - 1) * eps] + [eps] * (M - 1))
    assert np.allclose(G, want, atol=1e-15, rtol=0)
    assert abs(np.trace(G).real - 1.0) < 1e-14
    psi = np.zeros(N)
    psi[5] = 1
    assert np.allclose(m[:, 0], np.sqrt(1 - (M - 1) * eps) * psi)


# ---------------------------------------------------------------- model

def test_hamiltonian_matrix_elements():
    """Matrix elements of Eq. 1 (bare-mode form) from ladder-operator algebra."""
    wq, al, wr, g, wf, J = 2.0, -0.4, 3.0, 0.3, 3.2, 0.25
    mdl = Model((3, 2, 2), wq=wq, alpha=al, wr=wr, g=g, kappa=0.1, gamma=0.1,
                wf=wf, J=J, dense=True)
    H = mdl.H0
    idx = mdl.basis_index
    assert H[idx((2, 1, 1)), idx((2, 1, 1))] == pytest.approx(2 * wq + al + wr + wf)
    assert H[idx((1, 0, 0)), idx((0, 1, 0))] == pytest.approx(g)
    assert H[idx((2, 1, 0)), idx((1, 0, 0))] == pytest.approx(g * math.sqrt(2))
    assert H[idx((1, 1, 0)), idx((0, 0, 0))] == pytest.approx(g)       # counter-rotating
    assert H[idx((0, 1, 0)), idx((0, 0, 1))] == pytest.approx(J)
    assert H[idx((0, 1, 1)), idx((0, 0, 0))] == pytest.approx(J)       # counter-rotating
    assert H[idx((0, 0, 0)), idx((2, 0, 0))] == 0
    assert np.allclose(H, H.conj().T)
    Xd = mdl.Xd
    assert Xd[idx((1, 1, 1)), idx((1, 1, 0))] == pytest.approx(1.0)
    assert Xd[idx((1, 1, 0)), idx((1, 1, 1))] == pytest.approx(1.0)


# ---------------------------------------------------------------- pulses

def test_logistic_closed_forms():
    assert pulse.logistic(2.5, 2.5, 0.3) == 0.5
    for x in (0.1, 0.7, 2.0):
        assert pulse.logistic(1 + x, 1, 0.4) + pulse.logistic(1 - x, 1, 0.4) == pytest.approx(1.0, abs=1e-15)


def test_flat_top_shape():
    A, tr, tau = 0.3, 2.5, 40.0
    s = tr / 5
    assert pulse.flat_top_envelope(tau / 2, A, tr, tau) == pytest.approx(A, rel=1e-12)
    assert pulse.flat_top_envelope(6 * s, A, tr, tau) == pytest.approx(A / 2, rel=1e-12)
    assert pulse.flat_top_envelope(0.0, A, tr, tau) == pytest.approx(A / (1 + math.exp(6)), rel=1e-12)
    assert pulse.flat_top_envelope(tau - 6 * s, A, tr, tau) == pytest.approx(A / 2, rel=1e-12)


def test_two_segment_shape():
    A1, A2, tsw, trs, tfl, tsm, tau = 0.3, 0.1, 20.0, 2.0, 3.0, 1.0, 40.0
    env = lambda t: pulse.two_segment_envelope(t, A1, A2, tsw, trs, tfl, tsm, tau)  # noqa: E731
    # plateaus (logistic tails exp(-distance/sigma) below 1e-6 here)
    assert env(10.0) == pytest.approx(A1, rel=1e-7)
    assert env(26.0) == pytest.approx(A2, rel=1e-6)
    assert env(tsw) == pytest.approx((A1 + A2) / 2, rel=1e-7)
    assert abs(env(0.0)) < 0.01 * A1 and abs(env(tau)) < 0.01 * A1


# ---------------------------------------------------------------- signal

def test_erfc_tabulated():
    for x, want in _read_golden("erfc_values.txt"):
        assert math.erfc(float(x)) == pytest.approx(float(want), rel=1e-14)


def test_assignment_error_constant_difference():
    dt, n, kappa, gamma, eta = 1e-3, 5000, 0.3, 2e-5, 0.6
    delta = 0.7 - 0.2j
    bg = np.full(n + 1, 0.1 + 0.3j)
    be = bg + delta
    tau = n * dt
    want_snr = math.sqrt(2 * eta * kappa * tau) * abs(delta)
    assert signal.snr(bg, be, dt, kappa, eta) == pytest.approx(want_snr, rel=1e-13)
    want = 0.5 * math.erfc(want_snr / 2) + tau * gamma / 2
    assert signal.assignment_error(bg, be, dt, kappa, gamma, eta) == pytest.approx(want, rel=1e-13)
    # SNR = 2 gives eps_sep = erfc(1)/2 exactly (Table 7.1 value)
    d2 = 4.0 / (2 * eta * kappa * tau)
    be2 = bg + math.sqrt(d2)
    erfc1 = float(_read_golden("erfc_values.txt")[1][1])
    assert signal.assignment_error(bg, be2, dt, kappa, 0.0, eta) == pytest.approx(erfc1 / 2, rel=1e-13)


def test_trapezoid_exact_for_linear():
    dt, n = 0.01, 300
    t = np.arange(n + 1) * dt
    # |beta_e - beta_g|^2 = 1 + 3t exactly
    be = np.sqrt(1 + 3 * t)
    got = signal.integrated_separation(np.zeros(n + 1), be, dt)
    T = n * dt
    assert got == pytest.approx(T + 1.5 * T * T, rel=1e-13)


# ---------------------------------------------------------------- RHS identities

def _zero(t):
    return 0.0


def test_lindblad_rhs_trace_and_hermiticity():
    mdl = small_model()
    Z = random_state(mdl.N, mdl.N, 1)
    rho = Z @ Z.conj().T
    rho /= np.trace(rho)
    c = lambda t: 0.37  # noqa: E731
    d = lindblad.lindblad_rhs(rho, 0.0, mdl, c)
    assert abs(np.trace(d)) < 1e-13
    assert np.allclose(d, d.conj().T, atol=1e-13)


def test_lindblad_rhs_matches_vectorised_superoperator():
    """Eq. S4 against the Liouvillian built with Kronecker products
    (row-major vec: vec(A X B) = (A kron B^T) vec(X))."""
    mdl = small_model(dims=(2, 3))
    N = mdl.N
    c = 0.21
    H = mdl.hamiltonian(c)
    I = np.eye(N)
    Lv = -1j * (np.kron(H, I) - np.kron(I, H.T))
    for L in mdl.jumps:
        LdL = L.conj().T @ L
        Lv += np.kron(L, L.conj()) - 0.5 * (np.kron(LdL, I) + np.kron(I, LdL.T))
    Z = random_state(N, N, 2)
    rho = Z @ Z.conj().T
    want = (Lv @ rho.reshape(-1)).reshape(N, N)
    got = lindblad.lindblad_rhs(rho, 0.0, mdl, lambda t: c)
    assert np.allclose(got, want, atol=1e-12 * np.abs(want).max())


def test_lowrank_rhs_equals_lindblad_at_full_rank():
    """O m^dag + m O^dag = sum_k D[L_k] m m^dag defines O (Sec. S1.A); at M = N
    the low-rank right-hand side must reproduce the full Lindblad one."""
    mdl = small_model()
    Z = random_state(mdl.N, mdl.N, 3)
    c = lambda t: -0.44  # noqa: E731
    F = lowrank.nosse_rhs(Z, 0.0, mdl, c)
    rho = Z @ Z.conj().T
    lhs = F @ Z.conj().T + Z @ F.conj().T
    want = lindblad.lindblad_rhs(rho, 0.0, mdl, c)
    assert np.allclose(lhs, want, atol=1e-11 * np.abs(want).max())


def test_lowrank_rhs_projected_identity():
    """For M < N: F m^dag + m F^dag = -i[H,rho] - 1/2 sum{L^dag L, rho}
    + 1/2 sum (P L rho L^dag + L rho L^dag P), P the projector onto span(m)."""
    mdl = small_model()
    Z = random_state(mdl.N, 4, 4)
    c = lambda t: 0.9  # noqa: E731
    F = lowrank.nosse_rhs(Z, 0.0, mdl, c)
    rho = Z @ Z.conj().T
    H = mdl.hamiltonian(0.9)
    P = Z @ np.linalg.pinv(Z)
    want = -1j * (H @ rho - rho @ H)
    loss = 0.0
    for L in mdl.jumps:
        LdL = L.conj().T @ L
        J = L @ rho @ L.conj().T
        want += -0.5 * (LdL @ rho + rho @ LdL) + 0.5 * (P @ J + J @ P)
        loss += np.trace((np.eye(mdl.N) - P) @ J).real
    got = F @ Z.conj().T + Z @ F.conj().T
    assert np.allclose(got, want, atol=1e-11 * np.abs(want).max())
    # trace-loss law of the projected equation
    assert np.trace(got).real == pytest.approx(-loss, rel=1e-10)
    assert loss > 0


def test_lowrank_gauge_covariance():
    mdl = small_model()
    Z = random_state(mdl.N, 5, 5)
    U, _ = np.linalg.qr(random_state(5, 5, 6))
    c = lambda t: 0.3  # noqa: E731
    F = lowrank.nosse_rhs(Z, 0.0, mdl, c)
    FU = lowrank.nosse_rhs(Z @ U, 0.0, mdl, c)
    assert np.allclose(FU, F @ U, atol=1e-12 * np.abs(F).max())


# ---------------------------------------------------------------- trajectories

def test_schrodinger_without_jumps():
    """kappa = gamma = 0: each column follows exp(-iHt) (constant drive)."""
    mdl = small_model(kappa=0.0, gamma=0.0)
    c0 = 0.5
    Z0 = random_state(mdl.N, 3, 7) * 0.2
    dt, n = 2e-3, 1500
    out = lowrank.integrate(Z0, mdl, lambda t: c0, dt, n, pop_every=n, return_state=True)
    U = sla.expm(-1j * mdl.hamiltonian(c0) * (n * dt))
    assert np.allclose(out["m"], U @ Z0, atol=1e-10)
    # RK4's amplification factor has |R(ihw)|^2 = 1 - (hw)^6/72 + ..., so the
    # norm is conserved only to ~n (h|H|)^6/72 (~1e-8 here)
    assert out["trace"][-1] == pytest.approx(out["trace"][0], rel=1e-7)


def _coherent_alpha(t, wr, kappa, eps, wd, phi):
    lam = 1j * wr + kappa / 2
    tot = 0j
    for s in (+1, -1):
        c = -1j * eps * np.exp(1j * s * phi) / 2
        tot += c * (np.exp(1j * s * wd * t) - np.exp(-lam * t)) / (1j * s * wd + lam)
    return tot


def test_driven_damped_resonator_coherent_amplitude():
    """Single driven damped mode from vacuum stays coherent; rank 1 is exact and
    <a>(t) follows the closed form of d alpha/dt = -(i wr + kappa/2) alpha - i c(t)."""
    wr, kappa, eps, wd, phi = 2 * math.pi * 0.5, 0.5, 0.5, 3.0, 0.4
    mdl = Model((1, 30), wq=0.0, alpha=0.0, wr=wr, g=0.0, kappa=kappa, gamma=0.0, dense=True)
    coef = lambda t: eps * math.cos(wd * t + phi)  # noqa: E731
    dt, n = 1e-3, 5000
    z0 = np.zeros((mdl.N, 1), complex)
    z0[0, 0] = 1
    out = lowrank.integrate(z0, mdl, coef, dt, n, pop_every=500)
    t = np.arange(n + 1) * dt
    want = _coherent_alpha(t, wr, kappa, eps, wd, phi)
    assert np.max(np.abs(out["beta"] - want)) < 1e-10
    assert np.max(np.abs(out["trace"] - 1)) < 1e-10   # RK4 truncation only
    # photon number of a coherent state is |alpha|^2
    assert np.allclose(out["nr"], np.abs(want[::500]) ** 2, atol=1e-10)
    # the full master equation reaches the same amplitude
    rho0 = z0 @ z0.conj().T
    full = lindblad.integrate(rho0, mdl, coef, dt, 1000, pop_every=1000)
    assert np.max(np.abs(full["beta"] - want[:1001])) < 1e-10


@pytest.mark.parametrize("M", [1, 2])
def test_lone_transmon_level_decay(M):
    """L = sqrt(gamma) b from |1>: P_1 = P_1(0) exp(-gamma t). Rank 1 also loses
    trace as exp(-gamma t); rank 2 = N keeps it."""
    # |lambda dt| = 0.015 keeps RK4's own error (~|lambda dt|^5/120 per step,
    # ~2e-9 relative at the end) below the 1e-8 tolerance
    gamma, dt, n = 0.2, 5e-3, 1000
    mdl = Model((2, 1), wq=3.0, alpha=0.0, wr=0.0, g=0.0,
                kappa=0.0, gamma=gamma, dense=True)
    # The padding column of weight eps receives the decayed population at the
    # rate d|c|/dt = gamma |a|^2 / (2|c|), i.e. a transient of rate gamma/(2 eps)
    # that fixed-step RK4 must resolve; eps = 0.05 keeps it at 2/ns.
    eps = 0.05
    m0 = init_state.initial_state(2, M, 1, eps, seed=1, traj=1)
    out = lowrank.integrate(m0, mdl, _zero, dt, n, pop_every=100)
    t = np.arange(0, n + 1, 100) * dt
    p1 = (1 - (M - 1) * eps) * np.exp(-gamma * t)
    assert np.allclose(out["pops"][:, 1], p1, rtol=1e-8, atol=0)
    if M == 1:
        assert np.allclose(out["trace"], np.exp(-gamma * t), rtol=1e-8)
    else:
        assert np.allclose(out["trace"], 1.0, atol=1e-8)
    full = lindblad.integrate(m0 @ m0.conj().T, mdl, _zero, dt, n, pop_every=100)
    assert np.allclose(full["pops"][:, 1], p1 if M == 2 else np.exp(-gamma * t), rtol=1e-8)


def _c1_like(dims=(3, 4)):
    return small_model(dims=dims, kappa=0.3, gamma=0.05)


def test_rk4_fourth_order():
    mdl = _c1_like()
    coef = lambda t: 0.8 * math.cos(2.9 * t)  # noqa: E731
    Z0 = init_state.initial_state(mdl.N, 3, 4, 1e-2, seed=9, traj=0)
    T = 2.0

    def run(dt):
        n = int(round(T / dt))
        return lowrank.integrate(Z0, mdl, coef, dt, n, pop_every=n, return_state=True)["m"]

    ref = run(0.0025)
    r = ref @ ref.conj().T
    e1 = np.abs(run(0.04) @ run(0.04).conj().T - r).max()
    e2 = np.abs(run(0.02) @ run(0.02).conj().T - r).max()
    assert 12 < e1 / e2 < 20


def test_full_rank_lowrank_converges_to_master_equation():
    """At M = N the low-rank trajectory and the full ME agree up to the RK4
    discretisation gap, which shrinks ~16x when dt halves."""
    mdl = _c1_like(dims=(2, 4))
    coef = lambda t: 1.1 * math.cos(3.1 * t + 0.2)  # noqa: E731
    Z0 = init_state.initial_state(mdl.N, mdl.N, 4, 1e-2, seed=2, traj=3)
    rho0 = Z0 @ Z0.conj().T
    T = 2.0
    gaps = []
    for dt in (0.04, 0.02):
        n = int(round(T / dt))
        a = lowrank.integrate(Z0, mdl, coef, dt, n, pop_every=n, return_state=True)
        b = lindblad.integrate(rho0, mdl, coef, dt, n, pop_every=n, return_state=True)
        gaps.append(np.abs(a["m"] @ a["m"].conj().T - b["rho"]).max())
    assert gaps[1] < 2e-5
    assert 12 < gaps[0] / gaps[1] < 20


def test_full_master_equation_positivity_and_trace():
    mdl = _c1_like()
    coef = lambda t: 1.5 * math.cos(3.0 * t)  # noqa: E731
    psi = np.zeros((mdl.N, 1), complex)
    psi[mdl.basis_index((1, 0))] = 1
    out = lindblad.integrate(psi @ psi.conj().T, mdl, coef, 0.01, 300, pop_every=100, return_state=True)
    rho = out["rho"]
    assert np.allclose(rho, rho.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(rho).min() > -1e-12
    assert np.allclose(out["trace"], 1.0, atol=1e-12)


def test_lowrank_trace_decreases_below_full_rank():
    mdl = _c1_like()
    coef = lambda t: 1.5 * math.cos(3.0 * t)  # noqa: E731
    Z0 = init_state.initial_state(mdl.N, 2, 4, 1e-3, seed=5, traj=0)
    out = lowrank.integrate(Z0, mdl, coef, 0.01, 300, pop_every=10)
    assert np.all(np.diff(out["trace"]) <= 1e-15)


# ---------------------------------------------------------------- gradient

def _tiny_workload(n_steps=1500, dt=2e-3):
    import lr_inputs as li
    m = li.ModelParams(dims=(3, 6), wq=2.0, alpha=-0.4, wr=3.0, g=0.5,
                       kappa=2.0, gamma=0.05)
    pul = li.PulseParams(0, (1.2, 3.05, 1.0, 0.3))
    return li.Workload("tiny", [li.Candidate(m, 3, pul)], dt, n_steps,
                       n_steps * dt, init_seed=11, eps=1e-3)


def test_fd_gradient_exact_on_polynomial_stand_in(monkeypatch):
    """fd_gradient against the exact central difference of a known polynomial.

    The workload runner is replaced by a stand-in whose eps_a is
        e(theta) = sum_i c_i theta_i + sum_i d_i theta_i^2 + e01 theta_0 theta_1
                   + sum_i k_i theta_i^3,
    for which the central difference with step h_i = rel |theta_i| is exactly
        c_i + 2 d_i theta_i + e01 theta_(1-i) [i < 2] + k_i (3 theta_i^2 + h_i^2).
    Perturbing the wrong component, a one-sided step (error d_i h_i ~ 1e-4
    relative), a step of h instead of 2h in the denominator, or an absolute
    instead of a relative step each miss this by far more than rounding.
    A zero parameter uses the absolute step rel."""
    th0 = np.array([1.3, -0.7, 2.9, 0.0, 4.1, 0.55, 47.0, 1.9])
    c = np.array([0.3, -1.1, 0.25, 0.8, -0.4, 1.7, 0.02, -0.6])
    d = np.array([0.9, 0.2, -0.35, 1.4, 0.15, -0.8, 0.003, 0.45])
    k = np.array([0.05, -0.02, 0.01, 0.3, 0.004, 0.07, 1e-5, -0.03])
    e01 = 0.37

    def e_of(th):
        th = np.asarray(th, dtype=float)
        return float(c @ th + d @ th ** 2 + e01 * th[0] * th[1] + k @ th ** 3)

    import lr_inputs as li
    m = li.ModelParams(dims=(2, 3), wq=2.0, alpha=-0.4, wr=3.0, g=0.3, kappa=0.5, gamma=0.1)
    wl = li.Workload("stand-in", [li.Candidate(m, 2, li.PulseParams(1, tuple(th0)))], 1e-3, 1, 1e-3,
                     init_seed=1)
    calls = []

    def fake_run(wl_, cand_index, n_steps=None, pop_every=1, theta=None, model=None):
        assert cand_index == 0
        th = wl_.candidates[0].pulse.p if theta is None else theta
        calls.append(np.array(th, dtype=float))
        return {"eps_a": e_of(th)}

    monkeypatch.setattr(gradient, "run_candidate", fake_run)
    rel = 1e-4
    got = gradient.fd_gradient(wl, 0, rel=rel)
    h = np.where(th0 != 0.0, rel * np.abs(th0), rel)
    want = c + 2.0 * d * th0 + k * (3.0 * th0 ** 2 + h ** 2)
    want[0] += e01 * th0[1]
    want[1] += e01 * th0[0]
    assert len(calls) == 2 * th0.size
    # every call moves exactly one component, by +h_i then -h_i
    for i in range(th0.size):
        dp, dm = calls[2 * i] - th0, calls[2 * i + 1] - th0
        assert np.count_nonzero(dp) == 1 and np.count_nonzero(dm) == 1
        assert dp[i] == pytest.approx(h[i], rel=1e-9) and dm[i] == pytest.approx(-h[i], rel=1e-9)
    # rounding: eps_a values of size ~1e2 differenced over h ~ 1e-4: ~1e-10
    assert np.abs(got - want).max() <= 1e-8 * max(1.0, np.abs(want).max())
    # the one-sided difference would be off by d_i h_i: far above the bound
    assert np.abs(d * h).max() > 1e3 * 1e-8 * max(1.0, np.abs(want).max())


def test_fd_gradient_richardson_consistent():
    """Central differences at h and h/2 agree to O(h^2) (smooth eps_a)."""
    wl = _tiny_workload()
    g1 = gradient.fd_gradient(wl, 0, rel=1e-4)
    g2 = gradient.fd_gradient(wl, 0, rel=5e-5)
    assert np.all(np.isfinite(g1)) and np.abs(g1).max() > 1e-3
    assert np.allclose(g1, g2, rtol=1e-5, atol=1e-7 * np.abs(g1).max())


# ---------------------------------------------------------------- loss / SPSA (Sec. S3.B/C)

def test_ionization_closed_forms():
    n, dt_rec, tau = 41, 0.25, 10.0
    t = np.arange(n) * dt_rec
    pg = np.zeros((n, 4))
    pe = np.zeros((n, 4))
    pg[:, 2] = 0.01                      # constant level-2 population
    pe[:, 3] = 0.002 * t                 # linear level-3 population (trapezoid exact)
    pe[:, 1] = 0.7                       # levels < 2 do not count
    want = (0.01 * t[-1] + 0.001 * t[-1] ** 2) / tau
    assert signal.ionization(pg, pe, dt_rec, tau) == pytest.approx(want, rel=1e-13)
    assert signal.loss(1e-3, 0.0) == pytest.approx(-3.0, abs=1e-15)


def test_spsa_step_on_quadratic():
    """One SPSA step on L = sum_i (theta_i - t_i)^2 / s_i^2 equals the closed form
    g_i = sum_j 2 s_j Delta_j (theta_j - t_j)/s_j^2 / Delta_i (exact difference of
    a quadratic), and the loss decreases along the chain."""
    from oracle import spsa
    target = np.array([0.3, 47.2, 2.0, 1.0])
    scale = np.array([0.05, 0.01, 0.2, 0.1])
    th0 = np.array([0.5, 47.25, 2.5, 1.3])

    def L(th):
        return float(np.sum(((th - target) / scale) ** 2))
    rng = np.random.default_rng(3)
    deltas = rng.choice([-1.0, 1.0], size=(60, 4))
    hist, losses = spsa.spsa(lambda a, b: (L(a), L(b)), 0, th0, deltas, scale, a=0.5, c=0.1, A=5.0)
    ak, ck = spsa.gains(0, 0.5, 0.1, 5.0)
    d0 = deltas[0]
    gq = np.sum(2 * scale * d0 * (th0 - target) / scale ** 2) / d0
    assert np.allclose(hist[1], th0 - ak * scale * gq, rtol=1e-12, atol=1e-12)
    assert L(hist[-1]) < 1e-6 * L(hist[0])


# ---------------------------------------------------------------- diagnostics (Sec. S1.B)

def test_diagnostics_gram_forms_equal_rho_forms():
    """The M x M Gram forms of the spectrum and purity equal the N x N
    definitions on rho = m m^dag (independent computations)."""
    rng = np.random.default_rng(11)
    m = rng.normal(size=(30, 5)) + 1j * rng.normal(size=(30, 5))
    G = m.conj().T @ m
    assert np.allclose(diagnostics.gram_spectrum(G), diagnostics.rho_spectrum(m), rtol=1e-12, atol=0)
    assert abs(diagnostics.gram_purity(G) - diagnostics.rho_purity(m)) < 1e-11 * diagnostics.rho_purity(m)
    # rho beyond rank M has no further nonzero eigenvalues
    rho = m @ m.conj().T
    assert np.abs(np.linalg.eigvalsh(rho)[:-5]).max() < 1e-10 * np.abs(rho).max()


@pytest.mark.parametrize("M", [1, 4, 20])
def test_diagnostics_initial_state_closed_forms(M):
    """Fixed-rank initial state (Sec. S1.A): eigenvalues 1 - (M-1) eps (once)
    and eps (M-1 times), purity (1-(M-1)eps)^2 + (M-1) eps^2, and the rank
    indicator p_M / p_1 = eps / (1 - (M-1) eps)."""
    eps = 1e-5
    m = init_state.initial_state(200, M, 7, eps, seed=3, traj=1)
    p0 = 1.0 - (M - 1) * eps
    want = np.array([p0] + [eps] * (M - 1))
    got = diagnostics.rho_spectrum(m)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-16)
    assert abs(diagnostics.rho_purity(m) - (p0 ** 2 + (M - 1) * eps ** 2)) < 1e-13
    g = diagnostics.gram_spectrum(m.conj().T @ m)
    assert abs(g[-1] / g[0] - (eps / p0 if M > 1 else 1.0)) < 1e-9 * (eps / p0 if M > 1 else 1.0)


def test_diagnostics_full_rank_purity_matches_master_equation():
    """At M = N the low-rank purity follows the full ME's tr(rho^2) up to the
    RK4 gap (Eq. S4 vs Eq. S5), and decays under the jumps from a pure-ish start."""
    mdl = _c1_like(dims=(2, 4))
    coef = lambda t: 1.1 * math.cos(3.1 * t + 0.2)  # noqa: E731
    Z0 = init_state.initial_state(mdl.N, mdl.N, 4, 1e-2, seed=2, traj=3)
    n, dt = 100, 0.02
    a = lowrank.integrate(Z0, mdl, coef, dt, n, pop_every=n, return_state=True, gram=True)
    b = lindblad.integrate(Z0 @ Z0.conj().T, mdl, coef, dt, n, pop_every=n, return_state=True)
    pur_lra = diagnostics.gram_purity(a["gram"][-1])
    pur_me = float(np.trace(b["rho"] @ b["rho"]).real)
    assert abs(pur_lra - pur_me) < 1e-5
    assert diagnostics.gram_purity(a["gram"][0]) > pur_lra


# ---------------------------------------------------------------- rotating frame + RWA (Sec. S2)

def _excitation_number(mdl):
    """N = b^dag b + a^dag a [+ f^dag f] on the product basis (diagonal)."""
    levels = np.array(np.unravel_index(np.arange(mdl.N), mdl.dims)).sum(axis=0)
    return levels.astype(float)


@pytest.mark.parametrize("dims", [(3, 4), (3, 3, 2)])
def test_rwa_hamiltonian_is_excitation_conserving_part(dims):
    """The RWA Hamiltonian equals the part of H_lab - w_d N that conserves the
    excitation number N (the blocks N -> N of the lab Hamiltonian in the frame
    rotating at w_d); the counter-rotating terms are the N -> N+-2 blocks."""
    wd = 2.7
    lab = small_model(dims)
    rwa = Model(dims, wq=2.0, alpha=-0.4, wr=3.0, g=0.3, kappa=0.5, gamma=0.2, wf=3.2, J=0.25,
                dense=True, rwa=(wd, 0.0))
    nexc = _excitation_number(lab)
    shifted = lab.H0 - wd * np.diag(nexc)
    secular = np.where(nexc[:, None] == nexc[None, :], shifted, 0.0)
    assert np.allclose(rwa.H0, secular, atol=1e-13)
    assert np.abs(shifted - secular).max() > 0.1     # the lab model has counter-rotating terms


def test_rwa_drive_is_period_average_of_rotated_lab_drive():
    """(1/T) int_0^T U(t) cos(w_d t + phi) (r + r^dag) U(t)^dag dt with
    U = exp(i w_d t N), T = 2 pi / w_d, equals (1/2)(e^{i phi} r + e^{-i phi} r^dag)."""
    wd, phi = 2.3, 0.7
    lab = small_model((2, 3, 3))
    rwa = Model((2, 3, 3), wq=2.0, alpha=-0.4, wr=3.0, g=0.3, kappa=0.5, gamma=0.2, wf=3.2, J=0.25,
                dense=True, rwa=(wd, phi))
    nexc = _excitation_number(lab)
    T, K = 2 * math.pi / wd, 4000
    avg = np.zeros_like(lab.Xd)
    for k in range(K):       # rectangle rule: exact for trigonometric polynomials of degree < K
        t = k * T / K
        u = np.exp(1j * wd * t * nexc)
        avg += (u[:, None] * lab.Xd * u.conj()[None, :]) * math.cos(wd * t + phi) / K
    assert np.allclose(avg, 0.5 * rwa.Xd, atol=1e-12)


def test_rwa_driven_damped_resonator_closed_form():
    """Rotating frame, constant drive (Omega/2)(e^{i phi} a + e^{-i phi} a^dag),
    detuning Delta: <a>(t) = a_ss (1 - exp(-(i Delta + kappa/2) t)),
    a_ss = -i (Omega/2) e^{-i phi} / (i Delta + kappa/2); rank 1 is exact."""
    wr, wd, kappa, om, phi = 5.0, 4.6, 0.5, 0.8, 0.3
    mdl = Model((1, 30), wq=0.0, alpha=0.0, wr=wr, g=0.0, kappa=kappa, gamma=0.0, dense=True, rwa=(wd, phi))
    coef = lambda t: 0.5 * om  # noqa: E731
    dt, n = 2e-3, 4000
    z0 = np.zeros((mdl.N, 1), complex)
    z0[0, 0] = 1
    out = lowrank.integrate(z0, mdl, coef, dt, n, pop_every=400)
    t = np.arange(n + 1) * dt
    lam = 1j * (wr - wd) + 0.5 * kappa
    want = -1j * 0.5 * om * np.exp(-1j * phi) / lam * (1 - np.exp(-lam * t))
    assert np.max(np.abs(out["beta"] - want)) < 1e-10
    assert np.allclose(out["nr"], np.abs(want[::400]) ** 2, atol=1e-10)


def test_rwa_tracks_lab_frame_for_a_weak_near_resonant_drive():
    """Physics check of the approximation: for a weak drive near resonance
    (Omega, |w_r - w_d| << w_d) the lab-frame amplitude times e^{i w_d t}
    follows the RWA amplitude to O(Omega / w_d)."""
    wr, wd, kappa, om, phi = 30.0, 29.7, 0.5, 0.3, 0.3
    lab = Model((1, 12), wq=0.0, alpha=0.0, wr=wr, g=0.0, kappa=kappa, gamma=0.0, dense=True)
    rwa = Model((1, 12), wq=0.0, alpha=0.0, wr=wr, g=0.0, kappa=kappa, gamma=0.0, dense=True, rwa=(wd, phi))
    dt, n = 5e-4, 8000
    z0 = np.zeros((lab.N, 1), complex)
    z0[0, 0] = 1
    a = lowrank.integrate(z0, lab, lambda t: om * math.cos(wd * t + phi), dt, n, pop_every=n)
    b = lowrank.integrate(z0, rwa, lambda t: 0.5 * om, dt, n, pop_every=n)
    t = np.arange(n + 1) * dt
    diff = np.abs(a["beta"] * np.exp(1j * wd * t) - b["beta"]).max()
    assert diff < 3 * om / wd * np.abs(b["beta"]).max()


def _shot_signals(n=1500, dt=0.01):
    """A readout pair with a closed form: beta_g = 0, beta_e = A (1 - e^{-t/t0}) e^{i phi}."""
    t = np.arange(n + 1) * dt
    be = 0.8 * (1.0 - np.exp(-t / 2.0)) * np.exp(0.7j)
    return np.zeros(n + 1, np.complex128), be, dt


def test_assignment_shots_bins_of_one_step_are_the_trapezoid_snr():
    bg, be, dt = _shot_signals()
    kappa, gamma, eta = 0.9, 2e-4, 0.6
    r = signal.assignment_shots(bg, be, dt, kappa, gamma, eta, 16, 1, 7, 0)
    assert r["eps_bin"] == pytest.approx(signal.assignment_error(bg, be, dt, kappa, gamma, eta), rel=1e-13)
    assert r["snr_bin"] == pytest.approx(signal.snr(bg, be, dt, kappa, eta), rel=1e-13)


def test_assignment_shots_binning_loses_snr_except_for_a_constant_difference():
    """Cauchy-Schwarz: |q_b|^2 / W_b <= sum_b w |Delta|^2, equality for a constant
    difference Delta, where SNR_b = sqrt(2 eta kappa tau) |Delta| (the closed form)."""
    bg, be, dt = _shot_signals()
    r1 = signal.assignment_shots(bg, be, dt, 0.9, 0.0, 0.6, 4, 1, 1, 0)
    r50 = signal.assignment_shots(bg, be, dt, 0.9, 0.0, 0.6, 4, 50, 1, 0)
    assert r50["snr_bin"] < r1["snr_bin"]
    n, delta = 1500, 0.3 - 0.4j
    const = np.full(n + 1, delta)
    rc = signal.assignment_shots(np.zeros(n + 1), const, dt, 0.9, 0.0, 0.6, 4, 37, 1, 0)
    assert rc["snr_bin"] == pytest.approx(math.sqrt(2 * 0.6 * 0.9 * n * dt) * abs(delta), rel=1e-12)


def test_assignment_shots_converge_to_the_closed_form():
    """The misassignment rate of 40,000 seeded shots per state lies within four
    binomial standard deviations of erfc(SNR_b / 2) / 2; the noise statistic N
    has the variance D / (2 sqrt(2 eta kappa)) of the definition; the decay
    term tau gamma / 2 is added to both."""
    bg, be, dt = _shot_signals()
    kappa, gamma, eta, ns = 0.25, 1e-3, 0.6, 40000
    r = signal.assignment_shots(bg, be, dt, kappa, gamma, eta, ns, 25, 20250818, 3)
    dec = 0.5 * 1500 * dt * gamma
    p = r["eps_bin"] - dec
    assert 0.02 < p < 0.3                      # a regime where the rate is measurable
    got = r["eps_shots"] - dec
    assert abs(got - p) <= 4.0 * math.sqrt(p * (1 - p) / (2 * ns)), (got, p)
    var = np.var(np.concatenate([r["T_g"] + 0.5 * r["D"], r["T_e"] - 0.5 * r["D"]]))
    assert var == pytest.approx(r["D"] / (2 * math.sqrt(2 * eta * kappa)), rel=0.03)
    # the two states use different noise, the same seed gives the same shots
    assert not np.array_equal(r["T_g"] + 0.5 * r["D"], r["T_e"] - 0.5 * r["D"])
    r2 = signal.assignment_shots(bg, be, dt, kappa, gamma, eta, 64, 25, 20250818, 3)
    r3 = signal.assignment_shots(bg, be, dt, kappa, gamma, eta, 64, 25, 20250818, 3)
    assert np.array_equal(r2["T_g"], r3["T_g"]) and np.array_equal(r2["T_e"], r3["T_e"])
