"""Pins of the oracle for the paper's normal-mode model (Sec. S2.A, S2.D, S2.E).

Each test checks the oracle against something other than itself: Mathieu
characteristic values, the qubit figures printed in Sec. S2.B, the closed form
of two momentum-coupled oscillators, Fock-space commutators, the frame map
between the lab and rotated frames, and the full master equation.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import paper_model as pm

TP = 2.0 * np.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    out = {}
    with open(os.path.join(GOLDEN, "paper_model_sec_s2b.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def _paper_params():
    g = _golden()
    Ec = TP * g["Ec"]
    return dict(Ec=Ec, Ej=g["Ej_over_Ec"] * Ec, wr=TP * g["wr"], wf=TP * g["wf"], g=TP * g["g"],
                J=TP * g["J"], kappa=TP * g["kappa"], gamma=TP * g["gamma"], wd=TP * g["wd"])


@pytest.mark.parametrize("ratio", [51.0, 20.0])
def test_transmon_spectrum_is_mathieu(ratio):
    """4 Ec n^2 - Ej cos(phi) with 2pi-periodic states: with phi = 2x the
    equation is Mathieu's with a = E / Ec and q = -Ej / (2 Ec); the periodic
    solutions of period pi have characteristic values a_0, b_2, a_2, b_4, ..."""
    from scipy.special import mathieu_a, mathieu_b
    Ec = TP * 0.315
    Ej = ratio * Ec
    w, _ = pm.transmon(Ec, Ej, 6, n_cut=20)
    q = -Ej / (2.0 * Ec)
    chars = [mathieu_a(0, q)] + [mathieu_a(2 * k, q) for k in range(1, 5)] + [mathieu_b(2 * k, q) for k in range(1, 5)]
    want = Ec * np.sort(chars)[:6]
    assert np.allclose(w, want, rtol=0, atol=1e-9 * np.abs(want).max())


def test_transmon_charge_matrix():
    Ec = TP * 0.315
    Ej = 51.0 * Ec
    _, n = pm.transmon(Ec, Ej, 6)
    assert np.allclose(n, n.T)
    for j in range(6):
        for k in range(6):
            if (j + k) % 2 == 0:       # parity: n connects levels of opposite parity only
                assert abs(n[j, k]) < 1e-10
    assert all(n[j, j + 1] > 0 for j in range(5))
    # transmon limit (harmonic oscillator in phi): <0|n|1> -> (Ej / 8 Ec)^{1/4} / sqrt(2)
    assert abs(n[0, 1] / ((Ej / (8 * Ec)) ** 0.25 / np.sqrt(2.0)) - 1.0) < 0.05
    # more levels from a wider charge basis do not move the low ones
    w20, _ = pm.transmon(Ec, Ej, 6, n_cut=20)
    w30, _ = pm.transmon(Ec, Ej, 6, n_cut=30)
    assert np.abs(w20 - w30).max() < 1e-10


def test_normal_mode_frequencies_closed_form():
    """With a^dag - a = -i sqrt(2) p_a, H_rf = sum w (x^2 + p^2)/2 + 2 J p_a p_f, so
    x_a'' = -wr^2 x_a - 2 J wf x_f, x_f'' = -wf^2 x_f - 2 J wr x_a: the normal
    frequencies squared are the eigenvalues of [[wr^2, 2 J wf], [2 J wr, wf^2]]."""
    for wr, wf, J in ((TP * 7.2, TP * 7.21, TP * 0.03), (TP * 5.0, TP * 6.5, TP * 0.4)):
        wl, wu = pm.normal_modes(wr, wf, J)[:2]
        m = (wr ** 2 + wf ** 2) / 2
        d = np.sqrt(((wr ** 2 - wf ** 2) / 2) ** 2 + 4 * J ** 2 * wr * wf)
        assert abs(wl - np.sqrt(m - d)) < 1e-12 * wl
        assert abs(wu - np.sqrt(m + d)) < 1e-12 * wu


def test_normal_modes_diagonalise_h_rf_in_fock_space():
    """[H_rf, c_i] = -w_i c_i on the low Fock states of a 14 x 14 truncation."""
    wr, wf, J = TP * 7.2, TP * 7.21, TP * 0.3
    wl, wu, U, S, *_ = pm.normal_modes(wr, wf, J)
    d = 14
    lad = sp.diags(np.sqrt(np.arange(1, d)), 1, shape=(d, d)).toarray()
    I = np.eye(d)
    a, f = np.kron(lad, I), np.kron(I, lad)
    ad, fd = a.T, f.T
    H = wr * ad @ a + wf * fd @ f - J * (ad - a) @ (fd - f)
    low = [i * d + j for i in range(4) for j in range(4)]
    for col, w in ((2, wl), (3, wu)):
        al, be, ga, de = U[:, col]
        c = al * a + be * f + ga * ad + de * fd
        R = H @ c - c @ H + w * c
        assert np.abs(R[:, low]).max() < 1e-9 * w
    # the bare operators in terms of the normal ones: a = sum_i (alpha_i c_i - gamma_i c_i^dag)
    # gives s13 = alpha_l, s12 = -gamma_l, s14 = alpha_u, s11 = -gamma_u (and beta, delta for f)
    for row, (x, y) in ((0, (0, 2)), (1, (1, 3))):
        assert abs(S[row, 2] - U[x, 2]) < 1e-12 and abs(S[row, 1] + U[y, 2]) < 1e-12
        assert abs(S[row, 3] - U[x, 3]) < 1e-12 and abs(S[row, 0] + U[y, 3]) < 1e-12


def test_bogoliubov_preserves_commutators():
    """S Sigma_c S^T = Sigma_a (Sec. S2.D), for c = (c_u^dag, c_l^dag, c_l, c_u)."""
    S = pm.normal_modes(TP * 7.2, TP * 7.21, TP * 0.03)[3]
    sx = np.array([[0.0, 1.0], [1.0, 0.0]])
    Z2 = np.zeros((2, 2))
    Sa = np.block([[Z2, np.eye(2)], [-np.eye(2), Z2]])
    Sc = np.block([[Z2, -sx], [sx, Z2]])
    assert np.abs(S @ Sc @ S.T - Sa).max() < 1e-12


def test_dressed_qubit_matches_printed_figures():
    """Sec. S2.B prints the qubit frequency (6 GHz) and anharmonicity (-349 MHz)
    for its parameters: the dressed levels |g,0,0>, |e,0,0>, |f,0,0> of the
    undriven lab-frame model reproduce both (the bare transmon alone gives
    6.030 GHz and -361 MHz, so the coupling through mu_l, mu_u is tested too)."""
    g = _golden()
    P = _paper_params()
    Nl, Nu, Nt = 8, 4, 6
    M = pm.PaperModel(Nl, Nu, Nt, frame="lab", **P)
    H = M.h_terms[pm.channel_index(0, 0)].toarray()
    w, v = np.linalg.eigh(H)
    E = []
    for j in range(3):
        k = np.argmax(np.abs(v[j, :]) ** 2)       # |0_l, 0_u, j> has flat index j
        assert np.abs(v[j, k]) ** 2 > 0.95
        E.append(w[k])
    assert abs((E[1] - E[0]) / TP - g["qubit_frequency"]) < 0.01
    assert abs((E[2] - 2 * E[1] + E[0]) / TP - g["anharmonicity"]) < 0.0005
    wb, _ = pm.transmon(P["Ec"], P["Ej"], 3)
    assert abs((wb[2] - 2 * wb[1] + wb[0]) / TP - g["anharmonicity"]) > 0.01


def _small(frame, **over):
    P = dict(Ec=TP * 0.315, Ej=51 * TP * 0.315, wr=TP * 7.2, wf=TP * 7.21, g=TP * 0.4, J=TP * 0.2,
             kappa=2.0, gamma=0.3, wd=TP * 7.18)
    P.update(over)
    return pm.PaperModel(3, 2, 3, frame=frame, **P)


def test_rotated_hamiltonian_is_hermitian():
    M = _small("rot")
    for t, om in ((0.013, 1.7), (0.41, -0.6)):
        H = M.hamiltonian(t, om).toarray()
        assert np.abs(H - H.conj().T).max() < 1e-12
        A = sum(pm.channel_values(t, om, M.wd)[k] * X for k, X in M.heff_terms().items()).toarray()
        Ls = [L.toarray() for L in M.jumps(t, om)]
        want = -1j * H - 0.5 * sum(L.conj().T @ L for L in Ls)
        assert np.abs(A - want).max() < 1e-12


def test_rotated_frame_equals_lab_frame():
    """rho_rot(t) = V rho_lab(t) V^dag with V = exp(i w_d t N_exc): the rotated
    operators (coupling, drive, and the time-dependent jump operator) are the
    lab ones seen from the frame of the drive."""
    lab, rot = _small("lab"), _small("rot")
    env = lambda t: 3.0 * np.sin(2.0 * t) ** 2  # noqa: E731
    psi = np.zeros(lab.N, dtype=complex)
    psi[1] = 1.0                                    # |0_l, 0_u, e>
    rho0 = np.outer(psi, psi.conj())
    dt, n = 2.5e-4, 2400
    out_l = pm.integrate(rho0, lab, env, dt, n, pop_every=n, low_rank=False, return_state=True)
    out_r = pm.integrate(rho0, rot, env, dt, n, pop_every=n, low_rank=False, return_state=True)
    t = n * dt
    V = np.diag(np.exp(1j * lab.wd * t * lab.n_exc))
    want = V @ out_l["state"] @ V.conj().T
    assert np.abs(out_r["state"] - want).max() < 2e-7
    assert np.abs(out_r["state"] - out_l["state"]).max() > 1e-2    # the frames do differ
    assert np.allclose(out_r["pops"], out_l["pops"], atol=2e-7)
    # the filter field: beta_rot(t) = e^{i w_d t} tr(rho_lab f), photons equal
    tt = dt * np.arange(n + 1)
    assert np.abs(out_r["beta"] - np.exp(1j * lab.wd * tt) * out_l["beta"]).max() < 2e-7
    assert np.abs(out_l["beta"]).max() > 1e-2
    assert np.allclose(out_r["nr"], out_l["nr"], atol=2e-7)


def test_lowrank_at_full_rank_is_the_master_equation():
    """Eq. S5 at M = N reproduces Eq. S4 with the time-dependent L_1(t)."""
    rot = _small("rot")
    env = lambda t: 2.0 * np.cos(3.0 * t)  # noqa: E731
    rng = np.random.default_rng(5)
    m0 = rng.standard_normal((rot.N, rot.N)) + 1j * rng.standard_normal((rot.N, rot.N))
    m0 /= np.sqrt(np.sum(np.abs(m0) ** 2))
    dt, n = 5e-4, 400      # two RK4 discretisations of one flow: they agree to O(dt^4)
    lr = pm.integrate(m0, rot, env, dt, n, pop_every=50, low_rank=True, return_state=True)
    me = pm.integrate(m0 @ m0.conj().T, rot, env, dt, n, pop_every=50, low_rank=False, return_state=True)
    m = lr["state"]
    assert np.abs(m @ m.conj().T - me["state"]).max() < 1e-9
    assert np.abs(lr["beta"] - me["beta"]).max() < 1e-9
    assert np.abs(lr["pops"] - me["pops"]).max() < 1e-9
    assert me["trace"][-1] == pytest.approx(1.0, abs=1e-9)


def test_heff_channels_follow_the_jump_phases():
    """The e^{2i w_d t} channel of -i H_eff carries -kappa/2 A^dag B of L_1^dag L_1:
    <2_l, 0_u, g| A^dag B |0_l, 0_u, g> = s23 s22 <2|c_l^dag c_l^dag|0> = sqrt(2) s23 s22
    (the Hamiltonian's e^{2i w_d t} terms change the transmon level, so they do not
    reach this element)."""
    rot = _small("rot")
    T = rot.heff_terms()
    assert pm.channel_index(0, 2) in T and pm.channel_index(0, -2) in T
    S = rot.S
    s22, s23 = S[1, 1], S[1, 2]
    Nl, Nu, Nt = rot.dims
    dst = (2 * Nu + 0) * Nt + 0
    got = T[pm.channel_index(0, 2)].toarray()[dst, 0]
    assert abs(got - (-0.5 * rot.kappa * s23 * s22 * np.sqrt(2.0))) < 1e-12
    assert abs(s22) > 1e-4                            # the counter-rotating part is not zero


def test_rwa_operators_are_the_period_average_of_the_rotated_ones():
    """Eq. S(hamiltonian_rwa) drops the explicitly time-dependent terms of Eq.
    S(hamiltonian_rotated): at a fixed envelope, H_rwa is the average of
    H_rot(t) over one period pi / w_d of the e^{+-2i w_d t} factors, and the RWA
    jump operator and readout are the averages of L_1(t) and r(t). The average
    is taken by the trapezoid rule on 16 equal steps (exact for trigonometric
    polynomials of degree < 16)."""
    rot, rwa = _small("rot"), _small("rwa")
    T = np.pi / rot.wd
    ts = 0.37 + T * np.arange(16) / 16.0
    for om in (0.0, 1.3):
        Hbar = sum(rot.hamiltonian(t, om) for t in ts) / 16.0
        assert np.abs((Hbar - rwa.hamiltonian(0.37, om)).toarray()).max() < 1e-12
        Lbar = sum(rot.jumps(t, om)[0] for t in ts) / 16.0
        assert np.abs((Lbar - rwa.jumps(0.37, om)[0]).toarray()).max() < 1e-12
        Rbar = sum(rot.readout(t, om) for t in ts) / 16.0
        assert np.abs((Rbar - rwa.readout(0.37, om)).toarray()).max() < 1e-12
    # the RWA generator is static in time at fixed envelope; the rotated one is not
    assert np.abs((rwa.hamiltonian(0.1, 1.0) - rwa.hamiltonian(0.9, 1.0)).toarray()).max() == 0.0
    assert np.abs((rot.hamiltonian(0.1, 1.0) - rot.hamiltonian(0.13, 1.0)).toarray()).max() > 1e-3
    # and -i H_eff keeps only the slow part of L_1^dag L_1
    assert all(k in (pm.channel_index(0, 0), pm.channel_index(1, 0)) for k in rwa.heff_terms())


def test_rwa_tracks_the_rotated_frame():
    """With g, Omega << w_d the RWA dynamics follows the rotated-frame dynamics
    up to corrections of order (g, Omega) / w_d: populations and |beta| of a
    resonantly driven run agree to a few percent, and differ (the dropped terms
    are not zero)."""
    rot, rwa = _small("rot", g=TP * 0.05), _small("rwa", g=TP * 0.05)
    env = lambda t: TP * 0.2 * min(1.0, t / 0.5)  # noqa: E731
    psi = np.zeros(rot.N, dtype=complex)
    psi[1] = 1.0
    rho0 = np.outer(psi, psi.conj())
    dt, n = 2.5e-4, 8000
    a = pm.integrate(rho0, rot, env, dt, n, pop_every=400, low_rank=False)
    b = pm.integrate(rho0, rwa, env, dt, n, pop_every=400, low_rank=False)
    bs = np.abs(a["beta"]).max()
    assert bs > 1e-2
    d = np.abs(a["beta"] - b["beta"]).max() / bs
    assert 1e-4 < d < 0.1, d
    assert np.abs(a["pops"] - b["pops"]).max() < 0.02
