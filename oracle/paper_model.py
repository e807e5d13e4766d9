"""The paper's own readout model in its normal-mode basis (oracle; test
infrastructure only).

Sec. S2.A (Hilbert space), S2.D (normal modes of the resonator-filter pair)
and S2.E (frame of the drive, Eq. S(hamiltonian_rotated)).

Transmon (Sec. S2.A): H_t = 4 E_c n^2 - E_j cos(phi), diagonalised in the
charge basis |n>, n = -n_cut..n_cut, where cos(phi) = (|n><n+1| + h.c.)/2
(offset charge zero). The lowest N_t eigenstates |j> give the energies eps_j
and the charge matrix n_jk = <j|n|k>. Eigenvector signs: n_{j,j+1} > 0.

Normal modes (Sec. S2.D): the 4 x 4 matrix Omega acting on the coefficients
(alpha, beta, gamma, delta) of c = alpha a + beta f + gamma a^dag + delta f^dag
is diagonalised; the positive eigenvalues are w_l < w_u. Each positive-
frequency eigenvector is normalised to alpha^2 + beta^2 - gamma^2 - delta^2 = 1
with beta > 0 (the sign convention of this build); the negative-frequency
columns are their adjoint partners (gamma, delta, alpha, beta). U holds the
columns in the order (c_u^dag, c_l^dag, c_l, c_u), S = inv(U^T), and
mu_u = s14 - s11, mu_l = s13 - s12, nu_u = s24 - s21, nu_l = s23 - s22.

Hilbert space: |j_l> (x) |j_u> (x) |j_t>, flat index n = (j_l N_u + j_u) N_t + j_t.

Frame of the drive (Sec. S2.E). Readings of this build: the frame maps
psi_rot = V psi_lab with V = exp(i w_d t N_exc), N_exc = c_l^dag c_l +
c_u^dag c_u + sum_j j |j><j| (so that c -> c e^{-i w_d t} as the paper
states; global phases dropped); n_t^+ = sum_j n_{j,j+1} |j><j+1| and
n_t^- = (n_t^+)^dag keep only nearest neighbours, as the paper's
approximation does; the drive envelope Omega(t) is real (the flat-top and
two-segment forms), the pulse phase is not used, and the drive frequency is
the frame's w_d. Then

  H_rot(t) = H_t' + H_rf'
           + sum_x i g mu_x (n^+ c_x^dag - n^- c_x - n^+ c_x e^{-2i w_d t}
                              + n^- c_x^dag e^{2i w_d t})
           - sum_x (nu_x / 2) Omega(t) (c_x^dag + c_x - c_x^dag e^{2i w_d t}
                                         - c_x e^{-2i w_d t}),

  H_t' = sum_j (eps_j - eps_0 - j w_d) |j><j|,
  H_rf' = (w_l - w_d) c_l^dag c_l + (w_u - w_d) c_u^dag c_u,

x in {l, u}. Dissipators (Eq. 2): kappa D[f] + gamma D[b]. In the rotated
frame f = s21 c_u^dag + s22 c_l^dag + s23 c_l + s24 c_u picks up phases; with a
global phase removed (D[L] and the low-rank O[m] do not see it)

  L_1(t) = sqrt(kappa) (A + e^{2i w_d t} B),
  A = s23 c_l + s24 c_u,   B = s21 c_u^dag + s22 c_l^dag,

kept exactly (no secular approximation). L_2 = sqrt(gamma) b with the
transmon lowering operator b = sum_j sqrt(j) |j-1><j| in the eigenbasis (a
reading: the paper names b without a matrix form); V only multiplies it by a
phase. The readout signal is the filter field, beta = tr(rho f) (the caption of
Fig. 2; the SNR of Sec. S3.A uses the filter rate kappa). In the rotated frame
the operator is f(t) = A + e^{2i w_d t} B, the lab-frame f seen from the frame
times e^{i w_d t}: beta_rot(t) = e^{i w_d t} beta_lab(t), so |beta_e - beta_g|
and the photon number tr(rho f^dag f) are those of the lab frame.

Every operator is stored as a sum over time channels (a, q):
X(t) = sum Omega(t)^a e^{i q w_d t} X_{a,q}, a in {0, 1}, q in {-2..2}.

Parity: the transmon spectrum against Mathieu characteristic values and the
paper's printed qubit frequency and anharmonicity (Sec. S2.B); the normal-mode
frequencies against the closed form of two momentum-coupled oscillators and
the commutator [H_rf, c_i] = -w_i c_i in Fock space; S against the
commutation relations (Sec. S2.D); H_rot against the lab-frame model through
the frame map; the low-rank equation at M = N against the full master
equation with the same time-dependent operators (tests).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .lowrank import rk4_step

CHANNELS = [(a, q) for a in (0, 1) for q in (-2, -1, 0, 1, 2)]   # index = 5 a + q + 2


def channel_index(a: int, q: int) -> int:
    return 5 * a + q + 2


def channel_values(t: float, omega: float, wd: float) -> np.ndarray:
    """chi_{a,q}(t) = Omega(t)^a e^{i q w_d t} for the ten channels."""
    return np.array([(omega if a else 1.0) * np.exp(1j * q * wd * t) for a, q in CHANNELS])


# ---------------------------------------------------------------- transmon --
def transmon(Ec: float, Ej: float, Nt: int, n_cut: int = 20):
    """Lowest Nt energies eps_j and the charge matrix n_jk of 4 Ec n^2 - Ej cos(phi)."""
    n = np.arange(-n_cut, n_cut + 1, dtype=float)
    H = np.diag(4.0 * Ec * n ** 2)
    off = -0.5 * Ej * np.ones(2 * n_cut)
    H += np.diag(off, 1) + np.diag(off, -1)
    w, v = np.linalg.eigh(H)
    w, v = w[:Nt], v[:, :Nt].copy()
    for j in range(Nt - 1):          # sign convention: n_{j,j+1} > 0
        if v[:, j] @ (n * v[:, j + 1]) < 0:
            v[:, j + 1] *= -1.0
    nmat = v.T @ (n[:, None] * v)
    return w, nmat


# ------------------------------------------------------------ normal modes --
def omega_matrix(wr: float, wf: float, J: float) -> np.ndarray:
    """Omega of Sec. S2.D on (alpha, beta, gamma, delta)."""
    return np.array([[wr, J, 0.0, J],
                     [J, wf, J, 0.0],
                     [0.0, -J, -wr, -J],
                     [-J, 0.0, -J, -wf]])


def normal_modes(wr: float, wf: float, J: float):
    """Returns (w_l, w_u, U, S, mu_l, mu_u, nu_l, nu_u)."""
    ev, vec = np.linalg.eig(omega_matrix(wr, wf, J))
    ev, vec = ev.real, vec.real
    pos = np.argsort(ev)[2:]                     # w_l, w_u
    cols = {}
    for name, k in zip(("l", "u"), pos):
        x = vec[:, k]
        nrm = x[0] ** 2 + x[1] ** 2 - x[2] ** 2 - x[3] ** 2
        x = x / np.sqrt(nrm)
        if x[1] < 0:
            x = -x
        cols[name] = x
    partner = lambda x: np.array([x[2], x[3], x[0], x[1]])  # noqa: E731
    U = np.column_stack([partner(cols["u"]), partner(cols["l"]), cols["l"], cols["u"]])
    S = np.linalg.inv(U.T)
    mu_u, mu_l = S[0, 3] - S[0, 0], S[0, 2] - S[0, 1]
    nu_u, nu_l = S[1, 3] - S[1, 0], S[1, 2] - S[1, 1]
    return ev[pos[0]], ev[pos[1]], U, S, mu_l, mu_u, nu_l, nu_u


# ------------------------------------------------------------------- model --
def _ladder(d: int):
    return sp.diags(np.sqrt(np.arange(1, d, dtype=float)), 1, shape=(d, d), format="csr", dtype=complex)


def _kron3(x, y, z):
    return sp.kron(sp.kron(x, y, format="csr"), z, format="csr").tocsr()


class PaperModel:
    """Operators of the paper's model on |j_l> (x) |j_u> (x) |j_t>.

    ``frame="rot"``: Eq. S(hamiltonian_rotated) with the dissipators above.
    ``frame="rwa"``: Eq. S(hamiltonian_rwa), the rotated Hamiltonian without its
    explicitly time-dependent terms, with L_1 = sqrt(kappa) A and r = A (the slow
    parts of the rotated-frame f).
    ``frame="lab"``: the same model before the frame map (the nearest-neighbour
    n_t, H = H_t + w_l N_l + w_u N_u + i g n_t sum_x mu_x (c_x^dag - c_x)
    + i Omega(t) sin(w_d t) sum_x nu_x (c_x^dag - c_x), static f), for the frame pin.
    """

    def __init__(self, Nl, Nu, Nt, Ec, Ej, wr, wf, g, J, kappa, gamma, wd,
                 n_cut=20, frame="rot"):
        self.dims = (int(Nl), int(Nu), int(Nt))
        self.N = Nl * Nu * Nt
        self.wd, self.kappa, self.gamma = float(wd), float(kappa), float(gamma)
        self.eps, self.nmat = transmon(Ec, Ej, Nt, n_cut)
        (self.wl, self.wu, self.U, self.S, self.mu_l, self.mu_u,
         self.nu_l, self.nu_u) = normal_modes(wr, wf, J)
        S = self.S
        s21, s22, s23, s24 = S[1, 0], S[1, 1], S[1, 2], S[1, 3]
        I = lambda d: sp.identity(d, dtype=complex, format="csr")  # noqa: E731
        dag = lambda x: x.conj().T.tocsr()  # noqa: E731
        cl = _kron3(_ladder(Nl), I(Nu), I(Nt))
        cu = _kron3(I(Nl), _ladder(Nu), I(Nt))
        npl_t = sp.diags(np.array([self.nmat[j, j + 1] for j in range(Nt - 1)]), 1,
                         shape=(Nt, Nt), format="csr", dtype=complex)
        npl = _kron3(I(Nl), I(Nu), npl_t)            # n_t^+ : |j><j+1|
        nmi = dag(npl)                                # n_t^-
        b = _kron3(I(Nl), I(Nu), _ladder(Nt))
        jt = np.arange(Nt, dtype=float)
        terms = {}

        def add(a, q, X):
            k = channel_index(a, q)
            terms[k] = terms.get(k, sp.csr_matrix((self.N, self.N), dtype=complex)) + X

        modes = (("l", cl, self.mu_l, self.nu_l, self.wl), ("u", cu, self.mu_u, self.nu_u, self.wu))
        if frame in ("rot", "rwa"):
            # "rwa": Eq. S(hamiltonian_rwa), the explicitly time-dependent terms of
            # Eq. S(hamiltonian_rotated) dropped; the jump operator and the readout
            # keep their slow part A (reading: a slow generator, as the RWA intends)
            rot = frame == "rot"
            add(0, 0, _kron3(I(Nl), I(Nu), sp.diags(self.eps - self.eps[0] - jt * wd).astype(complex)))
            for _, c, mu, nu, w in modes:
                add(0, 0, (w - wd) * (dag(c) @ c))
                add(0, 0, 1j * g * mu * (npl @ dag(c) - nmi @ c))
                add(1, 0, -0.5 * nu * (dag(c) + c))
                if rot:
                    add(0, -2, -1j * g * mu * (npl @ c))
                    add(0, 2, 1j * g * mu * (nmi @ dag(c)))
                    add(1, 2, 0.5 * nu * dag(c))
                    add(1, -2, 0.5 * nu * c)
            A = s23 * cl + s24 * cu
            B = s21 * dag(cu) + s22 * dag(cl)
            if rot:
                self.jump_terms = [{channel_index(0, 0): np.sqrt(kappa) * A,
                                    channel_index(0, 2): np.sqrt(kappa) * B},
                                   {channel_index(0, 0): np.sqrt(gamma) * b}]
                self.r_terms = {channel_index(0, 0): A.tocsr(), channel_index(0, 2): B.tocsr()}
            else:
                self.jump_terms = [{channel_index(0, 0): np.sqrt(kappa) * A},
                                   {channel_index(0, 0): np.sqrt(gamma) * b}]
                self.r_terms = {channel_index(0, 0): A.tocsr()}
        elif frame == "lab":
            add(0, 0, _kron3(I(Nl), I(Nu), sp.diags(self.eps - self.eps[0]).astype(complex)))
            nt = npl + nmi
            for _, c, mu, nu, w in modes:
                add(0, 0, w * (dag(c) @ c))
                add(0, 0, 1j * g * mu * (nt @ (dag(c) - c)))
                # i Omega sin(w_d t) nu (c^dag - c) = (Omega nu / 2)(e^{i w_d t} - e^{-i w_d t})(c^dag - c)
                add(1, 1, 0.5 * nu * (dag(c) - c))
                add(1, -1, -0.5 * nu * (dag(c) - c))
            f = s21 * dag(cu) + s22 * dag(cl) + s23 * cl + s24 * cu
            self.jump_terms = [{channel_index(0, 0): np.sqrt(kappa) * f},
                               {channel_index(0, 0): np.sqrt(gamma) * b}]
            self.r_terms = {channel_index(0, 0): f.tocsr()}
        else:
            raise ValueError("frame must be 'rot', 'rwa' or 'lab'")
        self.frame = frame
        self.h_terms = {k: v.tocsr() for k, v in terms.items()}
        self.level = np.tile(np.arange(Nt), Nl * Nu)
        self.n_exc = np.array([jl + ju + j for jl in range(Nl) for ju in range(Nu) for j in range(Nt)], dtype=float)

    def _at(self, terms, t, omega):
        chi = channel_values(t, omega, self.wd)
        out = None
        for k, X in terms.items():
            out = chi[k] * X if out is None else out + chi[k] * X
        return out

    def hamiltonian(self, t: float, omega: float):
        return self._at(self.h_terms, t, omega)

    def jumps(self, t: float, omega: float):
        return [self._at(jt, t, omega) for jt in self.jump_terms]

    def readout(self, t: float, omega: float):
        """The readout operator f (lab frame) or f(t) (rotated frame)."""
        return self._at(self.r_terms, t, omega)

    def heff_terms(self):
        """Channel terms of -i H_eff = -i H - 1/2 sum_k L_k^dag L_k: the channel of
        L_{k,q1}^dag L_{k,q2} is q2 - q1 (the jump operators carry no Omega)."""
        out = {k: -1j * X for k, X in self.h_terms.items()}
        for jt in self.jump_terms:
            for k1, X1 in jt.items():
                for k2, X2 in jt.items():
                    q = (k2 - 2) - (k1 - 2)
                    k = channel_index(0, q)
                    term = -0.5 * (X1.conj().T @ X2)
                    out[k] = out[k] + term if k in out else term
        return {k: v.tocsr() for k, v in out.items()}


# ------------------------------------------------------------- integrators --
def nosse_rhs(m, t, model, envelope):
    """Eq. S5 with time-dependent H(t) and L_k(t)."""
    om = envelope(t)
    H = model.hamiltonian(t, om)
    gram = m.conj().T @ m
    chol = sla.cho_factor(gram, lower=False)
    out = -1j * (H @ m)
    for L in model.jumps(t, om):
        Lm = L @ m
        X = sla.cho_solve(chol, m.conj().T @ Lm)          # m^+ L_k m
        out += 0.5 * (Lm @ X.conj().T - L.conj().T @ Lm)
    return out


def lindblad_rhs(rho, t, model, envelope):
    """Eq. S4 with time-dependent H(t) and L_k(t)."""
    om = envelope(t)
    H = model.hamiltonian(t, om)
    Hr = H @ rho
    out = -1j * (Hr - Hr.conj().T)
    for L in model.jumps(t, om):
        Lr = L @ rho
        out += (L @ Lr.conj().T).conj().T
        LdLr = L.conj().T @ Lr
        out -= 0.5 * (LdLr + LdLr.conj().T)
    return out


def _obs(y, model, low_rank, t, omega):
    """beta = tr(rho r(t)), level populations, photons tr(rho r^dag r), trace."""
    r = model.readout(t, omega)
    if low_rank:
        rm = r @ y
        w = np.sum(np.abs(y) ** 2, axis=1)
        return np.trace(y.conj().T @ rm), np.bincount(model.level, w, model.dims[2]), np.vdot(rm, rm).real, w.sum()
    d = np.real(np.diag(y))
    return (np.trace(r @ y), np.bincount(model.level, d, model.dims[2]),
            np.trace(r.conj().T @ (r @ y)).real, d.sum())


def integrate(y0, model, envelope, dt, n_steps, pop_every=1, low_rank=True, return_state=False):
    """RK4 (the same classical scheme as the other oracles). y0 is m (N x M) or rho."""
    rhs = nosse_rhs if low_rank else lindblad_rhs
    y = np.array(y0, dtype=complex)
    beta = np.zeros(n_steps + 1, dtype=complex)
    pops, nrs, traces = [], [], []
    for n in range(n_steps + 1):
        if n > 0:
            y = rk4_step(lambda x, t: rhs(x, t, model, envelope), y, (n - 1) * dt, dt)
        t = n * dt
        b, p, nr, tr = _obs(y, model, low_rank, t, envelope(t))
        beta[n] = b
        if n % pop_every == 0:
            pops.append(p)
            nrs.append(nr)
            traces.append(tr)
    out = {"beta": beta, "pops": np.array(pops), "nr": np.array(nrs), "trace": np.array(traces)}
    if return_state:
        out["state"] = y
    return out
