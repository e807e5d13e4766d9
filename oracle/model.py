"""Readout model operators (oracle; test infrastructure only).

Hamiltonian, Eq. 1 of the paper, in the bare-mode form that the workloads
fix (transmon as a Duffing oscillator, no rotating-wave approximation, the
readout/drive mode last):

    H(t) = wq b^dag b + (alpha/2) b^dag b^dag b b + wr a^dag a
           + g (b + b^dag)(a + a^dag)
           [+ wf f^dag f + J (a + a^dag)(f + f^dag)]
           + c(t) X_d,         X_d = r + r^dag,

where r is the readout mode (a with two modes, the filter f with three; the
paper drives and reads out through the filter, Eq. 1 and Eq. 2), and c(t) is
the pulse coefficient Omega(t) cos(w_d t + phi).

Jump operators, Eq. 2: L_1 = sqrt(kappa) r (decay of the readout mode) and
L_2 = sqrt(gamma) b (transmon T1 decay).

Basis: |i_t> (x) |i_r> [(x) |i_f>], flat index n = (i_t N_r + i_r) N_f + i_f,
which is numpy's kron(transmon, kron(resonator, filter)) ordering.

Rotating frame (``rwa=(w_d, phi)``): the RWA Hamiltonian of Sec. S2, for
this model the frame rotating at w_d for every mode with the counter-rotating
terms dropped:

    H = (wq - w_d) b^dag b + (alpha/2) b^dag b^dag b b + (wr - w_d) a^dag a
        + g (b^dag a + b a^dag) [+ (wf - w_d) f^dag f + J (a^dag f + a f^dag)]
        + (Omega(t)/2) X_d,   X_d = e^{i phi} r + e^{-i phi} r^dag,

with the same jump operators (the frame only adds phases to them).

Parity: pinned by the closed-form tests (coherent-state amplitude of a
driven damped resonator in both frames, exponential level decay,
Schroedinger evolution against a matrix exponential); the rotating-frame
operators by their definitions as the excitation-conserving part of
H - w_d N and the period average of the rotated drive.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def annihilation(d: int) -> sp.csr_matrix:
    """Truncated bosonic annihilation operator: <n-1|a|n> = sqrt(n)."""
    return sp.diags(np.sqrt(np.arange(1, d, dtype=float)), offsets=1,
                    shape=(d, d), format="csr", dtype=complex)


def _embed(ops):
    out = ops[0]
    for o in ops[1:]:
        out = sp.kron(out, o, format="csr")
    return out.tocsr()


class Model:
    """Operators of the readout model on the full Hilbert space.

    Parameters mirror ``lr_inputs.ModelParams``; ``dense=True`` stores numpy
    arrays instead of sparse matrices (faster for tiny N).
    """

    def __init__(self, dims, wq, alpha, wr, g, kappa, gamma, wf=0.0, J=0.0,
                 dense=None, rwa=None):
        dims = tuple(int(d) for d in dims)
        if len(dims) not in (2, 3):
            raise ValueError("dims must be (N_t, N_r) or (N_t, N_r, N_f)")
        self.dims = dims
        self.N = int(np.prod(dims))
        eye = [sp.identity(d, dtype=complex, format="csr") for d in dims]

        def mode_op(k, op):
            ops = list(eye)
            ops[k] = op
            return _embed(ops)

        b = mode_op(0, annihilation(dims[0]))
        a = mode_op(1, annihilation(dims[1]))
        dag = lambda x: x.conj().T.tocsr()  # noqa: E731
        if rwa is None:
            H0 = (wq * (dag(b) @ b) + 0.5 * alpha * (dag(b) @ dag(b) @ b @ b)
                  + wr * (dag(a) @ a) + g * ((b + dag(b)) @ (a + dag(a))))
        else:
            wd, phi = float(rwa[0]), float(rwa[1])
            H0 = ((wq - wd) * (dag(b) @ b) + 0.5 * alpha * (dag(b) @ dag(b) @ b @ b)
                  + (wr - wd) * (dag(a) @ a) + g * (dag(b) @ a + b @ dag(a)))
        if len(dims) == 3:
            f = mode_op(2, annihilation(dims[2]))
            if rwa is None:
                H0 = H0 + wf * (dag(f) @ f) + J * ((a + dag(a)) @ (f + dag(f)))
            else:
                H0 = H0 + (wf - wd) * (dag(f) @ f) + J * (dag(a) @ f + a @ dag(f))
            r = f
        else:
            r = a
        self.b, self.a, self.r = b, a, r
        self.H0 = H0.tocsr()
        if rwa is None:
            self.Xd = (r + dag(r)).tocsr()
        else:
            self.Xd = (np.exp(1j * phi) * r + np.exp(-1j * phi) * dag(r)).tocsr()
        self.rwa = rwa
        self.jumps = [np.sqrt(kappa) * r, np.sqrt(gamma) * b]
        self.jumps_dag = [dag(L) for L in self.jumps]
        self.kappa, self.gamma = float(kappa), float(gamma)
        self.n_r = (dag(r) @ r).tocsr()
        # transmon level of every basis state (for level populations)
        self.level = np.repeat(np.arange(dims[0]), self.N // dims[0])
        if dense is None:
            dense = self.N <= 64
        if dense:
            self.H0 = self.H0.toarray()
            self.Xd = self.Xd.toarray()
            self.jumps = [L.toarray() for L in self.jumps]
            self.jumps_dag = [L.toarray() for L in self.jumps_dag]
            self.r = self.r.toarray()
            self.n_r = self.n_r.toarray()
        self.dense = dense

    @classmethod
    def from_params(cls, p, dense=None, rwa=None) -> "Model":
        return cls(p.dims, p.wq, p.alpha, p.wr, p.g, p.kappa, p.gamma,
                   wf=p.wf, J=p.J, dense=dense, rwa=rwa)

    def hamiltonian(self, c: float):
        """H(t) for a given pulse coefficient c(t)."""
        return self.H0 + c * self.Xd

    def apply_hamiltonian(self, c: float, x):
        """H(t) x = H0 x + c(t) X_d x (same operator as ``hamiltonian``)."""
        return self.H0 @ x + c * (self.Xd @ x)

    def basis_index(self, levels) -> int:
        """Flat index of the product basis state |i_t, i_r[, i_f]>."""
        n = 0
        for i, d in zip(levels, self.dims):
            n = n * d + int(i)
        return n
