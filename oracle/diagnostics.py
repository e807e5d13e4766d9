"""Validity diagnostics of the low-rank ansatz (oracle; test infrastructure).

Sec. S1.B of the paper judges a rank-M run by the spectrum of
rho = m m^dag, in particular the ratio p_M / p_1 of its smallest to its
largest nonzero eigenvalue (Fig. S1), next to the purity tr(rho^2).

Definitions, written out:
  rho_spectrum(m) - the M largest eigenvalues of rho = m m^dag (N x N);
  rho_purity(m)   - tr(rho rho).
Forming rho costs O(N^2 M); the Gram forms use G = m^dag m (M x M), which has
the same nonzero eigenvalues as m m^dag, and tr((m m^dag)^2) = tr((m^dag m)^2):
  gram_spectrum(G) - eigenvalues of G, descending;
  gram_purity(G)   - tr(G G).
Parity: pinned by the rho forms at small N (the two forms computed
independently), and by the closed forms of the fixed-rank initial state
(eigenvalues 1 - (M-1) eps and eps, M-1 times).
"""
from __future__ import annotations

import numpy as np


def rho_spectrum(m: np.ndarray) -> np.ndarray:
    rho = m @ m.conj().T
    ev = np.linalg.eigvalsh(rho)[::-1]
    return ev[: m.shape[1]]


def rho_purity(m: np.ndarray) -> float:
    rho = m @ m.conj().T
    return float(np.trace(rho @ rho).real)


def gram_spectrum(G: np.ndarray) -> np.ndarray:
    return np.linalg.eigvalsh(G)[::-1]


def gram_purity(G: np.ndarray) -> float:
    return float(np.trace(G @ G).real)
