"""Fixed-rank initial condition (oracle; test infrastructure only).

Sec. S1.A of the paper: a pure initial state has rank 1, so the Gram matrix
m^dag m would be singular. The remaining M-1 columns are random orthonormal
states with small weight p_j = eps:

    m(0) = ( sqrt(1 - (M-1) eps) psi,  sqrt(eps) q_2, ..., sqrt(eps) q_M ),

with psi = |i_t = g or e, 0, 0> (Eq. S(initial states)) and q_j orthonormal
to psi and to each other, so tr rho(0) = 1.

Random numbers (the method's own draws; implemented independently of the
CUDA library from the published definitions):

* SplitMix64 (Steele, Lea & Flood 2014): for seed s the k-th output
  (k = 0, 1, ...) is mix64(s + (k+1) * 0x9E3779B97F4A7C15) with
  mix64(z): z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
  z *= 0x94D049BB133111EB; z ^= z>>31 (all mod 2^64).
* trajectory seed: output number `traj` of the user seed;
* uniforms in (0, 1]: u = ((x >> 11) + 1) * 2^-53;
* Box-Muller: for pair index p = (j-1) N + n (column j = 1..M-1, row n),
  u1 = U(2p), u2 = U(2p+1) from the trajectory seed and
  xi = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2).

The q_j are the Gram-Schmidt orthonormalisation of (psi, xi_1, ..., xi_{M-1})
in that order; here computed with a Householder QR (numpy), which gives the
same vectors up to a phase per column. rho = m m^dag does not depend on those
phases.

Parity: SplitMix64 pinned by its published first outputs for seed 0;
Box-Muller by Gaussian moments; the state by orthonormality and trace (tests).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    """k-th SplitMix64 output (0-based) for the given seed, vectorised over k."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (k + np.uint64(1)) * GOLDEN)


def trajectory_seed(seed: int, traj: int) -> int:
    return int(splitmix64(seed, np.array([traj]))[0])


def uniforms(seed: int, k: np.ndarray) -> np.ndarray:
    x = splitmix64(seed, k)
    return ((x >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def gaussian_columns(traj_seed: int, N: int, n_cols: int) -> np.ndarray:
    """n_cols complex Gaussian vectors of length N (Box-Muller), shape (N, n_cols)."""
    p = np.arange(N * n_cols, dtype=np.uint64)
    u1 = uniforms(traj_seed, 2 * p)
    u2 = uniforms(traj_seed, 2 * p + np.uint64(1))
    r = np.sqrt(-2.0 * np.log(u1))
    xi = r * (np.cos(2.0 * np.pi * u2) + 1j * np.sin(2.0 * np.pi * u2))
    return xi.reshape(n_cols, N).T


def initial_state(N: int, M: int, psi_index: int, eps: float, seed: int,
                  traj: int) -> np.ndarray:
    """m(0) for one trajectory, shape (N, M), complex128."""
    if not (1 <= M <= N):
        raise ValueError("need 1 <= M <= N")
    psi = np.zeros(N, dtype=complex)
    psi[psi_index] = 1.0
    m = np.zeros((N, M), dtype=complex)
    m[:, 0] = np.sqrt(1.0 - (M - 1) * eps) * psi
    if M > 1:
        xi = gaussian_columns(trajectory_seed(seed, traj), N, M - 1)
        q, _ = np.linalg.qr(np.column_stack([psi, xi]))
        m[:, 1:] = np.sqrt(eps) * q[:, 1:]
    return m
