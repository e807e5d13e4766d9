"""Pins of the oracle's rank growth (adaptive rank, Sec. S1.B)."""
import numpy as np

from oracle import adaptive, init_state


def test_grow_pads_with_orthonormal_columns():
    rng = np.random.default_rng(1)
    N, Ms, Md, eps = 30, 3, 7, 1e-4
    m = rng.standard_normal((N, Ms)) + 1j * rng.standard_normal((N, Ms))
    g = adaptive.grow(m, Md, eps, seed=9, traj=2)
    assert g.shape == (N, Md)
    assert np.array_equal(g[:, :Ms], m)                         # kept columns unchanged
    q = g[:, Ms:] / np.sqrt(eps)
    assert np.abs(q.conj().T @ q - np.eye(Md - Ms)).max() < 1e-12   # orthonormal
    assert np.abs(m.conj().T @ q).max() < 1e-12                   # orthogonal to span(m)
    rho0, rho1 = m @ m.conj().T, g @ g.conj().T
    assert abs(np.trace(rho1 - rho0).real - eps * (Md - Ms)) < 1e-14
    # the new subspace depends on span(m) only: a gauge change m -> m U gives the same rho
    u, _ = np.linalg.qr(rng.standard_normal((Ms, Ms)) + 1j * rng.standard_normal((Ms, Ms)))
    g2 = adaptive.grow(m @ u, Md, eps, seed=9, traj=2)
    assert np.abs(g2 @ g2.conj().T - rho1).max() < 1e-12


def test_grow_uses_the_initial_state_generator():
    """Growing a rank-1 state psi with weight eps reproduces the fixed-rank
    initial condition's padding (same draws, pair index (j-1) N + n)."""
    N, M, eps, seed, traj = 12, 4, 1e-3, 77, 5
    m0 = init_state.initial_state(N, M, 2, eps, seed, traj)
    psi = np.zeros((N, 1), complex)
    psi[2, 0] = np.sqrt(1.0 - (M - 1) * eps)
    g = adaptive.grow(psi, M, eps, seed, traj)
    assert np.abs(g @ g.conj().T - m0 @ m0.conj().T).max() < 1e-14


def test_ratio_is_the_spectrum_extreme():
    p = np.array([0.7, 0.2, 1e-3])
    v, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((5, 3)))
    m = v * np.sqrt(p)
    assert abs(adaptive.ratio(m) - 1e-3 / 0.7) < 1e-12
