"""GPU adaptive rank control (lr_grow_rank + lr_diagnostics) against the
oracle's controller: the same growth decisions, beta at every step and the
populations at the segment ends, FP64."""
import types

import numpy as np
import pytest

from oracle import adaptive as oad
from oracle import init_state
from oracle import pulse as opulse
from oracle.model import Model

pytestmark = pytest.mark.gpu

TP = 2.0 * np.pi


def _setup():
    p = types.SimpleNamespace(dims=(3, 8), wq=TP * 6.0, alpha=-TP * 0.3, wr=TP * 7.0, g=TP * 0.15, kappa=3.0,
                              gamma=0.5)
    pulses = [(0, (TP * 0.8, TP * 7.0, 0.05, 0.0)), (0, (TP * 0.3, TP * 7.0, 0.05, 0.0))]
    return p, pulses


@pytest.mark.parametrize("engine", ["plain", "fused"])
def test_adaptive_rank_matches_oracle(engine):
    from paper_2508_18114_gb300.adaptive import adaptive_run
    p, pulses = _setup()
    # tol = 8e-6: growth at steps 100 (both candidates), 300 (candidate 0 only:
    # uneven ranks in one batch) and 400; every ratio is >= 6% away from tol
    tau, dt, n, seg, seed, eps, tol = 0.6, 1e-3, 600, 100, 5, 1e-5, 8e-6
    b, hist = adaptive_run([p, p], pulses, tau, dt, n, rank0=2, max_rank=6, d_rank=2, tol=tol, segment=seg,
                           seed=seed, eps=eps, precision="fp64", engine=engine)
    got = b.observables()
    m = Model(p.dims, p.wq, p.alpha, p.wr, p.g, p.kappa, p.gamma)
    coefs = [opulse.coefficient(k, q, tau) for k, q in pulses]
    m0s = [init_state.initial_state(m.N, 2, m.basis_index((tj % 2, 0)), eps, seed, tj) for tj in range(4)]
    betas, pops, ohist = oad.adaptive_run([m, m], coefs, dt, n, 2, 6, 2, tol, seg, m0s, eps)
    assert [h["ranks"] for h in hist] == [h["ranks"] for h in ohist]
    assert [h["ranks"] for h in hist] == [[4, 4], [4, 4], [6, 4], [6, 6], [6, 6], [6, 6]]
    for h, o in zip(hist, ohist):
        assert np.allclose(h["ratio"], o["ratio"], rtol=1e-6, atol=0)
    assert b.ranks == [6, 6]
    for tj in range(4):
        bo = betas[tj]
        assert np.abs(got["beta"][tj][: n + 1] - bo).max() <= 1e-10 * np.abs(bo).max(), tj
        po = pops[tj]
        gp = got["pops"][tj][: po.shape[0], : po.shape[1]]
        assert np.abs(gp - po).max() <= 1e-10, tj
