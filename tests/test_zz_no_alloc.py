"""lr_integrate_plain_noalloc: the plain FP64 engine for one trajectory with
its scratch in a static device array, for callers that cannot allocate
device memory (they cannot bind a workspace). Checked against lr_integrate
(plain FP64 engine, caller-bound workspace) on the same state, for two calls
in a row, within the FP64 parity tolerance (1e-10 relative). This file is
collected last on purpose."""
import numpy as np
import pytest

import lr_inputs as li
from paper_2508_18114_gb300 import lr, runner

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_noalloc_matches_workspace_engine_two_calls():
    import torch
    wl = li.c2(n_steps=120)
    cand = wl.candidates[0]
    N, M = cand.model.N, cand.M
    ref = runner.make_batch(wl, precision="fp64", engine="plain", max_steps=120, pop_every=60)
    ref.set_initial(wl.init_seed, wl.eps)
    z0 = ref.get_state(1)                              # |e> trajectory
    Z = torch.from_numpy(z0.copy()).to("cuda")
    beta = torch.zeros(121, dtype=torch.complex128, device="cuda")
    steps = (50, 70)
    pulse = (cand.pulse.kind, cand.pulse.p)
    ref.integrate(wl.dt, steps[0])
    st = lr.integrate_plain_noalloc(cand.model, M, pulse, wl.tau, Z, beta[: steps[0] + 1], wl.dt, 0, steps[0])
    assert st == 0, lr.STATUS[st]
    torch.cuda.synchronize()
    assert _rel(Z.cpu().numpy(), ref.get_state(1)) <= TOL
    obs = ref.observables()
    assert _rel(beta[: steps[0] + 1].cpu().numpy(), obs["beta"][1][: steps[0] + 1]) <= TOL
    # second call continues from the first one's output (scratch reused)
    ref.integrate(wl.dt, steps[1])
    st = lr.integrate_plain_noalloc(cand.model, M, pulse, wl.tau, Z, beta[steps[0]:], wl.dt, steps[0], steps[1])
    assert st == 0, lr.STATUS[st]
    torch.cuda.synchronize()
    assert _rel(Z.cpu().numpy(), ref.get_state(1)) <= TOL
    obs = ref.observables()
    assert _rel(beta.cpu().numpy(), obs["beta"][1]) <= TOL
    ref.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    m = li.c5(n_candidates=1).candidates[0]          # N = 8000 > 4096
    Z = torch.zeros(1, dtype=torch.complex128, device="cuda")
    st = lr.integrate_plain_noalloc(m.model, m.M, (m.pulse.kind, m.pulse.p), 40.0, Z, Z, 5e-4, 0, 1)
    assert st == 9   # LR_ERR_UNSUPPORTED, nothing launched
