"""The device-wait timeout path of the fused engine.

Every spin-wait in the fused kernel carries an SM-cycle budget, after which it
gives up, sets the device error word to the timeout code and lets the launch
finish, so that the host reads LR_ERR_TIMEOUT and the context stays usable.
The test hook LR_DEBUG_WAIT_CYCLES makes one thread per CTA wait, with that
budget, on an mbarrier that nothing arrives on: the wait has to run out (no
asynchronous copy or MMA is in flight, nothing else waits on it)."""
import numpy as np
import pytest

import lr_inputs as li
from paper_2508_18114_gb300 import lr, runner

pytestmark = pytest.mark.gpu


def _run(wl, steps):
    b = runner.make_batch(wl, precision="fp64", engine="fused", pop_every=10, max_steps=2 * steps)
    b.set_initial(wl.init_seed, wl.eps)
    return b


def test_wait_budget_runs_out_and_is_reported(monkeypatch):
    wl = li.c1(n_steps=40)
    ref = _run(wl, 20)
    ref.integrate(wl.dt, 20)
    want = ref.observables()
    z_want = ref.get_state(1)
    ref.close()

    monkeypatch.setenv("LR_DEBUG_WAIT_CYCLES", "20000")
    b = _run(wl, 20)
    b.integrate(wl.dt, 20)
    with pytest.raises(lr.LrError) as ei:
        b.sync()
    assert ei.value.status == 7, str(ei.value)          # LR_ERR_TIMEOUT
    with pytest.raises(lr.LrError):
        b.observables()
    # the launch ran to its end: the state is the one of a run without the hook
    assert np.array_equal(b.get_state(1), z_want)
    monkeypatch.delenv("LR_DEBUG_WAIT_CYCLES")
    # the context stays usable: a new run from the initial state reports OK
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, 20)
    b.sync()
    got = b.observables()
    b.close()
    # entries up to the current step (20 steps, records every 10) are the meaningful ones
    assert np.array_equal(got["beta"][:, :21], want["beta"][:, :21])
    assert np.array_equal(got["pops"][:, :3], want["pops"][:, :3])
