"""lr_integrate captured in a CUDA graph (fused engine).

The step counter lives in device memory, so each replay of a captured
integrate continues the pulse run: three replays of a 20-step capture must
give exactly (bitwise) what three direct 20-step calls give. A replay that
would pass max_steps must run nothing and report LR_ERR_STATE; the plain
engine refuses capture.
"""
import numpy as np
import pytest

import lr_inputs as li
from paper_2508_18114_gb300 import LrError, runner

pytestmark = pytest.mark.gpu


def test_graph_replays_continue_the_pulse_run():
    wl = li.c4(n_candidates=8, n_steps=60)
    n = 20
    a = runner.make_batch(wl, engine="fused", pop_every=10, max_steps=60)
    a.set_initial(wl.init_seed, wl.eps)
    for _ in range(3):
        a.integrate(wl.dt, n)
    oa = a.observables()
    za = [a.get_state(j) for j in (0, 7, 15)]
    a.close()

    b = runner.make_batch(wl, engine="fused", pop_every=10, max_steps=60)
    b.set_initial(wl.init_seed, wl.eps)
    g = b.capture_integrate(wl.dt, n)
    assert b.query().step == 0          # capture ran nothing
    for _ in range(3):
        g.replay()
    b.sync()
    assert b.query().step == 60
    ob = b.observables()
    for k in ("beta", "pops", "nphot", "trace", "eps_a"):
        assert np.array_equal(oa[k], ob[k]), k
    for j, z in zip((0, 7, 15), za):
        assert np.array_equal(b.get_state(j), z)
    # a fourth replay would pass max_steps: it runs nothing and reports the error
    g.replay()
    with pytest.raises(LrError) as ei:
        b.sync()
    assert ei.value.status == 8   # LR_ERR_STATE
    assert b.query().step == 60
    assert np.array_equal(b.get_state(0), za[0])
    b.close()


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")   # the refused capture records nothing
def test_plain_engine_refuses_capture():
    wl = li.c1(n_steps=10)
    b = runner.make_batch(wl, precision="fp64", engine="plain", pop_every=5, max_steps=10)
    b.set_initial(wl.init_seed, wl.eps)
    with pytest.raises(LrError) as ei:
        b.capture_integrate(wl.dt, 5)
    assert ei.value.status == 9   # LR_ERR_UNSUPPORTED
    b.close()
