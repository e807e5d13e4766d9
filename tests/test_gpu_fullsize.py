"""Full-size batches in the launch configuration the benchmark uses, checked
on sampled trajectories against the oracle.

The whole batch runs on the GPU (all 512 trajectories of the N=2000, M=20
workload; the 512 uneven trajectories; the 128 trajectories at N=8000, M=32).
The oracle integrates only a few sampled candidates, each from the same seeded
initial state (trajectory index 2c + level), which it can afford. Tolerances
as elsewhere: 5e-5 for FP32_G64, 1e-10 for FP64.
"""
import numpy as np
import pytest

import lr_inputs as li
from oracle import parallel
from paper_2508_18114_gb300 import runner

from _compare import compare_observables

pytestmark = pytest.mark.gpu
TOL32, TOL64 = 5e-5, 1e-10


def _select(gpu, cands):
    idx = [2 * c + lv for c in cands for lv in (0, 1)]
    return {"beta": gpu["beta"][idx], "pops": gpu["pops"][idx], "nphot": gpu["nphot"][idx],
            "trace": gpu["trace"][idx], "eps_a": gpu["eps_a"][list(cands)]}


def _run(wl, cands, precision, n_steps, pe):
    job = parallel.OracleJob(wl, n_steps, pe, candidates=cands, traj_base=[2 * c for c in cands])
    b = runner.make_batch(wl, precision=precision, engine="fused", pop_every=pe, max_steps=n_steps)
    info = b.query()
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, n_steps)
    gpu = b.observables()
    b.close()
    ora = job.result()
    nts = [wl.candidates[c].model.dims[0] for c in cands for _ in (0, 1)]
    return info, _select(gpu, cands), ora, nts


def test_c4_whole_batch_sampled():
    wl = li.c4()
    cands = [0, 97, 255]
    info, gpu, ora, nts = _run(wl, cands, "fp32_g64", 120, 40)
    # the plan the benchmark times: teams of 2 CTAs, stage state in L2, CUDA-core projection
    assert info.engine == 2 and info.team_size == 2 and info.stage_in_smem == 0 and info.tensor_passes == 0
    print(compare_observables(gpu, ora, 2 * len(cands), nts, TOL32, TOL32, "c4 sampled"))


def _extremes(wl):
    Ms = [c.M for c in wl.candidates]
    Ns = [c.model.N for c in wl.candidates]
    pick = {int(np.argmin(Ms)), int(np.argmax(Ms)), int(np.argmin(Ns)), int(np.argmax(Ns))}
    return sorted(pick)


@pytest.mark.parametrize("precision,tol,n_steps", [("fp32_g64", TOL32, 80), ("fp64", TOL64, 40)])
def test_c3_uneven_batch_sampled(precision, tol, n_steps):
    wl = li.c3()
    cands = _extremes(wl)
    info, gpu, ora, nts = _run(wl, cands, precision, n_steps, 40)
    assert info.engine == 2
    print(compare_observables(gpu, ora, 2 * len(cands), nts, tol, tol, "c3 %s sampled %s" % (precision, cands)))


def test_c5_large_batch_sampled():
    wl = li.c5()
    cands = [0, 63]
    info, gpu, ora, nts = _run(wl, cands, "fp32_g64", 20, 10)
    assert info.engine == 2
    print(compare_observables(gpu, ora, 2 * len(cands), nts, TOL32, TOL32, "c5 sampled"))
