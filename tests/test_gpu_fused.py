"""FUSED engine (persistent cluster kernel) against the FP64 oracle.

FP64 (complex128): 1e-10 relative / absolute, as for every FP64 path.
FP32_G64 (complex64 bulk, FP64-class Gram, FP64 Cholesky/inverse/signal):
the state is rounded to FP32 once per RK4 stage, a random walk of relative
size u32 * sqrt(4 n_steps) = 6e-8 * 400 = 2.4e-5 after the 40k steps of a
full pulse; the bound is twice that: 5e-5 relative for beta, photons and
eps_a, 5e-5 absolute for populations and tr(rho) (which are O(1)).
"""
import os

import numpy as np
import pytest

import lr_inputs as li
from oracle import parallel
from paper_2508_18114_gb300 import LrError, runner

from _compare import compare_observables

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
TOL32, TOL32_POP = 5e-5, 5e-5


def _nts(wl):
    return [c.model.dims[0] for c in wl.candidates for _ in (0, 1)]


def _filter(nt, nr, nf):
    return li.ModelParams(dims=(nt, nr, nf), wq=li.TWO_PI * 6.0, alpha=-li.TWO_PI * 0.3,
                          wr=li.TWO_PI * 7.5, g=li.TWO_PI * 0.15, kappa=li.TWO_PI * 0.05,
                          gamma=1.0 / 50000.0, wf=li.TWO_PI * 7.51, J=li.TWO_PI * 0.1)


def _three_mode_batch(n_steps=400):
    """Uneven N and M, ragged resonator splits, maximum rank 32."""
    cands = [
        li.Candidate(_filter(3, 7, 5), 7, li.pulse_two_segment(31, li.TWO_PI * 7.5)),
        li.Candidate(_filter(5, 6, 3), 12, li.pulse_two_segment(32, li.TWO_PI * 7.5)),
        li.Candidate(_filter(4, 9, 6), 32, li.pulse_two_segment(33, li.TWO_PI * 7.5)),
        li.Candidate(_filter(2, 5, 4), 5, li.pulse_two_segment(34, li.TWO_PI * 7.5)),
    ]
    return li.Workload("ragged3", cands, 5e-4, n_steps, 2.0, init_seed=91, eps=1e-5)


def _tc_batch(n_steps=400):
    """Uneven N and M up to 20 (operand tiles fit in shared memory), with
    576 rows for the largest trajectory: several 128-row tensor-core tiles and
    a ragged last tile at team sizes 1, 2 and 4."""
    cands = [
        li.Candidate(_filter(3, 7, 5), 7, li.pulse_two_segment(41, li.TWO_PI * 7.5)),
        li.Candidate(_filter(5, 6, 3), 12, li.pulse_two_segment(42, li.TWO_PI * 7.5)),
        li.Candidate(_filter(6, 12, 8), 20, li.pulse_two_segment(43, li.TWO_PI * 7.5)),
        li.Candidate(_filter(2, 5, 4), 5, li.pulse_two_segment(44, li.TWO_PI * 7.5)),
    ]
    return li.Workload("ragged_tc", cands, 5e-4, n_steps, 2.0, init_seed=92, eps=1e-5)


class _env:
    def __init__(self, **kw):
        self.kw = kw

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kw}
        for k, v in self.kw.items():
            os.environ[k] = str(v)

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def test_c1_full_pulse_fp64_and_fp32():
    wl = li.c1()
    job = parallel.OracleJob(wl, None, 100)
    g64 = runner.run(wl, precision="fp64", engine="fused", pop_every=100)
    g32 = runner.run(wl, precision="fp32_g64", engine="fused", pop_every=100)
    ora = job.result()
    w64 = compare_observables(g64, ora, 2, _nts(wl), TOL64, TOL64, "c1 fused fp64")
    w32 = compare_observables(g32, ora, 2, _nts(wl), TOL32, TOL32_POP, "c1 fused fp32_g64")
    print("c1 full pulse fused fp64:", w64)
    print("c1 full pulse fused fp32_g64:", w32)
    assert g64["engine"] == "fused"


def test_c2_full_size_fp64_and_fp32():
    wl = li.c2(n_steps=300)
    job = parallel.OracleJob(wl, None, 50)
    g64 = runner.run(wl, precision="fp64", engine="fused", pop_every=50)
    g32 = runner.run(wl, precision="fp32_g64", engine="fused", pop_every=50)
    ora = job.result()
    print("c2 fused fp64:", compare_observables(g64, ora, 2, _nts(wl), TOL64, TOL64, "c2 fused fp64"))
    print("c2 fused fp32:", compare_observables(g32, ora, 2, _nts(wl), TOL32, TOL32_POP, "c2 fused fp32"))


@pytest.mark.parametrize("C,zs", [(1, "smem"), (2, "smem"), (3, "smem"), (5, "smem"), (2, "global")])
def test_cluster_shapes_fp64(C, zs):
    wl = _three_mode_batch()
    ora = parallel.run_workload(wl, None, 40)
    with _env(LR_FUSED_C=C, LR_FUSED_ZS=zs):
        b = runner.make_batch(wl, precision="fp64", engine="fused", pop_every=40)
    assert b.query().team_size == C
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    gpu = b.observables()
    b.close()
    compare_observables(gpu, ora, 2 * len(wl.candidates), _nts(wl), TOL64, TOL64, "C=%d %s" % (C, zs))


@pytest.mark.parametrize("C", [1, 4])
def test_cluster_shapes_fp32(C):
    wl = _three_mode_batch()
    ora = parallel.run_workload(wl, None, 40)
    with _env(LR_FUSED_C=C):
        b = runner.make_batch(wl, precision="fp32_g64", engine="fused", pop_every=40)
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    gpu = b.observables()
    b.close()
    compare_observables(gpu, ora, 2 * len(wl.candidates), _nts(wl), TOL32, TOL32_POP, "fp32 C=%d" % C)


@pytest.mark.parametrize("C,tc", [(1, 3), (2, 3), (4, 3), (2, 0)])
def test_projection_on_tensor_cores_fp32_g64(C, tc):
    """FP32_G64 with the projection term as three TF32 tensor-core passes
    (two-term split of both operands, FP32-class products) against the oracle
    at the FP32 tolerance; tc = 0 forces the CUDA-core projection. Ragged rows:
    the 128-row tiles end inside a CTA's rows."""
    wl = _tc_batch()
    ora = parallel.run_workload(wl, None, 40)
    with _env(LR_FUSED_C=C, LR_FUSED_TC=tc):
        b = runner.make_batch(wl, precision="fp32_g64", engine="fused", pop_every=40)
    info = b.query()
    assert info.team_size == C and info.tensor_passes == tc
    if tc:
        assert info.stage_in_smem == 0
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    gpu = b.observables()
    b.close()
    print(compare_observables(gpu, ora, 2 * len(wl.candidates), _nts(wl), TOL32, TOL32_POP,
                              "fp32_g64 C=%d tc=%d" % (C, tc)))


# One TF32 pass rounds both operands of the projection term to 11 significant
# bits (unit roundoff u = 2^-11 = 4.9e-4). The error this puts into F is a
# fraction u of the projection term, whose size is set by the decay rates
# (kappa ~ 0.3/ns here), so over a pulse of length tau it grows to about
# u kappa tau relative; at tau = 0.2 ns that is 3e-5. Populations and eps_a are
# held to 50x that, the size of the effect where the Moore-Penrose inverse
# amplifies it (1/sqrt(eps) ~ 300 for the padding columns).
TOL_TF32 = 50 * 2.0 ** -11 * (li.TWO_PI * 0.05) * 0.2


def test_tf32_variant_error():
    wl = _tc_batch()
    ora = parallel.run_workload(wl, None, 40)
    b = runner.make_batch(wl, precision="tf32_g64", engine="fused", pop_every=40)
    info = b.query()
    assert info.tensor_passes == 1 and info.stage_in_smem == 0
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, wl.n_steps)
    gpu = b.observables()
    b.close()
    print("tf32 variant:", compare_observables(gpu, ora, 2 * len(wl.candidates), _nts(wl), TOL_TF32, TOL_TF32,
                                               "tf32_g64"))


def test_fused_resume_is_bitwise():
    wl = _three_mode_batch(200)
    outs = []
    for split in ((200,), (120, 80), (1, 199)):
        b = runner.make_batch(wl, precision="fp32_g64", engine="fused", pop_every=20)
        b.set_initial(wl.init_seed, wl.eps)
        for n in split:
            b.integrate(wl.dt, n)
        outs.append((b.observables(), [b.get_state(j) for j in range(b.n_traj)]))
        b.close()
    for o, zs in outs[1:]:
        for k in ("beta", "pops", "nphot", "trace", "eps_a"):
            assert np.array_equal(o[k], outs[0][0][k]), k
        for z, z0 in zip(zs, outs[0][1]):
            assert np.array_equal(z, z0)


def test_fused_not_positive_definite_is_reported():
    wl = _three_mode_batch(20)
    b = runner.make_batch(wl, precision="fp64", engine="fused", max_steps=20)
    b.set_initial(wl.init_seed, wl.eps)
    z = b.get_state(3)
    z[:, 2] = z[:, 4]
    b.set_state(3, z)
    b.integrate(wl.dt, 5)
    with pytest.raises(LrError) as ei:
        b.observables()
    assert ei.value.status == 5
    b.close()


def test_auto_engine_choice():
    """AUTO runs the fused kernel, except in FP64 when its plan would spread one
    trajectory over teams of more than two CTAs (the single pulse at N = 2000),
    where the plain kernels are faster."""
    assert runner.make_batch(li.c2(n_steps=10), precision="fp64", max_steps=10).engine == "plain"
    assert runner.make_batch(li.c2(n_steps=10), precision="fp32_g64", max_steps=10).engine == "fused"
    assert runner.make_batch(li.c1(n_steps=10), precision="fp64", max_steps=10).engine == "fused"
