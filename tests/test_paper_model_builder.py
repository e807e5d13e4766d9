"""The library's host builder of the paper's model (lr_paper_model_build)
against the oracle's operators, channel by channel. Host code only: no GPU
work is issued."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import paper_model as pm
from paper_2508_18114_gb300 import lr

TP = 2.0 * np.pi


@pytest.fixture(scope="module")
def sparse_mod():
    if not os.path.exists(lr.LIB_PATH):
        from paper_2508_18114_gb300 import build
        build.build()
    from paper_2508_18114_gb300 import sparse
    return sparse


def _ops(m):
    """{operator: {channel: csr}} from the builder's arrays."""
    N = m["N"]
    val = m["val"][0::2] + 1j * m["val"][1::2]
    out = []
    for o in range(m["n_jumps"] + 2):
        rp = m["rowptr"][o * (N + 1):(o + 1) * (N + 1)]
        rows = np.repeat(np.arange(N), np.diff(rp))
        sl = slice(rp[0], rp[-1])
        by = {}
        for ch in np.unique(m["chan"][sl]):
            k = m["chan"][sl] == ch
            by[int(ch)] = sp.csr_matrix((val[sl][k], (rows[k], m["col"][sl][k])), shape=(N, N))
        out.append(by)
    return out


def _close(got, want, scale):
    keys = set(got) | set(want)
    for k in keys:
        g = got.get(k, None)
        w = want.get(k, None)
        g = g.toarray() if g is not None else 0.0
        w = w.toarray() if w is not None else 0.0
        assert np.abs(g - w).max() <= 1e-11 * scale, k


@pytest.mark.parametrize("frame", ["rot", "rwa"])
@pytest.mark.parametrize("dims,over", [
    ((6, 3, 4), {}),
    ((5, 4, 6), dict(g=TP * 0.4, J=TP * 0.2, kappa=2.0, gamma=0.3)),
    ((3, 2, 3), dict(wr=TP * 5.0, wf=TP * 6.5)),
])
def test_builder_matches_oracle(sparse_mod, dims, over, frame):
    P = dict(Ec=TP * 0.315, Ej=51 * TP * 0.315, wr=TP * 7.2, wf=TP * 7.21, g=TP * 0.15, J=TP * 0.03,
             kappa=TP * 0.03, gamma=TP * 8e-6, wd=TP * 7.18)
    P.update(over)
    Nl, Nu, Nt = dims
    m = sparse_mod.paper_model(Nl, Nu, Nt, frame=frame, **P)
    ora = pm.PaperModel(Nl, Nu, Nt, frame=frame, **P)
    assert m["N"] == ora.N
    ops = _ops(m)
    scale = max(abs(P["wd"]) * Nt, 1.0)
    _close(ops[0], ora.heff_terms(), scale)
    _close(ops[1], ora.jump_terms[0], 1.0)
    _close(ops[2], ora.jump_terms[1], 1.0)
    _close(ops[3], ora.r_terms, 1.0)
    assert np.array_equal(m["level"], ora.level)
    q = m["params"]
    assert abs(q["w_l"] - ora.wl) < 1e-12 * ora.wl and abs(q["w_u"] - ora.wu) < 1e-12 * ora.wu
    for name in ("mu_l", "mu_u", "nu_l", "nu_u"):
        assert abs(q[name] - getattr(ora, name)) < 1e-12, name
    S = ora.S
    for name, (i, j) in (("s21", (1, 0)), ("s22", (1, 1)), ("s23", (1, 2)), ("s24", (1, 3))):
        assert abs(q[name] - S[i, j]) < 1e-12, name
    assert abs(q["qubit_frequency"] - (ora.eps[1] - ora.eps[0])) < 1e-9


def test_builder_rejects_bad_cutoffs(sparse_mod):
    P = dict(Ec=TP * 0.315, Ej=51 * TP * 0.315, wr=TP * 7.2, wf=TP * 7.21, g=TP * 0.15, J=TP * 0.03,
             kappa=0.2, gamma=1e-4, wd=TP * 7.18)
    for dims, n_cut in (((0, 2, 3), 20), ((4, 2, 17), 20), ((4, 2, 6), 3), ((4, 2, 6), 65)):
        with pytest.raises(lr.LrError):
            sparse_mod.paper_model(*dims, n_cut=n_cut, **P)


def _model_args():
    return dict(Ec=TP * 0.315, Ej=51 * TP * 0.315, wr=TP * 7.2, wf=TP * 7.21, g=TP * 0.15, J=TP * 0.03,
                kappa=TP * 0.03, gamma=TP * 8e-6, wd=TP * 7.18)


def test_sparse_create_validates_arguments(sparse_mod):
    """lr_sparse_create checks its arguments on the host (no device work)."""
    import ctypes as C
    lib = lr.load_library()
    m = sparse_mod.paper_model(4, 2, 3, **_model_args())
    wd = m["wd"]
    arrs = [np.ascontiguousarray(m[k]) for k in ("rowptr", "col", "val", "chan", "level")]

    def create(model_over=None, M=2, pulse=(0, [1.0, wd, 0.5, 0.0]), n=2, prec=0):
        a = [x.copy() for x in arrs]
        if model_over:
            model_over(a)
        sm = sparse_mod.lr_sparse_model(m["N"], 2, 3, m["nnz"], wd, *[C.c_void_p(x.ctypes.data) for x in a])
        pl = (lr.lr_pulse * n)(*[lr.make_pulse(*pulse)] * n)
        h = C.c_void_p()
        st = lib.lr_sparse_create(C.byref(sm), n, M, prec, pl, 4.0, 100, 1, C.byref(h))
        if st == 0:
            sz = C.c_size_t()
            assert lib.lr_sparse_workspace_size(h, C.byref(sz)) == 0 and sz.value > 0
            lib.lr_sparse_destroy(h)
        return st

    assert create() == 0 and create(prec=1) == 0
    assert create(prec=2) == 9 and create(prec=3) == 9             # LR_ERR_UNSUPPORTED
    assert create(M=0) == 1 and create(M=33) == 1 and create(n=0) == 1
    assert create(pulse=(0, [1.0, wd, 0.5, 0.3])) == 1            # pulse phase must be 0
    assert create(pulse=(0, [1.0, wd * 1.001, 0.5, 0.0])) == 1    # drive frequency = frame frequency
    N = m["N"]

    def bad_col(a):
        a[1][0] = N

    def bad_chan(a):
        a[3][0] = 10                                               # channels are 0 .. 9

    def bad_level(a):
        a[4][0] = 7

    assert create(bad_col) == 1 and create(bad_chan) == 1 and create(bad_level) == 1
