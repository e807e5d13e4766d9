"""The C-ABI library loads and exports what include/lr.h declares; host-side
argument validation (no GPU compute is issued here)."""
import ctypes as C
import os
import re

import pytest

from paper_2508_18114_gb300 import lr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lr_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(lr.LIB_PATH):
        from paper_2508_18114_gb300 import build
        build.build()
    return lr.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "lr_integrate" in names and "lr_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lr.EXPORTS)


def _opts(**kw):
    o = dict(precision=0, engine=1, max_steps=100, pop_every=1, eta=0.6)
    o.update(kw)
    return lr.lr_options(o["precision"], o["engine"], o["max_steps"], o["pop_every"], o["eta"])


def _model(dims=(4, 10)):
    class P:
        pass
    p = P()
    p.dims, p.wq, p.alpha, p.wr, p.g, p.kappa, p.gamma = dims, 37.7, -1.88, 47.1, 0.94, 0.06, 2e-5
    p.wf, p.J = 47.2, 0.63
    return lr.make_model(p)


def _create(lib, models, ranks, opt):
    n = len(models)
    h = C.c_void_p()
    st = lib.lr_create(n, (lr.lr_model * n)(*models), (C.c_int * n)(*ranks), C.byref(opt), C.byref(h))
    return st, h


def test_create_and_workspace_size(lib):
    st, h = _create(lib, [_model()], [4], _opts())
    assert st == 0
    sz = C.c_size_t()
    assert lib.lr_workspace_size(h, C.byref(sz)) == 0
    N, M = 40, 4
    # state arrays alone: Z_n + 3 scratch copies, complex128
    assert sz.value >= 4 * N * M * 16
    info = lr.lr_info()
    assert lib.lr_query(h, C.byref(info)) == 0
    assert (info.n_cand, info.n_traj, info.nt_max, info.n_rec) == (1, 2, 4, 101)
    lib.lr_destroy(h)


@pytest.mark.parametrize("bad", [
    dict(ranks=[0]), dict(ranks=[33]), dict(ranks=[41]),
    dict(opt=dict(max_steps=0)), dict(opt=dict(pop_every=0)), dict(opt=dict(eta=0.0)),
    dict(opt=dict(precision=7)), dict(opt=dict(engine=9)),
    dict(dims=(17, 4)), dict(dims=(0, 4)),
])
def test_create_rejects_bad_arguments(lib, bad):
    dims = bad.get("dims", (4, 10))
    st, h = _create(lib, [_model(dims)], bad.get("ranks", [4]), _opts(**bad.get("opt", {})))
    assert st == 1 and not h.value


def test_plain_engine_rejects_fp32(lib):
    st, h = _create(lib, [_model()], [4], _opts(precision=1, engine=1))
    assert st == 9


def test_calls_before_binding_fail_cleanly(lib):
    st, h = _create(lib, [_model()], [4], _opts())
    assert st == 0
    assert lib.lr_integrate(h, 1e-3, 10, None) == 4      # LR_ERR_WORKSPACE
    assert b"workspace" in lib.lr_last_error(h)
    assert lib.lr_set_initial(h, 1, 1e-5, None) == 4
    assert lib.lr_status_string(5) == b"Gram matrix not positive definite"
    lib.lr_destroy(h)
