"""GPU parity of the sparse-operator engine on the paper's own model (Sec. S2)
against the FP64 oracle (Eq. S5 with the time-dependent operators of the frame
of the drive), through the C ABI."""
import numpy as np
import pytest

from oracle import init_state
from oracle import paper_model as pm
from oracle import pulse as opulse

pytestmark = pytest.mark.gpu

TP = 2.0 * np.pi
SEED, EPS = 20250818, 1e-5


def _params(**over):
    P = dict(Ec=TP * 0.315, Ej=51 * TP * 0.315, wr=TP * 7.2, wf=TP * 7.21, g=TP * 0.15, J=TP * 0.03,
             kappa=TP * 0.03, gamma=TP * 8e-6, wd=TP * 7.18)
    P.update(over)
    return P


# FP64: rounding-order differences only. FP32_G64: the state and the bulk
# products carry FP32 rounding (2^-24 relative) over a few hundred steps; the
# Gram matrix and the signal stay FP64-class. Bounds as for the fused engine.
TOL = {"fp64": dict(beta=1e-10, pops=1e-10, nphot=1e-10, trace=1e-11),
       "fp32_g64": dict(beta=5e-5, pops=5e-5, nphot=5e-5, trace=2e-5)}


def _run(dims, M, pulses, tau, dt, n_steps, pop_every, check_traj, params, split=None, precision="fp64",
         frame="rot", team=None):
    import torch
    from paper_2508_18114_gb300 import sparse
    Nl, Nu, Nt = dims
    model = sparse.paper_model(Nl, Nu, Nt, frame=frame, **params)
    T = len(pulses)
    psi = [i % 2 for i in range(T)]          # |0_l, 0_u, g> and |0_l, 0_u, e>
    b = sparse.SparseBatch(model, M, pulses, tau, n_steps, pop_every=pop_every, precision=precision)
    if team is not None:
        assert b.team == team
    b.set_initial(psi, SEED, EPS)
    if split:
        b.integrate(dt, split)
        b.integrate(dt, n_steps - split)
    else:
        b.integrate(dt, n_steps)
    got = b.observables()
    torch.cuda.synchronize()
    ora_model = pm.PaperModel(Nl, Nu, Nt, frame=frame, **params)
    for tj in check_traj:
        kind, p = pulses[tj]
        env = lambda t, kind=kind, p=p: opulse.envelope(kind, p, t, tau)  # noqa: E731
        m0 = init_state.initial_state(ora_model.N, M, psi[tj], EPS, SEED, tj)
        want = pm.integrate(m0, ora_model, env, dt, n_steps, pop_every=pop_every, low_rank=True)
        tol = TOL[precision]
        bs = np.abs(want["beta"]).max()
        assert np.abs(got["beta"][tj] - want["beta"]).max() <= tol["beta"] * max(bs, 1e-3), tj
        assert np.abs(got["pops"][tj] - want["pops"]).max() <= tol["pops"], tj
        assert np.abs(got["nphot"][tj] - want["nr"]).max() <= tol["nphot"] * max(want["nr"].max(), 1.0), tj
        assert np.abs(got["trace"][tj] - want["trace"]).max() <= tol["trace"], tj
    return got


@pytest.mark.parametrize("precision", ["fp64", "fp32_g64"])
def test_small_model_parity(precision):
    """N = 72 (6 x 3 x 4), M = 4, two candidates x {g, e}, strong short drive."""
    P = _params(g=TP * 0.3, kappa=1.0, gamma=0.05)
    wd = P["wd"]
    tau = 0.4
    pulses = [(0, [TP * 1.0, wd, 0.05, 0.0]), (0, [TP * 0.6, wd, 0.08, 0.0])] * 2
    pulses = [pulses[0], pulses[0], pulses[1], pulses[1]]
    got = _run((6, 3, 4), 4, pulses, tau, 5e-4, 800, 100, [0, 1, 3], P, precision=precision)
    assert np.abs(got["beta"][0]).max() > 1e-2           # the drive does displace the readout mode


@pytest.mark.parametrize("precision", ["fp64", "fp32_g64"])
def test_rwa_model_parity(precision):
    """The rotating-wave approximation of Eq. S(hamiltonian_rwa) on the same
    engine: N = 72 (6 x 3 x 4), M = 4, at a 5x larger step (2.5 ps) than the
    rotated-frame runs, two candidates x {g, e}."""
    P = _params(g=TP * 0.3, kappa=1.0, gamma=0.05)
    wd = P["wd"]
    tau = 2.0
    pulses = [(0, [TP * 1.0, wd, 0.25, 0.0])] * 2 + [(0, [TP * 0.6, wd, 0.4, 0.0])] * 2
    got = _run((6, 3, 4), 4, pulses, tau, 2.5e-3, 800, 100, [0, 1, 3], P, precision=precision, frame="rwa")
    assert np.abs(got["beta"][0]).max() > 1e-2


@pytest.mark.parametrize("precision", ["fp64", "fp32_g64"])
def test_ragged_blocks_and_split_integrate(precision):
    """N = 150 (10 x 3 x 5): nine full 16-row blocks and a 6-row tail; two
    integrate calls continue one run; two-segment pulse."""
    P = _params(kappa=2.0, gamma=0.1)
    wd = P["wd"]
    tau = 0.3
    pulses = [(1, [TP * 0.8, TP * 0.3, 0.15, 0.05, 0.05, 0.03, wd, 0.0])] * 2
    _run((10, 3, 5), 6, pulses, tau, 5e-4, 600, 50, [0, 1], P, split=257, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_g64"])
def test_full_size_sampled(precision):
    """The paper's Hilbert-space size N = 2000 (N_l = 100, N_u = 4, N_t = 5)
    at M = 20, 32 trajectories, 40 steps; trajectories 0 and 31 against the
    oracle. With 32 trajectories each Gram block sums 1 or 2 row tiles (63
    tiles of 32 rows in FP32, 125 of 16 in FP64, over 38 blocks)."""
    P = _params()
    wd = P["wd"]
    tau = 40.0
    pulses = [(0, [TP * (0.10 + 0.01 * (i // 2)), wd, 2.5, 0.0]) for i in range(32)]
    _run((100, 4, 5), 20, pulses, tau, 5e-4, 40, 10, [0, 31], P, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_g64"])
def test_large_rank(precision):
    """M = 28 (K = 2: 2352 partial sums per row tile, 10 per thread) on N = 150."""
    P = _params(kappa=2.0, gamma=0.1)
    wd = P["wd"]
    pulses = [(0, [TP * 0.8, wd, 0.05, 0.0])] * 2
    _run((10, 3, 5), 28, pulses, 0.3, 5e-4, 120, 40, [0, 1], P, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_g64"])
def test_assignment_error_and_loss(precision):
    """eps_a, T and Lambda (Sec. S3.A, S3.B) from the device records against the
    oracle's signal functions on the oracle's beta and populations."""
    from oracle import signal
    from paper_2508_18114_gb300 import sparse
    P = _params(g=TP * 0.3, kappa=1.0, gamma=0.05)
    wd, tau, dt, n, pe = P["wd"], 0.4, 5e-4, 800, 100
    dims, M = (6, 3, 4), 4
    pulses = [(0, [TP * 1.0, wd, 0.05, 0.0])] * 2 + [(0, [TP * 0.6, wd, 0.08, 0.0])] * 2
    model = sparse.paper_model(*dims, **P)
    b = sparse.SparseBatch(model, M, pulses, tau, n, pop_every=pe, precision=precision)
    b.set_initial([0, 1, 0, 1], SEED, EPS)
    b.integrate(dt, n)
    got = b.loss(P["kappa"], P["gamma"], eta=0.6)
    ora_model = pm.PaperModel(*dims, frame="rot", **P)
    # FP64: rounding order only. FP32_G64: eps_a relative 5e-5 (beta carries
    # ~1e-6 relative error); T is a sum of populations, absolute 5e-5 as the
    # populations; Lambda = log10(eps_a + T) then moves by at most ~5e-4.
    tol = 1e-10 if precision == "fp64" else 5e-5
    tol_T = (lambda T: 1e-10 * max(T, 1e-12)) if precision == "fp64" else (lambda T: 5e-5)
    tol_L = 1e-10 if precision == "fp64" else 5e-4
    for c in range(2):
        outs = []
        for tj in (2 * c, 2 * c + 1):
            kind, p = pulses[tj]
            env = lambda t, kind=kind, p=p: opulse.envelope(kind, p, t, tau)  # noqa: E731
            m0 = init_state.initial_state(ora_model.N, M, tj % 2, EPS, SEED, tj)
            outs.append(pm.integrate(m0, ora_model, env, dt, n, pop_every=pe, low_rank=True))
        ea = signal.assignment_error(outs[0]["beta"], outs[1]["beta"], dt, P["kappa"], P["gamma"], 0.6)
        T = signal.ionization(outs[0]["pops"], outs[1]["pops"], pe * dt, n * dt)
        assert abs(got["eps_a"][c] - ea) <= tol * ea, c
        assert abs(got["ion"][c] - T) <= tol_T(T) + 1e-15, c
        assert abs(got["loss"][c] - signal.loss(ea, T)) <= tol_L, c
    eps_sep = got["eps_a"] - 0.5 * n * dt * P["gamma"]   # minus eps_decay = tau gamma / 2
    assert np.all(eps_sep < 0.5) and np.all(eps_sep > 0.0)  # SNR > 0: the signals do separate


def test_capacity_and_errors():
    from paper_2508_18114_gb300 import lr, sparse
    P = _params()
    model = sparse.paper_model(4, 2, 3, **P)
    b = sparse.SparseBatch(model, 3, [(0, [1.0, P["wd"], 0.5, 0.0])] * 2, 1.0, 10)
    b.set_initial([0, 1], SEED, EPS)
    b.integrate(1e-3, 10)
    with pytest.raises(lr.LrError) as e:
        b.integrate(1e-3, 1)
    assert e.value.status == 8                           # LR_ERR_STATE past max_steps
    with pytest.raises(lr.LrError):
        b.set_initial([0, 99], SEED, EPS)                 # basis index out of range
    obs = b.observables()
    assert np.all(np.isfinite(obs["beta"]))


def test_fp32_state_round_trip():
    """set_state / get_state through the FP32 state: complex64 rounding only."""
    from paper_2508_18114_gb300 import sparse
    P = _params()
    model = sparse.paper_model(4, 2, 3, **P)
    b = sparse.SparseBatch(model, 3, [(0, [1.0, P["wd"], 0.5, 0.0])] * 2, 1.0, 10, precision="fp32_g64")
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((2, model["N"], 3)) + 1j * rng.standard_normal((2, model["N"], 3))
    b.set_state(Z, step=2)
    back = b.get_state()
    assert np.abs(back - Z.astype(np.complex64)).max() == 0.0


def _add_dephasing(model, gphi):
    """The builder's operator set plus a third jump operator sqrt(gphi) n_t
    (transmon dephasing, diagonal): the row entries of L_3 and -gphi/2 n_t^2 on
    the diagonal of A = -i H_eff."""
    N, K = model["N"], model["n_jumps"]
    Nt = model["dims"][2]
    rp, col, val, ch = model["rowptr"], model["col"], model["val"], model["chan"]
    jt = np.arange(N) % Nt
    ops = []
    for o in range(K + 2):
        r = rp[o * (N + 1):(o + 1) * (N + 1)]
        rows = []
        for n in range(N):
            sl = slice(r[n], r[n + 1])
            rows.append((col[sl].copy(), val[2 * r[n]:2 * r[n + 1]].copy(), ch[sl].copy()))
        ops.append(rows)
    for n in range(N):   # diagonal of A, channel 2 (static)
        c, v, h = ops[0][n]
        k = np.nonzero((c == n) & (h == 2))[0]
        assert k.size == 1
        v[2 * k[0]] += -0.5 * gphi * jt[n] ** 2
    l3 = [(np.array([n], np.int32), np.array([np.sqrt(gphi) * jt[n], 0.0]), np.array([2], np.uint8))
          for n in range(N)]
    ops = ops[:K + 1] + [l3] + ops[K + 1:]
    rowptr, cols, vals, chans, pos = [], [], [], [], 0
    for rows in ops:
        rowptr.append(pos)
        for c, v, h in rows:
            cols.append(c)
            vals.append(v)
            chans.append(h)
            pos += c.size
            rowptr.append(pos)
        rowptr.pop()
        rowptr.append(pos)
    out = dict(model)
    out.update(n_jumps=K + 1, nnz=pos, rowptr=np.array(rowptr, np.int32), col=np.concatenate(cols).astype(np.int32),
               val=np.concatenate(vals), chan=np.concatenate(chans).astype(np.uint8))
    assert out["rowptr"].size == (K + 3) * (N + 1)
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32_g64"])
def test_three_jump_operators(precision):
    """K = 3 (the engine's maximum): the paper model plus transmon dephasing."""
    import scipy.sparse as sp
    import torch
    from paper_2508_18114_gb300 import sparse
    P = _params(g=TP * 0.3, kappa=1.0, gamma=0.05)
    gphi = 0.7
    dims, M, dt, n, pe, tau = (6, 3, 4), 5, 5e-4, 400, 100, 0.2
    wd = P["wd"]
    pulses = [(0, [TP * 1.0, wd, 0.05, 0.0])] * 2
    model = _add_dephasing(sparse.paper_model(*dims, **P), gphi)
    b = sparse.SparseBatch(model, M, pulses, tau, n, pop_every=pe, precision=precision)
    b.set_initial([0, 1], SEED, EPS)
    b.integrate(dt, n)
    got = b.observables()
    torch.cuda.synchronize()
    ora = pm.PaperModel(*dims, frame="rot", **P)
    Nl, Nu, Nt = dims
    nt_op = sp.kron(sp.identity(Nl * Nu), sp.diags(np.arange(Nt, dtype=float)), format="csr").astype(complex)
    ora.jump_terms.append({pm.channel_index(0, 0): np.sqrt(gphi) * nt_op})
    tol = TOL[precision]
    for tj in (0, 1):
        env = lambda t: opulse.envelope(0, pulses[tj][1], t, tau)  # noqa: E731
        m0 = init_state.initial_state(ora.N, M, tj, EPS, SEED, tj)
        want = pm.integrate(m0, ora, env, dt, n, pop_every=pe, low_rank=True)
        bs = np.abs(want["beta"]).max()
        assert np.abs(got["beta"][tj] - want["beta"]).max() <= tol["beta"] * max(bs, 1e-3), tj
        assert np.abs(got["pops"][tj] - want["pops"]).max() <= tol["pops"], tj
        assert np.abs(got["trace"][tj] - want["trace"]).max() <= tol["trace"], tj


def test_two_contexts_keep_their_solve_memory():
    """A rank-32 context (solve shared memory above 48 KB) still integrates
    after a rank-4 context is bound: the kernel's limit only grows."""
    from paper_2508_18114_gb300 import sparse
    P = _params(kappa=2.0, gamma=0.1)
    wd = P["wd"]
    pulses = [(0, [TP * 0.8, wd, 0.05, 0.0])] * 2
    model = sparse.paper_model(10, 3, 5, **P)
    big = sparse.SparseBatch(model, 32, pulses, 0.1, 20, pop_every=10)
    small = sparse.SparseBatch(model, 4, pulses, 0.1, 20, pop_every=10)
    for b in (big, small):
        b.set_initial([0, 1], SEED, EPS)
    small.integrate(5e-4, 20)
    big.integrate(5e-4, 20)
    for b in (big, small):
        o = b.observables()
        assert np.all(np.isfinite(o["beta"])) and np.abs(o["trace"][:, -1] - 1.0).max() < 1e-3


def test_fused_kernel_runs_fp32_and_matches_the_launch_path(monkeypatch):
    """FP32_G64 contexts run the fused persistent kernel; it agrees with the
    four-launch path (same precision split, different summation order) within
    the FP32 rounding of a few hundred steps, on a batch with a ragged row
    count (N = 150) and three trajectories."""
    from paper_2508_18114_gb300 import sparse
    P = _params(kappa=2.0, gamma=0.1)
    wd = P["wd"]
    model = sparse.paper_model(10, 3, 5, **P)
    pulses = [(0, [TP * 0.8, wd, 0.05, 0.0]), (0, [TP * 0.5, wd, 0.05, 0.0]), (0, [TP * 0.3, wd, 0.05, 0.0])]
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("LR_SPARSE_FUSED", mode)
        b = sparse.SparseBatch(model, 6, pulses, 0.3, 600, pop_every=50, precision="fp32_g64")
        assert b.fused == (mode == "1")
        b.set_initial([0, 1, 0], SEED, EPS)
        b.integrate(5e-4, 257)
        b.integrate(5e-4, 343)
        out[mode] = b.observables()
        del b
    f, l = out["1"], out["0"]
    assert np.abs(f["beta"] - l["beta"]).max() <= 5e-5 * np.abs(l["beta"]).max()
    assert np.abs(f["pops"] - l["pops"]).max() <= 5e-5
    assert np.abs(f["trace"] - l["trace"]).max() <= 5e-5
    # FP64 contexts keep the four-launch path
    monkeypatch.delenv("LR_SPARSE_FUSED")
    b = sparse.SparseBatch(model, 6, pulses[:2], 0.3, 10, precision="fp64")
    assert not b.fused


def test_fused_split_schedule_is_bitwise(monkeypatch):
    """A batch with more trajectories than the grid has CTAs runs the equal-span
    schedule (trajectories cut between two CTAs hand their state over through
    global memory); every trajectory's arithmetic is unchanged, so the results
    equal bitwise those of the whole-trajectory schedule, over two calls whose
    spans cut trajectories at different steps."""
    import torch
    from paper_2508_18114_gb300 import sparse
    P = _params(kappa=2.0, gamma=0.1)
    wd = P["wd"]
    model = sparse.paper_model(10, 3, 5, **P)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    T = 2 * n_sm + 36
    pulses = [(0, [TP * (0.2 + 0.6 * ((7 * j) % 11) / 10.0), wd, 0.05, 0.0]) for j in range(T)]
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("LR_SPARSE_SPLIT", mode)
        b = sparse.SparseBatch(model, 6, pulses, 0.3, 100, pop_every=10, precision="fp32_g64")
        assert b.fused
        b.set_initial([j % 2 for j in range(T)], SEED, EPS)
        b.integrate(5e-4, 37)
        b.integrate(5e-4, 23)
        out[mode] = (b.observables(), b.get_state())
        del b
    (o1, z1), (o0, z0) = out["1"], out["0"]
    assert np.array_equal(o1["beta"][:, :61], o0["beta"][:, :61])
    for k in ("pops", "nphot", "trace"):   # records at steps 0, 10, ..., 60
        assert np.array_equal(o1[k][:, :7], o0[k][:, :7]), k
    assert np.array_equal(z1, z0)
    assert np.all(np.isfinite(o1["beta"][:, :61])) and np.abs(o1["trace"][:, 6] - 1.0).max() < 1e-3


@pytest.mark.parametrize("team", [2, 3, 7, 16])
def test_fused_teams_parity(monkeypatch, team):
    """Small batches run the fused kernel on teams of C CTAs (a cluster; each
    CTA owns N/C rows, the team adds its partial G, T_k and signal sums in
    rank order through distributed shared memory): parity with the oracle at
    the FP32_G64 bounds, N = 150 (ragged row ranges for C = 7 and 16), two
    integrate calls."""
    monkeypatch.setenv("LR_SPARSE_C", str(team))
    P = _params(g=TP * 0.3, kappa=1.0, gamma=0.05)
    wd = P["wd"]
    pulses = [(0, [TP * 0.9, wd, 0.05, 0.0]), (0, [TP * 0.9, wd, 0.05, 0.0]), (0, [TP * 0.5, wd, 0.08, 0.0]),
              (0, [TP * 0.5, wd, 0.08, 0.0])]
    got = _run((10, 3, 5), 6, pulses, 0.3, 5e-4, 600, 50, [0, 3], P, split=233, precision="fp32_g64", team=team)
    assert np.abs(got["beta"][0]).max() > 1e-2


def test_fused_team_default_for_small_batches():
    """Without an override, a two-trajectory batch of the N = 2000 model runs
    on teams of several CTAs, and a batch as large as the grid on one CTA per
    trajectory."""
    import torch
    from paper_2508_18114_gb300 import sparse
    P = _params()
    model = sparse.paper_model(100, 4, 5, **P)
    p = (0, [TP * 0.15, P["wd"], 2.5, 0.0])
    b = sparse.SparseBatch(model, 20, [p, p], 40.0, 10, precision="fp32_g64")
    assert b.team > 1
    del b
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    b = sparse.SparseBatch(model, 20, [p] * n_sm, 40.0, 10, precision="fp32_g64")
    assert b.team == 1


@pytest.mark.parametrize("dims,n_steps", [((10, 3, 5), 400), ((100, 4, 5), 120)])
def test_fused_gram_on_tensor_cores(monkeypatch, dims, n_steps):
    """LR_SPARSE_GRAM=tc at M = 20 runs the Gram matrix on the tensor cores
    (exact bf16 slices, accumulation windows of at most 1024 rows: two per
    stage at N = 2000, one at N = 150). Against the oracle at the FP32_G64
    bounds, and against the default double-word CUDA-core Gram within FP32
    rounding."""
    from paper_2508_18114_gb300 import sparse
    P = _params(kappa=2.0, gamma=0.1) if dims[0] == 10 else _params()
    wd = P["wd"]
    amp = TP * (0.8 if dims[0] == 10 else 0.15)
    pulses = [(0, [amp, wd, 0.05, 0.0])] * 2 + [(0, [0.6 * amp, wd, 0.05, 0.0])] * 2
    got = {}
    for mode in ("tc", "dw"):
        if mode == "tc":
            monkeypatch.setenv("LR_SPARSE_GRAM", "tc")
        else:
            monkeypatch.delenv("LR_SPARSE_GRAM", raising=False)
        model = sparse.paper_model(*dims, **P)
        b = sparse.SparseBatch(model, 20, pulses, 0.4, n_steps, pop_every=40, precision="fp32_g64")
        assert b.fused and b.gram_tc == (mode == "tc")
        b.set_initial([j % 2 for j in range(4)], SEED, EPS)
        b.integrate(5e-4, n_steps // 3)
        b.integrate(5e-4, n_steps - n_steps // 3)
        got[mode] = b.observables()
        del b
    t, d = got["tc"], got["dw"]
    scale = np.abs(d["beta"][:, :n_steps + 1]).max()
    assert np.abs(t["beta"][:, :n_steps + 1] - d["beta"][:, :n_steps + 1]).max() <= 2e-6 * max(scale, 1e-3)
    assert np.abs(t["pops"] - d["pops"]).max() <= 2e-6
    if dims[0] == 10:   # the oracle at the small size, tensor-core Gram
        monkeypatch.setenv("LR_SPARSE_GRAM", "tc")
        _run(dims, 20, pulses, 0.4, 5e-4, n_steps, 40, [0, 3], P, precision="fp32_g64")
