"""Thin ctypes binding of ``include/lr.h`` (argument marshalling only).

Every computation happens in the CUDA library ``liblr.so``; this module only
converts Python values to the C structs, owns the device workspace (a torch
uint8 tensor) and passes torch's current CUDA stream. If the library is
missing the import fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblr.so")

LR_MAX_RANK = 32
LR_MAX_NT = 16

STATUS = {
    0: "LR_OK", 1: "LR_ERR_ARG", 2: "LR_ERR_CUDA", 3: "LR_ERR_NOMEM",
    4: "LR_ERR_WORKSPACE", 5: "LR_ERR_NOT_PD", 6: "LR_ERR_NONFINITE",
    7: "LR_ERR_TIMEOUT", 8: "LR_ERR_STATE", 9: "LR_ERR_UNSUPPORTED",
}
PRECISION = {"fp64": 0, "fp32_g64": 1, "fp32": 2, "tf32_g64": 3}
ENGINE = {"auto": 0, "plain": 1, "fused": 2}
FRAME = {"lab": 0, "rwa": 1}
ENGINE_NAME = {v: k for k, v in ENGINE.items()}

# exported names declared in include/lr.h
EXPORTS = (
    "lr_create", "lr_workspace_size", "lr_bind_workspace", "lr_set_pulse",
    "lr_set_initial", "lr_set_state", "lr_get_state", "lr_integrate",
    "lr_observables", "lr_sync", "lr_query", "lr_status_string",
    "lr_last_error", "lr_destroy", "lr_integrate_plain_noalloc",
    "lr_backward_workspace_size", "lr_backward", "lr_loss", "lr_diagnostics",
    "lr_paper_model_size", "lr_paper_model_build", "lr_sparse_create", "lr_sparse_workspace_size",
    "lr_sparse_bind_workspace", "lr_sparse_set_initial", "lr_sparse_set_state", "lr_sparse_get_state",
    "lr_sparse_integrate", "lr_sparse_observables", "lr_sparse_loss", "lr_sparse_last_error",
    "lr_sparse_destroy", "lr_grow_rank", "lr_measure_peak", "lr_sparse_query",
    "lr_full_create", "lr_full_workspace_size", "lr_full_bind_workspace", "lr_full_set_initial",
    "lr_full_set_state", "lr_full_set_state_lowrank", "lr_full_get_state", "lr_full_integrate", "lr_full_observables", "lr_full_last_error",
    "lr_full_destroy", "lr_assignment_shots",
)


class LrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class lr_model(C.Structure):
    _fields_ = [("n_modes", C.c_int), ("dims", C.c_int * 3),
                ("wq", C.c_double), ("alpha", C.c_double),
                ("wr", C.c_double), ("wf", C.c_double),
                ("g", C.c_double), ("J", C.c_double),
                ("kappa", C.c_double), ("gamma", C.c_double)]


class lr_pulse(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 8)]


class lr_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("engine", C.c_int),
                ("max_steps", C.c_long), ("pop_every", C.c_int),
                ("eta", C.c_double), ("record_gram", C.c_int), ("frame", C.c_int)]


class lr_info(C.Structure):
    _fields_ = [("n_cand", C.c_int), ("n_traj", C.c_int), ("nt_max", C.c_int),
                ("n_rec", C.c_long), ("max_steps", C.c_long), ("step", C.c_long),
                ("engine", C.c_int), ("team_size", C.c_int),
                ("stage_in_smem", C.c_int), ("tensor_passes", C.c_int), ("gram_tc", C.c_int)]


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load liblr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("liblr.so not found at %s: build it with "
                          "`python -m paper_2508_18114_gb300.build`" % path)
    lib = C.CDLL(path)
    vp, i, l, d = C.c_void_p, C.c_int, C.c_long, C.c_double
    lib.lr_create.argtypes = [i, C.POINTER(lr_model), C.POINTER(C.c_int), C.POINTER(lr_options), C.POINTER(vp)]
    lib.lr_workspace_size.argtypes = [vp, C.POINTER(C.c_size_t)]
    lib.lr_bind_workspace.argtypes = [vp, vp, C.c_size_t]
    lib.lr_set_pulse.argtypes = [vp, C.POINTER(lr_pulse), d, vp]
    lib.lr_set_initial.argtypes = [vp, C.c_uint64, d, vp]
    lib.lr_set_state.argtypes = [vp, i, vp, l, vp]
    lib.lr_get_state.argtypes = [vp, i, vp, vp]
    lib.lr_integrate.argtypes = [vp, d, l, vp]
    lib.lr_observables.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.lr_sync.argtypes = [vp, vp]
    lib.lr_query.argtypes = [vp, C.POINTER(lr_info)]
    lib.lr_status_string.argtypes = [i]
    lib.lr_status_string.restype = C.c_char_p
    lib.lr_last_error.argtypes = [vp]
    lib.lr_last_error.restype = C.c_char_p
    lib.lr_destroy.argtypes = [vp]
    lib.lr_destroy.restype = None
    lib.lr_integrate_plain_noalloc.argtypes = [C.POINTER(lr_model), i, C.POINTER(lr_pulse), d, vp, vp, d, l, l, vp]
    lib.lr_backward_workspace_size.argtypes = [vp, i, C.POINTER(C.c_size_t)]
    lib.lr_backward.argtypes = [vp, vp, C.c_size_t, vp, vp, i, vp]
    lib.lr_loss.argtypes = [vp, vp, vp, vp]
    lib.lr_assignment_shots.argtypes = [vp, d, l, i, C.c_uint64, vp, vp, vp, vp]
    lib.lr_diagnostics.argtypes = [vp, vp, vp, vp]
    lib.lr_paper_model_size.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_long)]
    lib.lr_paper_model_build.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.lr_sparse_create.argtypes = [vp, i, i, i, vp, d, l, i, C.POINTER(vp)]
    lib.lr_sparse_workspace_size.argtypes = [vp, C.POINTER(C.c_size_t)]
    lib.lr_sparse_bind_workspace.argtypes = [vp, vp, C.c_size_t, vp]
    lib.lr_sparse_set_initial.argtypes = [vp, vp, C.c_uint64, d, vp]
    lib.lr_sparse_set_state.argtypes = [vp, vp, l, vp]
    lib.lr_sparse_get_state.argtypes = [vp, vp, vp]
    lib.lr_sparse_integrate.argtypes = [vp, d, l, vp]
    lib.lr_sparse_observables.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.lr_sparse_loss.argtypes = [vp, d, d, d, vp, vp, vp, vp]
    lib.lr_grow_rank.argtypes = [vp, vp, C.c_uint64, d, vp]
    lib.lr_measure_peak.argtypes = [i, C.POINTER(d), C.POINTER(d), vp]
    lib.lr_sparse_query.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.lr_full_create.argtypes = [vp, C.POINTER(lr_pulse), d, l, i, C.POINTER(vp)]
    lib.lr_full_workspace_size.argtypes = [vp, C.POINTER(C.c_size_t)]
    lib.lr_full_bind_workspace.argtypes = [vp, vp, C.c_size_t, vp]
    lib.lr_full_set_initial.argtypes = [vp, i, vp]
    lib.lr_full_set_state.argtypes = [vp, vp, l, vp]
    lib.lr_full_get_state.argtypes = [vp, vp, vp]
    lib.lr_full_set_state_lowrank.argtypes = [vp, vp, i, l, vp]
    lib.lr_full_integrate.argtypes = [vp, d, l, vp]
    lib.lr_full_observables.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.lr_full_last_error.argtypes = [vp]
    lib.lr_full_last_error.restype = C.c_char_p
    lib.lr_full_destroy.argtypes = [vp]
    lib.lr_full_destroy.restype = None
    lib.lr_sparse_last_error.argtypes = [vp]
    lib.lr_sparse_last_error.restype = C.c_char_p
    lib.lr_sparse_destroy.argtypes = [vp]
    lib.lr_sparse_destroy.restype = None
    for name in EXPORTS:
        if name not in ("lr_status_string", "lr_last_error", "lr_destroy", "lr_sparse_last_error",
                        "lr_sparse_destroy", "lr_full_last_error", "lr_full_destroy"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_model(p) -> lr_model:
    """lr_model from an object with dims, wq, alpha, wr, g, kappa, gamma[, wf, J]."""
    m = lr_model()
    dims = tuple(p.dims)
    m.n_modes = len(dims)
    for k in range(3):
        m.dims[k] = dims[k] if k < len(dims) else 1
    m.wq, m.alpha, m.wr = p.wq, p.alpha, p.wr
    m.wf, m.g, m.J = getattr(p, "wf", 0.0), p.g, getattr(p, "J", 0.0)
    m.kappa, m.gamma = p.kappa, p.gamma
    return m


def make_pulse(kind: int, params: Sequence[float]) -> lr_pulse:
    q = lr_pulse()
    q.kind = int(kind)
    for k, v in enumerate(params):
        q.p[k] = float(v)
    return q


PEAK_KIND = {"fp32_fma": 0, "fp64_fma": 1, "tf32_mma": 2}


def measure_peak(kind: str, stream=None):
    """(flop/s, seconds) of the arithmetic-pipe microbenchmark lr_measure_peak."""
    lib = load_library()
    f, sec = C.c_double(), C.c_double()
    st = lib.lr_measure_peak(PEAK_KIND[kind], C.byref(f), C.byref(sec), C.c_void_p(_stream_ptr(stream)))
    if st != 0:
        raise LrError(st, "lr_measure_peak(%s)" % kind)
    return f.value, sec.value


def integrate_plain_noalloc(model, M, pulse, tau, Z, beta, dt, step0, n_steps, stream=None):
    """lr_integrate_plain_noalloc on caller device tensors (no workspace).

    Z: complex128 device tensor [N, M], advanced in place; beta: complex128
    device tensor with at least n_steps + 1 entries. Returns the lr status.
    """
    lib = load_library()
    m = make_model(model)
    q = make_pulse(*pulse)
    return lib.lr_integrate_plain_noalloc(C.byref(m), int(M), C.byref(q), float(tau),
                                          C.c_void_p(Z.data_ptr()), C.c_void_p(beta.data_ptr()),
                                          float(dt), int(step0), int(n_steps),
                                          C.c_void_p(_stream_ptr(stream)))


class LowRankBatch:
    """A batch of candidates (pulses) x {|g>, |e>} trajectories on one GPU.

    models / ranks: per candidate. The device workspace is a torch tensor
    owned by this object.
    """

    def __init__(self, models, ranks, precision="fp64", engine="auto", max_steps=1000,
                 pop_every=1, eta=0.6, device="cuda:0", record_gram=False, frame="lab"):
        import torch
        self._lib = load_library()
        n = len(models)
        if n == 0 or len(ranks) != n:
            raise ValueError("need one rank per model")
        arr = (lr_model * n)(*[make_model(m) for m in models])
        rk = (C.c_int * n)(*[int(r) for r in ranks])
        opt = lr_options(PRECISION[precision], ENGINE[engine], int(max_steps), int(pop_every), float(eta),
                         1 if record_gram else 0, FRAME[frame])
        h = C.c_void_p()
        st = self._lib.lr_create(n, arr, rk, C.byref(opt), C.byref(h))
        if st != 0:
            raise LrError(st, "lr_create failed")
        self._h = h
        self.models = list(models)
        self.ranks = [int(r) for r in ranks]
        self.precision = precision
        self.options = dict(precision=precision, engine=engine, max_steps=int(max_steps), pop_every=int(pop_every),
                            eta=float(eta), record_gram=bool(record_gram), frame=frame)
        self.device = torch.device(device)
        sz = C.c_size_t()
        self._check(self._lib.lr_workspace_size(h, C.byref(sz)))
        self.workspace_bytes = int(sz.value)
        self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self._check(self._lib.lr_bind_workspace(h, C.c_void_p(self._ws_ptr), C.c_size_t(self.workspace_bytes)))
        self.info = self.query()

    # ------------------------------------------------------------ helpers
    def _check(self, st: int):
        if st != 0:
            msg = self._lib.lr_last_error(self._h)
            raise LrError(st, msg.decode() if msg else "")

    def query(self) -> lr_info:
        info = lr_info()
        self._check(self._lib.lr_query(self._h, C.byref(info)))
        return info

    @property
    def engine(self) -> str:
        return ENGINE_NAME[self.query().engine]

    @property
    def n_traj(self) -> int:
        return 2 * len(self.models)

    # ------------------------------------------------------------ calls
    def set_pulse(self, pulses, tau: float, stream=None):
        """pulses: sequence of (kind, params)."""
        n = len(self.models)
        arr = (lr_pulse * n)(*[make_pulse(k, p) for k, p in pulses])
        self._check(self._lib.lr_set_pulse(self._h, arr, float(tau), C.c_void_p(_stream_ptr(stream))))

    def set_initial(self, seed: int, eps: float = 1e-5, stream=None):
        self._check(self._lib.lr_set_initial(self._h, C.c_uint64(seed), float(eps),
                                             C.c_void_p(_stream_ptr(stream))))

    def _NM(self, traj: int):
        m = self.models[traj // 2]
        N = int(np.prod(m.dims))
        return N, self.ranks[traj // 2]

    def set_state(self, traj: int, Z: np.ndarray, step: int = 0, stream=None):
        N, M = self._NM(traj)
        z = np.ascontiguousarray(np.asarray(Z, dtype=np.complex128).reshape(N, M))
        self._check(self._lib.lr_set_state(self._h, int(traj), z.ctypes.data_as(C.c_void_p), int(step),
                                           C.c_void_p(_stream_ptr(stream))))

    def get_state(self, traj: int, stream=None) -> np.ndarray:
        N, M = self._NM(traj)
        z = np.empty((N, M), dtype=np.complex128)
        self._check(self._lib.lr_get_state(self._h, int(traj), z.ctypes.data_as(C.c_void_p),
                                           C.c_void_p(_stream_ptr(stream))))
        return z

    def integrate(self, dt: float, n_steps: int, stream=None):
        self._check(self._lib.lr_integrate(self._h, float(dt), int(n_steps), C.c_void_p(_stream_ptr(stream))))

    def capture_integrate(self, dt: float, n_steps: int):
        """A CUDA graph (torch.cuda.CUDAGraph) of lr_integrate(dt, n_steps) on
        the fused engine: every graph.replay() continues the pulse run by
        n_steps (the step counter is read and advanced on the device). Call
        sync() after replays to refresh the host's view of the step counter."""
        import torch
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.graph(g, stream=side):
            self._check(self._lib.lr_integrate(self._h, float(dt), int(n_steps), C.c_void_p(side.cuda_stream)))
        torch.cuda.current_stream(self.device).wait_stream(side)
        self.sync()   # capture ran nothing: bring the host's step counter back
        return g

    def sync(self, stream=None):
        self._check(self._lib.lr_sync(self._h, C.c_void_p(_stream_ptr(stream))))

    def observables(self, stream=None, out=None):
        """Host copies of the recorded observables (numpy), see lr_observables."""
        info = self.query()
        nt, nrec, ms = info.nt_max, info.n_rec, info.max_steps
        o = out or {}
        beta = o.get("beta", np.empty((self.n_traj, ms + 1, 2)))
        pops = o.get("pops", np.empty((self.n_traj, nrec, nt)))
        nphot = o.get("nphot", np.empty((self.n_traj, nrec)))
        trace = o.get("trace", np.empty((self.n_traj, nrec)))
        eps = o.get("eps_a", np.empty(len(self.models)))
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
        self._check(self._lib.lr_observables(self._h, ptr(beta), ptr(pops), ptr(nphot), ptr(trace), ptr(eps),
                                             C.c_void_p(_stream_ptr(stream))))
        step = info.step
        return {
            "beta": beta[..., 0] + 1j * beta[..., 1],
            "pops": pops, "nphot": nphot, "trace": trace, "eps_a": eps, "step": step,
        }

    def observables_device(self, tensors, stream=None):
        """Copy observables into caller device tensors (dict of torch tensors)."""
        ptr = lambda k: C.c_void_p(tensors[k].data_ptr()) if k in tensors else None  # noqa: E731
        self._check(self._lib.lr_observables(self._h, ptr("beta"), ptr("pops"), ptr("nphot"),
                                             ptr("trace"), ptr("eps_a"), C.c_void_p(_stream_ptr(stream))))

    def loss(self, stream=None):
        """(ionization T, loss log10(eps_a + T)) per candidate (lr_loss)."""
        n = len(self.models)
        ion, loss = np.empty(n), np.empty(n)
        self._check(self._lib.lr_loss(self._h, ion.ctypes.data_as(C.c_void_p), loss.ctypes.data_as(C.c_void_p),
                                      C.c_void_p(_stream_ptr(stream))))
        return ion, loss

    def assignment_shots(self, n_shots: int, seed: int, bin_steps: int = 1, eta: float = None, stream=None) -> dict:
        """Seeded single-shot readout (lr_assignment_shots): per candidate the
        empirical assignment error eps_shots, the binned closed form eps_bin it
        converges to, and the misassigned g and e shots."""
        n = len(self.models)
        es, eb = np.empty(n), np.empty(n)
        err = np.empty((n, 2), dtype=np.int64)
        self._check(self._lib.lr_assignment_shots(self._h, float(self.options["eta"] if eta is None else eta), int(n_shots),
                                                  int(bin_steps), C.c_uint64(seed), es.ctypes.data_as(C.c_void_p),
                                                  eb.ctypes.data_as(C.c_void_p), err.ctypes.data_as(C.c_void_p),
                                                  C.c_void_p(_stream_ptr(stream))))
        return {"eps_shots": es, "eps_bin": eb, "errors": err}

    def grown(self, ranks, seed: int, eps: float = 1e-5, stream=None) -> "LowRankBatch":
        """A new batch with ranks >= the current ones that continues this pulse
        run (lr_grow_rank): the states keep their columns and gain orthonormal
        padding columns of weight eps; pulses, step and records are copied."""
        dst = LowRankBatch(self.models, ranks, device=self.device, **self.options)
        dst._check(self._lib.lr_grow_rank(dst._h, self._h, C.c_uint64(seed), float(eps),
                                          C.c_void_p(_stream_ptr(stream))))
        dst.info = dst.query()
        return dst

    def diagnostics(self, stream=None):
        """(purity [n_traj, n_rec], eigenvalues [n_traj, n_rec, max_M] descending)
        of rho = Z Z^dag at the record steps (lr_diagnostics; needs record_gram)."""
        info = self.query()
        nrec, mm = info.n_rec, max(self.ranks)
        pur = np.zeros((self.n_traj, nrec))
        eig = np.zeros((self.n_traj, nrec, mm))
        self._check(self._lib.lr_diagnostics(self._h, pur.ctypes.data_as(C.c_void_p), eig.ctypes.data_as(C.c_void_p),
                                             C.c_void_p(_stream_ptr(stream))))
        return pur, eig

    def backward(self, d_eps_a, ckpt_every=200, stream=None):
        """dL/dtheta [n_cand, 8] for cotangents dL/deps_a (lr_backward)."""
        import torch
        n = len(self.models)
        g = np.ascontiguousarray(np.asarray(d_eps_a, dtype=np.float64).reshape(n))
        sz = C.c_size_t()
        self._check(self._lib.lr_backward_workspace_size(self._h, int(ckpt_every), C.byref(sz)))
        ws = torch.empty(int(sz.value) + 256, dtype=torch.uint8, device=self.device)
        ptr = (ws.data_ptr() + 255) // 256 * 256
        out = np.zeros((n, 8))
        self._check(self._lib.lr_backward(self._h, C.c_void_p(ptr), sz, g.ctypes.data_as(C.c_void_p),
                                          out.ctypes.data_as(C.c_void_p), int(ckpt_every),
                                          C.c_void_p(_stream_ptr(stream))))
        del ws
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
