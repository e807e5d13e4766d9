"""Binding of the paper's own model and the sparse-operator engine (argument
marshalling only; ``lr_paper_model_*`` and ``lr_sparse_*`` in include/lr.h).

``paper_model`` returns the CSR operator set that the library's host builder
makes for the normal-mode model of Sec. S2 (rotated frame, Eq.
S(hamiltonian_rotated)); ``SparseBatch`` integrates trajectories of any such
operator set on the GPU. The device workspace is a torch uint8 tensor owned by
the batch; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from typing import Sequence

import numpy as np

from .lr import PRECISION, LrError, _stream_ptr, load_library, make_pulse, lr_pulse

N_JUMPS_PAPER = 2       # kappa D[f] and gamma D[b]
PAPER_DERIVED = ("w_l", "w_u", "mu_l", "mu_u", "nu_l", "nu_u", "s21", "s22", "s23", "s24",
                 "qubit_frequency", "anharmonicity")


class lr_paper_params(C.Structure):
    _fields_ = [("Nl", C.c_int), ("Nu", C.c_int), ("Nt", C.c_int), ("n_cut", C.c_int),
                ("Ec", C.c_double), ("Ej", C.c_double), ("wr", C.c_double), ("wf", C.c_double),
                ("g", C.c_double), ("J", C.c_double), ("kappa", C.c_double), ("gamma", C.c_double),
                ("wd", C.c_double), ("frame", C.c_int)]


FRAME = {"rot": 0, "rwa": 1}


class lr_sparse_model(C.Structure):
    _fields_ = [("N", C.c_int), ("n_jumps", C.c_int), ("n_levels", C.c_int), ("nnz", C.c_long),
                ("wd", C.c_double), ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("chan", C.c_void_p), ("level", C.c_void_p)]


def _ptr(a: np.ndarray) -> C.c_void_p:
    return C.c_void_p(a.ctypes.data)


def paper_model(Nl: int, Nu: int, Nt: int, Ec: float, Ej: float, wr: float, wf: float, g: float,
                J: float, kappa: float, gamma: float, wd: float, n_cut: int = 20, frame: str = "rot") -> dict:
    """Operator set of the paper's model built by the library (host code).
    frame "rot": Eq. S(hamiltonian_rotated) with its counter-rotating terms;
    "rwa": the rotating-wave approximation, Eq. S(hamiltonian_rwa)."""
    lib = load_library()
    p = lr_paper_params(int(Nl), int(Nu), int(Nt), int(n_cut), float(Ec), float(Ej), float(wr), float(wf),
                        float(g), float(J), float(kappa), float(gamma), float(wd), FRAME[frame])
    N, nnz = C.c_int(), C.c_long()
    st = lib.lr_paper_model_size(C.byref(p), C.byref(N), C.byref(nnz))
    if st != 0:
        raise LrError(st, "lr_paper_model_size")
    n, z = N.value, nnz.value
    out = dict(N=n, nnz=z, n_jumps=N_JUMPS_PAPER, n_levels=int(Nt), wd=float(wd), dims=(Nl, Nu, Nt), frame=frame,
               rowptr=np.zeros(4 * (n + 1), np.int32), col=np.zeros(z, np.int32), val=np.zeros(2 * z),
               chan=np.zeros(z, np.uint8), level=np.zeros(n, np.int32), derived=np.zeros(16))
    st = lib.lr_paper_model_build(C.byref(p), _ptr(out["rowptr"]), _ptr(out["col"]), _ptr(out["val"]),
                                  _ptr(out["chan"]), _ptr(out["level"]), _ptr(out["derived"]))
    if st != 0:
        raise LrError(st, "lr_paper_model_build")
    out["params"] = dict(zip(PAPER_DERIVED, out["derived"][:len(PAPER_DERIVED)]))
    return out


class SparseBatch:
    """n_traj trajectories of rank M on one operator set (a ``paper_model`` dict
    or any dict with the same keys); pulse i drives trajectory i. precision:
    "fp64" or "fp32_g64"."""

    def __init__(self, model: dict, M: int, pulses: Sequence, tau: float, max_steps: int,
                 pop_every: int = 1, device="cuda:0", precision: str = "fp64"):
        import torch
        self._lib = load_library()
        self.model = model
        self._arrays = [np.ascontiguousarray(model[k], dtype=t) for k, t in
                        (("rowptr", np.int32), ("col", np.int32), ("val", np.float64), ("chan", np.uint8),
                         ("level", np.int32))]
        rp, col, val, ch, lev = self._arrays
        m = lr_sparse_model(int(model["N"]), int(model["n_jumps"]), int(model["n_levels"]), int(model["nnz"]),
                            float(model["wd"]), _ptr(rp), _ptr(col), _ptr(val), _ptr(ch),
                            _ptr(lev))
        pl = [q if isinstance(q, lr_pulse) else make_pulse(*q) for q in pulses]
        self.n_traj = len(pl)
        arr = (lr_pulse * self.n_traj)(*pl)
        h = C.c_void_p()
        self.precision = precision
        st = self._lib.lr_sparse_create(C.byref(m), self.n_traj, int(M), PRECISION[precision], arr, float(tau),
                                        int(max_steps), int(pop_every), C.byref(h))
        if st != 0:
            raise LrError(st, "lr_sparse_create")
        self._h = h
        self.N, self.M, self.max_steps, self.pop_every = int(model["N"]), int(M), int(max_steps), int(pop_every)
        self.n_rec = self.max_steps // self.pop_every + 1
        self.device = torch.device(device)
        sz = C.c_size_t()
        self._check(self._lib.lr_sparse_workspace_size(h, C.byref(sz)))
        self.workspace_bytes = int(sz.value)
        self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
        self._ws_ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        self._check(self._lib.lr_sparse_bind_workspace(h, C.c_void_p(self._ws_ptr), C.c_size_t(self.workspace_bytes),
                                                       C.c_void_p(_stream_ptr(None))))

    @property
    def fused(self) -> bool:
        """True when the context runs the fused persistent kernel."""
        f = C.c_int()
        self._check(self._lib.lr_sparse_query(self._h, C.byref(f), None, None))
        return bool(f.value)

    @property
    def gram_tc(self) -> bool:
        """True when the fused kernel forms the Gram matrix on the tensor cores."""
        f, g = C.c_int(), C.c_int()
        self._check(self._lib.lr_sparse_query(self._h, C.byref(f), None, C.byref(g)))
        return bool(g.value)

    @property
    def team(self) -> int:
        """CTAs per trajectory of the fused kernel (0: the four-launch path)."""
        f, t = C.c_int(), C.c_int()
        self._check(self._lib.lr_sparse_query(self._h, C.byref(f), C.byref(t), None))
        return t.value

    def _check(self, st: int):
        if st != 0:
            msg = self._lib.lr_sparse_last_error(self._h)
            raise LrError(st, msg.decode() if msg else "")

    def set_initial(self, psi: Sequence[int], seed: int, eps: float = 1e-5, stream=None):
        a = (C.c_int * self.n_traj)(*[int(x) for x in psi])
        self._check(self._lib.lr_sparse_set_initial(self._h, a, C.c_uint64(seed), float(eps),
                                                    C.c_void_p(_stream_ptr(stream))))

    def set_state(self, Z: np.ndarray, step: int = 0, stream=None):
        z = np.ascontiguousarray(Z, dtype=np.complex128).reshape(self.n_traj, self.N, self.M)
        self._check(self._lib.lr_sparse_set_state(self._h, _ptr(z), int(step), C.c_void_p(_stream_ptr(stream))))

    def get_state(self, stream=None) -> np.ndarray:
        z = np.zeros((self.n_traj, self.N, self.M), np.complex128)
        self._check(self._lib.lr_sparse_get_state(self._h, _ptr(z), C.c_void_p(_stream_ptr(stream))))
        return z

    def integrate(self, dt: float, n_steps: int, stream=None):
        self._check(self._lib.lr_sparse_integrate(self._h, float(dt), int(n_steps), C.c_void_p(_stream_ptr(stream))))

    def observables(self, stream=None) -> dict:
        beta = np.zeros((self.n_traj, self.max_steps + 1), np.complex128)
        pops = np.zeros((self.n_traj, self.n_rec, int(self.model["n_levels"])))
        nphot = np.zeros((self.n_traj, self.n_rec))
        trace = np.zeros((self.n_traj, self.n_rec))
        self._check(self._lib.lr_sparse_observables(self._h, _ptr(beta), _ptr(pops), _ptr(nphot), _ptr(trace),
                                                    C.c_void_p(_stream_ptr(stream))))
        return dict(beta=beta, pops=pops, nphot=nphot, trace=trace)

    def loss(self, kappa: float, gamma: float, eta: float = 0.6, stream=None) -> dict:
        """eps_a, ionization T and Lambda per candidate (trajectories 2c, 2c+1 =
        |g>, |e>) over the steps integrated so far (Sec. S3.A, S3.B)."""
        nc = self.n_traj // 2
        out = {k: np.zeros(nc) for k in ("eps_a", "ion", "loss")}
        self._check(self._lib.lr_sparse_loss(self._h, float(eta), float(kappa), float(gamma), _ptr(out["eps_a"]),
                                             _ptr(out["ion"]), _ptr(out["loss"]), C.c_void_p(_stream_ptr(stream))))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and self._lib is not None:
            self._lib.lr_sparse_destroy(h)
            self._h = None


class FullME:
    """One trajectory of the full master equation (FP64, N x N density matrix)
    for an operator set from ``paper_model`` (lr_full_*): the reference run that
    low-rank batches of the same model are compared with and timed against."""

    def __init__(self, model: dict, pulse, tau: float, max_steps: int, pop_every: int = 1, device="cuda:0"):
        import torch
        self._lib = load_library()
        self.model = model
        self._arrays = [np.ascontiguousarray(model[k], dtype=t) for k, t in
                        (("rowptr", np.int32), ("col", np.int32), ("val", np.float64), ("chan", np.uint8),
                         ("level", np.int32))]
        rp, col, val, ch, lev = self._arrays
        m = lr_sparse_model(int(model["N"]), int(model["n_jumps"]), int(model["n_levels"]), int(model["nnz"]),
                            float(model["wd"]), _ptr(rp), _ptr(col), _ptr(val), _ptr(ch), _ptr(lev))
        pl = pulse if isinstance(pulse, lr_pulse) else make_pulse(*pulse)
        h = C.c_void_p()
        st = self._lib.lr_full_create(C.byref(m), C.byref(pl), float(tau), int(max_steps), int(pop_every),
                                      C.byref(h))
        if st != 0:
            raise LrError(st, "lr_full_create")
        self._h = h
        self.N, self.max_steps, self.pop_every = int(model["N"]), int(max_steps), int(pop_every)
        self.n_rec = self.max_steps // self.pop_every + 1
        sz = C.c_size_t()
        self._check(self._lib.lr_full_workspace_size(h, C.byref(sz)))
        self.workspace = torch.empty(int(sz.value) + 256, dtype=torch.uint8, device=torch.device(device))
        ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        self._check(self._lib.lr_full_bind_workspace(h, C.c_void_p(ptr), sz, C.c_void_p(_stream_ptr(None))))

    def _check(self, st: int):
        if st != 0:
            msg = self._lib.lr_full_last_error(self._h)
            raise LrError(st, msg.decode() if msg else "")

    def set_initial(self, psi: int, stream=None):
        self._check(self._lib.lr_full_set_initial(self._h, int(psi), C.c_void_p(_stream_ptr(stream))))

    def set_state(self, rho: np.ndarray, step: int = 0, stream=None):
        r = np.ascontiguousarray(rho, dtype=np.complex128).reshape(self.N, self.N)
        self._check(self._lib.lr_full_set_state(self._h, _ptr(r), int(step), C.c_void_p(_stream_ptr(stream))))

    def set_state_lowrank(self, Z: np.ndarray, step: int = 0, stream=None):
        """rho = Z Z^dag from a low-rank factor Z [N][M] (computed on the device)."""
        z = np.ascontiguousarray(Z, dtype=np.complex128)
        self._check(self._lib.lr_full_set_state_lowrank(self._h, _ptr(z), int(z.shape[1]), int(step),
                                                        C.c_void_p(_stream_ptr(stream))))

    def get_state(self, stream=None) -> np.ndarray:
        r = np.zeros((self.N, self.N), np.complex128)
        self._check(self._lib.lr_full_get_state(self._h, _ptr(r), C.c_void_p(_stream_ptr(stream))))
        return r

    def integrate(self, dt: float, n_steps: int, stream=None):
        self._check(self._lib.lr_full_integrate(self._h, float(dt), int(n_steps), C.c_void_p(_stream_ptr(stream))))

    def observables(self, stream=None) -> dict:
        beta = np.zeros(self.max_steps + 1, np.complex128)
        pops = np.zeros((self.n_rec, int(self.model["n_levels"])))
        nphot = np.zeros(self.n_rec)
        trace = np.zeros(self.n_rec)
        self._check(self._lib.lr_full_observables(self._h, _ptr(beta), _ptr(pops), _ptr(nphot), _ptr(trace),
                                                  C.c_void_p(_stream_ptr(stream))))
        return dict(beta=beta, pops=pops, nphot=nphot, trace=trace)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and self._lib is not None:
            self._lib.lr_full_destroy(h)
            self._h = None
