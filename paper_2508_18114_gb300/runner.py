"""Convenience wrapper: run a batch of pulse candidates through the library.

A *workload* is any object with ``candidates`` (each with ``model``, ``M``
and ``pulse.kind`` / ``pulse.p``), ``dt``, ``n_steps``, ``tau``,
``init_seed``, ``eps`` and ``eta`` (``lr_inputs.Workload`` fits). This only
marshals arguments into :class:`LowRankBatch`; all arithmetic runs in the
CUDA library.
"""
from __future__ import annotations

from .lr import LowRankBatch


def make_batch(wl, precision=None, engine="auto", pop_every=1, max_steps=None, candidates=None,
               device="cuda:0", record_gram=False) -> LowRankBatch:
    """Batch for a workload's candidates, in the workload's frame (lab or rwa)."""
    cands = wl.candidates if candidates is None else [wl.candidates[i] for i in candidates]
    prec = precision or getattr(wl, "precision", "fp64")
    ms = wl.n_steps if max_steps is None else max_steps
    b = LowRankBatch([c.model for c in cands], [c.M for c in cands], precision=prec, engine=engine,
                     max_steps=ms, pop_every=pop_every, eta=wl.eta, device=device, record_gram=record_gram,
                     frame=getattr(wl, "frame", "lab"))
    b.set_pulse([(c.pulse.kind, c.pulse.p) for c in cands], wl.tau)
    return b


def run(wl, n_steps=None, precision=None, engine="auto", pop_every=1, candidates=None, device="cuda:0"):
    """Integrate from the seeded initial state; return host observables."""
    ns = wl.n_steps if n_steps is None else n_steps
    b = make_batch(wl, precision, engine, pop_every, ns, candidates, device)
    b.set_initial(wl.init_seed, wl.eps)
    b.integrate(wl.dt, ns)
    out = b.observables()
    out["engine"] = b.engine
    b.close()
    return out
