"""Seeded input recipes (model, pulse, batch shape) for the readout workloads.

Nothing here evaluates the physics; it only fixes numbers. The random draws
use a SplitMix64 stream (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): the k-th output for seed s is
mix64(s + (k+1)*0x9E3779B97F4A7C15) and a uniform in [0,1) is
(output >> 11) * 2**-53.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

TWO_PI = 2.0 * math.pi
_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64Stream:
    """Counter-based SplitMix64 uniform stream used for input draws."""

    def __init__(self, seed: int):
        self.seed = seed & _M64
        self.k = 0

    @staticmethod
    def mix(z: int) -> int:
        z &= _M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def next_u64(self) -> int:
        self.k += 1
        return self.mix(self.seed + self.k * _GOLDEN)

    def uniform(self) -> float:
        """Uniform in [0, 1)."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def uniform_open_low(self, hi: float) -> float:
        """Uniform in (0, hi]."""
        return hi * (1.0 - self.uniform())

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in {lo, ..., hi}."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


@dataclasses.dataclass(frozen=True)
class ModelParams:
    """Transmon (Duffing) x resonator [x filter] readout model parameters.

    ``dims`` = (N_t, N_r) or (N_t, N_r, N_f). The last mode is the driven,
    decaying readout mode. Frequencies in rad/ns, rates in 1/ns.
    """

    dims: tuple
    wq: float
    alpha: float
    wr: float
    g: float
    kappa: float
    gamma: float
    wf: float = 0.0
    J: float = 0.0

    @property
    def n_modes(self) -> int:
        return len(self.dims)

    @property
    def N(self) -> int:
        n = 1
        for d in self.dims:
            n *= d
        return n


@dataclasses.dataclass(frozen=True)
class PulseParams:
    """Pulse parameter vector.

    kind 0 (flat-top): p = (A, w_d, t_r, phi)
    kind 1 (two-segment): p = (A1, A2, t_sw, t_rise, t_fall, t_sm, w_d, phi)
    """

    kind: int
    p: tuple

    @property
    def n_params(self) -> int:
        return 4 if self.kind == 0 else 8


@dataclasses.dataclass(frozen=True)
class Candidate:
    model: ModelParams
    M: int
    pulse: PulseParams


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    candidates: List[Candidate]
    dt: float
    n_steps: int
    tau: float
    init_seed: int
    eps: float = 1e-5
    eta: float = 0.6
    precision: str = "fp64"
    note: str = ""
    frame: str = "lab"   # "rwa": frame rotating at w_d with the rotating-wave approximation

    @property
    def n_traj(self) -> int:
        return 2 * len(self.candidates)


def _c1_model() -> ModelParams:
    return ModelParams(dims=(4, 10), wq=TWO_PI * 6.0, alpha=-TWO_PI * 0.3,
                       wr=TWO_PI * 7.5, g=TWO_PI * 0.15,
                       kappa=TWO_PI * 0.01, gamma=1.0 / 50000.0)


def _filter_model(nt: int, nr: int, nf: int) -> ModelParams:
    wr = TWO_PI * 7.5
    return ModelParams(dims=(nt, nr, nf), wq=TWO_PI * 6.0, alpha=-TWO_PI * 0.3,
                       wr=wr, g=TWO_PI * 0.15, kappa=TWO_PI * 0.05,
                       gamma=1.0 / 50000.0, wf=wr + TWO_PI * 0.01,
                       J=TWO_PI * 0.1)


def pulse_flat_top(seed: int, wr: float) -> PulseParams:
    """Flat-top pulse draw: A in (0, 2pi*50 MHz], w_d in w_r +- 2pi*30 MHz,
    rise time in [1, 5] ns, phase in [0, 2pi)."""
    s = SplitMix64Stream(seed)
    A = s.uniform_open_low(TWO_PI * 0.05)
    wd = s.uniform_range(wr - TWO_PI * 0.03, wr + TWO_PI * 0.03)
    tr = s.uniform_range(1.0, 5.0)
    phi = s.uniform_range(0.0, TWO_PI)
    return PulseParams(0, (A, wd, tr, phi))


def pulse_two_segment(seed: int, wr: float) -> PulseParams:
    """Two-segment pulse draw: A1 in (0, 2pi*50 MHz], A2 in (0, A1],
    t_sw in [10, 30] ns, t_rise, t_fall, t_sm in [1, 5] ns,
    w_d in w_r +- 2pi*30 MHz, phase in [0, 2pi)."""
    s = SplitMix64Stream(seed)
    A1 = s.uniform_open_low(TWO_PI * 0.05)
    A2 = s.uniform_open_low(A1)
    t_sw = s.uniform_range(10.0, 30.0)
    t_rise = s.uniform_range(1.0, 5.0)
    t_fall = s.uniform_range(1.0, 5.0)
    t_sm = s.uniform_range(1.0, 5.0)
    wd = s.uniform_range(wr - TWO_PI * 0.03, wr + TWO_PI * 0.03)
    phi = s.uniform_range(0.0, TWO_PI)
    return PulseParams(1, (A1, A2, t_sw, t_rise, t_fall, t_sm, wd, phi))


def c1(n_steps: Optional[int] = None) -> Workload:
    m = _c1_model()
    cand = Candidate(m, 4, pulse_flat_top(1, m.wr))
    dt = 1e-3
    ns = 40000 if n_steps is None else n_steps
    return Workload("c1", [cand], dt, ns, ns * dt, init_seed=1001)


def c2(n_steps: Optional[int] = None, M: int = 20) -> Workload:
    m = _filter_model(10, 20, 10)
    cand = Candidate(m, M, pulse_two_segment(2, m.wr))
    dt = 5e-4
    ns = 80000 if n_steps is None else n_steps
    return Workload("c2", [cand], dt, ns, ns * dt, init_seed=1002)


def c3(n_candidates: int = 256, n_steps: Optional[int] = None, first: int = 0) -> Workload:
    """Candidates first .. first + n_candidates - 1 of the c3 population."""
    cands = []
    for i in range(first, first + n_candidates):
        s = SplitMix64Stream(0xC3000000 + i)
        nt = s.integer(6, 12)
        nr = s.integer(15, 30)
        nf = s.integer(8, 12)
        M = s.integer(10, 30)
        m = _filter_model(nt, nr, nf)
        cands.append(Candidate(m, M, pulse_two_segment(3 + i, m.wr)))
    dt = 5e-4
    ns = 80000 if n_steps is None else n_steps
    return Workload("c3", cands, dt, ns, ns * dt, init_seed=1003)


def c4(n_candidates: int = 256, n_steps: Optional[int] = None, first: int = 0) -> Workload:
    """Candidates first .. first + n_candidates - 1 of the c4 population."""
    m = _filter_model(10, 20, 10)
    cands = [Candidate(m, 20, pulse_two_segment(3 + i, m.wr)) for i in range(first, first + n_candidates)]
    dt = 5e-4
    ns = 80000 if n_steps is None else n_steps
    return Workload("c4", cands, dt, ns, ns * dt, init_seed=1004, precision="fp32_g64")


def c5(n_candidates: int = 64, n_steps: Optional[int] = None, first: int = 0) -> Workload:
    """Candidates first .. first + n_candidates - 1 of the c5 population."""
    m = _filter_model(10, 40, 20)
    cands = [Candidate(m, 32, pulse_two_segment(5 + i, m.wr)) for i in range(first, first + n_candidates)]
    dt = 5e-4
    ns = 80000 if n_steps is None else n_steps
    return Workload("c5", cands, dt, ns, ns * dt, init_seed=1005, precision="fp32_g64")


@dataclasses.dataclass(frozen=True)
class PaperWorkload:
    """Inputs of the paper's own model: parameters of Sec. S2.B (rad/ns, 1/ns),
    cutoffs, rank, step and a population of flat-top pulses (Sec. S2.C, ramp
    2.5 ns, drive at the frame frequency w_d, no phase)."""
    name: str
    params: dict
    dims: tuple
    M: int
    dt: float
    tau: float
    eps: float
    init_seed: int
    pulses: tuple        # ((kind, p), ...) per candidate


def paper_params() -> dict:
    """Sec. S2.B: E_c/2pi = 315 MHz, E_j/E_c = 51, g/2pi = 150 MHz,
    J/2pi = 30 MHz, w_r/2pi = 7.2 GHz, w_f/2pi = 7.21 GHz, kappa/2pi = 30 MHz
    (filter), gamma/2pi = 8 kHz (transmon), w_d/2pi = 7.18 GHz."""
    Ec = TWO_PI * 0.315
    return dict(Ec=Ec, Ej=51.0 * Ec, wr=TWO_PI * 7.2, wf=TWO_PI * 7.21, g=TWO_PI * 0.15, J=TWO_PI * 0.03,
                kappa=TWO_PI * 0.03, gamma=TWO_PI * 8e-6, wd=TWO_PI * 7.18)


def paper(n_candidates: int = 256, first: int = 0, dims=(100, 4, 5), M: int = 20) -> PaperWorkload:
    """Candidates first .. first + n_candidates - 1: flat-top amplitudes
    Omega/2pi drawn in (0, 300] MHz around the paper's 150 MHz square pulse.
    N = N_l N_u N_t = 2000 at the default cutoffs (the paper's Fig. 2 size)."""
    P = paper_params()
    pulses = []
    for i in range(first, first + n_candidates):
        s = SplitMix64Stream(8 + i)
        pulses.append((0, (s.uniform_open_low(TWO_PI * 0.3), P["wd"], 2.5, 0.0)))
    return PaperWorkload("paper", P, tuple(dims), M, 5e-4, 40.0, 1e-5, 1008, tuple(pulses))


def workload(name: str, **kw) -> Workload:
    return {"c1": c1, "c2": c2, "c3": c3, "c4": c4, "c5": c5}[name](**kw)


def sizes(w: Workload) -> Sequence[tuple]:
    """(N, M) per candidate."""
    return [(c.model.N, c.M) for c in w.candidates]
