"""Seeded synthetic inputs for the low-rank readout workloads.

This module only *draws inputs*: model parameters, pulse parameters and the
uneven batch sizes of the five workloads. It holds none of the method's
arithmetic (no Hamiltonian, no equation of motion, no observable), so both
the CUDA path and the FP64 oracle may consume it.

Units are ns and rad/ns throughout (2*pi*1 GHz = 6.2832 rad/ns).

Workloads (each is a list of *candidates*; every candidate is run twice,
from the transmon ground state |g> and the first excited state |e>):

* ``c1`` - transmon 4 x resonator 10 (N=40), rank M=4, flat-top pulse,
  dt=1 ps, tau=40 ns.
* ``c2`` - transmon 10 x resonator 20 x filter 10 (N=2000), M=20,
  two-segment pulse, dt=0.5 ps.
* ``c3`` - 256 candidates with uneven truncations (N_t 6-12, N_r 15-30,
  N_f 8-12) and ranks (M 10-30).
* ``c4`` - 256 candidates on the c2 model (N=2000, M=20).
* ``c5`` - 64 candidates on transmon 10 x resonator 40 x filter 20
  (N=8000), M=32.
* ``paper`` - the paper's own normal-mode model (Sec. S2.B parameters),
  lower x upper normal mode x transmon = 100 x 4 x 5 (N=2000), M=20, 256
  flat-top pulses at the frame frequency.
"""
from .configs import (  # noqa: F401
    TWO_PI, Candidate, ModelParams, PulseParams, Workload, SplitMix64Stream,
    workload, sizes, c1, c2, c3, c4, c5, pulse_flat_top, pulse_two_segment,
    PaperWorkload, paper, paper_params,
)
