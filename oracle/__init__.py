"""Plain FP64 CPU oracle for the low-rank Lindblad readout path.

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously-correct
reference that the CUDA path is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the product library never does and shares no code with it.

Everything here is complex128 / float64 and follows the paper's equations in
their printed order:

* ``model``      - the Hamiltonian (Eq. 1, in the bare-mode Duffing form of
                   the workloads) and the jump operators (Eq. 2).
* ``pulse``      - logistic flat-top and smoothed stepwise envelopes
                   (Eq. S(square pulse) and the stepwise form of Sec. S2.C).
* ``lowrank``    - the non-stochastic matrix Schroedinger equation
                   (Eq. S5 with O[m] and the Moore-Penrose inverse, Sec. S1.A)
                   integrated with classical RK4.
* ``lindblad``   - the full N x N Lindblad master equation (Eq. 2 / Eq. S4),
                   classical RK4.
* ``signal``     - SNR, separation error and assignment error (Eqs. S-SNR,
                   S-separation_error, S-assignment_error, Sec. S3.A).
* ``init_state`` - the fixed-rank initial condition of Sec. S1.A (random
                   orthonormal padding states with weight eps).
* ``gradient``   - central finite-difference gradient of the assignment error
                   with respect to the pulse parameters.
* ``diagnostics`` - spectrum of rho = m m^dag and purity tr(rho^2) (Sec. S1.B).
* ``adaptive``   - rank control: spectrum test after each segment and rank
                   growth by orthonormal padding columns (Sec. S1.B).
* ``paper_model`` - the paper's own model: charge-basis transmon, normal modes
                   of the resonator-filter pair, the Hamiltonian in the frame of
                   the drive with its e^{+-2i w_d t} terms (Sec. S2.A, S2.D,
                   S2.E), and RK4 integrators of Eq. S5 and Eq. S4 with
                   time-dependent operators.

Parity status of each function is stated in its module docstring.
"""
from . import model, pulse, lowrank, lindblad, signal, init_state, gradient, diagnostics, paper_model, adaptive  # noqa: F401
