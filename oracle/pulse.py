"""Drive pulse envelopes (oracle; test infrastructure only).

Sec. S2.C of the paper, Eq. S(square pulse) and the smoothed stepwise
function that follows it:

* logistic step  f(t, t0, sigma) = 1 / (1 + exp(-(t - t0) / sigma));
* flat-top       Omega(t) = A f(t, t0, sigma) [1 - f(t, t0 + T, sigma)],
  ramp time ~ 5 sigma;
* stepwise       sum_j (h_{j+1} - h_j) f(t, t_j, sigma_j).

Readings used (the paper fixes t0 = 3 ns, sigma = 0.5 ns, i.e. t0 = 6 sigma,
and leaves T implicit):

* flat-top, theta = (A, w_d, t_r, phi): sigma = t_r / 5, t0 = 6 sigma,
  T = tau - 2 t0, so the pulse is symmetric inside [0, tau];
* two-segment, theta = (A1, A2, t_sw, t_rise, t_fall, t_sm, w_d, phi): the
  stepwise form with heights (0, A1, A2, 0) and steps at
  t0r = 6 t_rise/5 (width t_rise/5), t_sw (width t_sm/5) and
  tau - 6 t_fall/5 (width t_fall/5).

The lab-frame coefficient multiplying X_d is c(t) = Omega(t) cos(w_d t + phi).

Parity: pinned by the logistic's closed-form values (f(t0) = 1/2, the
symmetry f(t0 + x) + f(t0 - x) = 1) and the plateau/edge limits in tests.
"""
from __future__ import annotations

import math


def logistic(t: float, t0: float, sigma: float) -> float:
    """f(t, t0, sigma) of Sec. S2.C."""
    return 1.0 / (1.0 + math.exp(-(t - t0) / sigma))


def flat_top_envelope(t: float, A: float, t_r: float, tau: float) -> float:
    sigma = t_r / 5.0
    t0 = 6.0 * sigma
    T = tau - 2.0 * t0
    return A * logistic(t, t0, sigma) * (1.0 - logistic(t, t0 + T, sigma))


def two_segment_envelope(t: float, A1: float, A2: float, t_sw: float,
                         t_rise: float, t_fall: float, t_sm: float,
                         tau: float) -> float:
    s_r, s_f, s_m = t_rise / 5.0, t_fall / 5.0, t_sm / 5.0
    t0r, t0f = 6.0 * s_r, tau - 6.0 * s_f
    heights = (0.0, A1, A2, 0.0)
    steps = ((t0r, s_r), (t_sw, s_m), (t0f, s_f))
    out = 0.0
    for j, (tj, sj) in enumerate(steps):
        out += (heights[j + 1] - heights[j]) * logistic(t, tj, sj)
    return out


def envelope(kind: int, p, t: float, tau: float) -> float:
    if kind == 0:
        A, _wd, t_r, _phi = p
        return flat_top_envelope(t, A, t_r, tau)
    if kind == 1:
        A1, A2, t_sw, t_rise, t_fall, t_sm, _wd, _phi = p
        return two_segment_envelope(t, A1, A2, t_sw, t_rise, t_fall, t_sm, tau)
    raise ValueError("unknown pulse kind")


def drive_frequency_phase(kind: int, p):
    if kind == 0:
        return p[1], p[3]
    return p[6], p[7]


def coefficient(kind: int, p, tau: float):
    """Return c(t) = Omega(t) cos(w_d t + phi) as a callable."""
    wd, phi = drive_frequency_phase(kind, p)
    p = tuple(float(x) for x in p)

    def c(t: float) -> float:
        return envelope(kind, p, t, tau) * math.cos(wd * t + phi)

    return c


def rwa_coefficient(kind: int, p, tau: float):
    """Return Omega(t)/2 as a callable: in the frame rotating at w_d, with the
    rotating-wave approximation, the drive Omega(t) cos(w_d t + phi)(r + r^dag)
    becomes (Omega(t)/2)(e^{i phi} r + e^{-i phi} r^dag), whose operator part
    is ``Model(..., rwa=(w_d, phi)).Xd``."""
    p = tuple(float(x) for x in p)

    def c(t: float) -> float:
        return 0.5 * envelope(kind, p, t, tau)

    return c
