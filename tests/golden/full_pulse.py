"""Reader of the full-pulse expected values written by make_full_pulse.py.

``load(kind)`` returns, for kind "c4" or "paper", a dict with the step
size, the decimation factors and, per candidate, eps_a, T and per level
(0 = |g>, 1 = |e>) the decimated beta and the records (pops, nphot, trace).
Plain parsing only: the values come from the FP64 oracle via the script.
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def path(kind: str) -> str:
    return os.path.join(HERE, "full_pulse_%s.txt" % kind)


def available(kind: str) -> bool:
    return os.path.exists(path(kind))


def load(kind: str) -> dict:
    out = {"cands": {}}
    header = []
    sec = None
    rows = []

    def flush():
        if sec is None:
            return
        parts = sec.split()
        if parts[0] == "candidate":
            c = int(parts[1])
            d = out["cands"].setdefault(c, {})
            for r in rows:
                if r[0] in ("eps_a", "T"):
                    d[r[0]] = float(r[1])
        else:
            c, lv = int(parts[1]), int(parts[2])
            d = out["cands"].setdefault(c, {}).setdefault(lv, {})
            a = np.array([[float(x) for x in r] for r in rows])
            if parts[0] == "beta":
                d["beta"] = a[:, 0] + 1j * a[:, 1]
            else:
                d["pops"] = a[:, :-2]
                d["nphot"] = a[:, -2]
                d["trace"] = a[:, -1]

    with open(path(kind)) as fh:
        for line in fh:
            line = line.strip()
            if not line:
                continue
            if line.startswith("#"):
                header.append(line[1:].strip())
            elif line.startswith("["):
                flush()
                sec, rows = line[1:-1], []
            else:
                rows.append(line.split())
    flush()
    for h in header:
        if h.startswith("dt "):
            w = h.replace(",", "").split()
            out["dt"] = float(w[1])
            out["n_steps"] = int(w[3])
        if h.startswith("beta every"):
            w = h.replace(":", "").split()
            out["beta_every"] = int(w[2])
            out["rec_every"] = int(w[[i for i, x in enumerate(w) if x == "records"][0] + 2])
    return out


def errors(golden: dict, got: dict, cands, eps_a=None, ion=None) -> dict:
    """Worst errors of a GPU run against the full-pulse values, over the
    candidates `cands` (trajectories 2k, 2k+1 of the run hold candidate
    cands[k] from |g> and |e>): beta relative to its largest magnitude (at the
    decimated steps), populations and tr rho absolute, photons relative to
    their largest value, eps_a and T relative. got["beta"] is [traj][step]
    (complex) over the whole pulse; pops/nphot/trace are [traj][rec][...] on a
    record grid that contains the golden one."""
    be, re_ = golden["beta_every"], golden["rec_every"]
    out = {"beta_rel": 0.0, "pops_abs": 0.0, "nphot_rel": 0.0, "trace_abs": 0.0, "eps_a_rel": 0.0, "T_rel": 0.0}
    pe = got.get("pop_every", re_)
    for k, c in enumerate(cands):
        g = golden["cands"][c]
        for lv in (0, 1):
            j = 2 * k + lv
            w = g[lv]
            b = np.asarray(got["beta"][j])[: golden["n_steps"] + 1][::be]
            out["beta_rel"] = max(out["beta_rel"], float(np.abs(b - w["beta"]).max() / np.abs(w["beta"]).max()))
            idx = np.arange(w["pops"].shape[0]) * (re_ // pe)
            p = np.asarray(got["pops"][j])[idx][:, : w["pops"].shape[1]]
            out["pops_abs"] = max(out["pops_abs"], float(np.abs(p - w["pops"]).max()))
            n = np.asarray(got["nphot"][j])[idx]
            out["nphot_rel"] = max(out["nphot_rel"], float(np.abs(n - w["nphot"]).max() / np.abs(w["nphot"]).max()))
            t = np.asarray(got["trace"][j])[idx]
            out["trace_abs"] = max(out["trace_abs"], float(np.abs(t - w["trace"]).max()))
        if eps_a is not None:
            out["eps_a_rel"] = max(out["eps_a_rel"], abs(eps_a[k] - g["eps_a"]) / abs(g["eps_a"]))
        if ion is not None:
            out["T_rel"] = max(out["T_rel"], abs(ion[k] - g["T"]) / abs(g["T"]))
    return out
