"""Shared comparison helpers for the GPU parity tests."""
import numpy as np


def rel_inf(got, want):
    got, want = np.asarray(got), np.asarray(want)
    scale = max(np.abs(want).max(), 1e-300)
    return float(np.abs(got - want).max() / scale)


def compare_observables(gpu, ora, n_traj, nt_list, tol_rel, tol_pop, what=""):
    """Element-by-element comparison of beta, pops, photons, trace and eps_a."""
    report = {}
    for j in range(n_traj):
        b_g, b_o = gpu["beta"][j][: ora["beta"][j].shape[0]], ora["beta"][j]
        report.setdefault("beta", []).append(rel_inf(b_g, b_o))
        nt = nt_list[j]
        pg = gpu["pops"][j][:, :nt]
        report.setdefault("pops", []).append(float(np.abs(pg - ora["pops"][j]).max()))
        report.setdefault("nphot", []).append(rel_inf(gpu["nphot"][j], ora["nphot"][j]))
        report.setdefault("trace", []).append(float(np.abs(gpu["trace"][j] - ora["trace"][j]).max()))
        if gpu["pops"][j].shape[1] > nt:
            assert np.all(gpu["pops"][j][:, nt:] == 0.0)
    report["eps_a"] = [abs(a - b) / abs(b) for a, b in zip(gpu["eps_a"], ora["eps_a"])]
    worst = {k: max(v) for k, v in report.items()}
    msg = "%s worst errors: %s" % (what, worst)
    assert worst["beta"] <= tol_rel, msg
    assert worst["nphot"] <= tol_rel, msg
    assert worst["eps_a"] <= tol_rel, msg
    assert worst["pops"] <= tol_pop, msg
    assert worst["trace"] <= tol_pop, msg
    return worst
