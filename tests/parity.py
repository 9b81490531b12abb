"""Comparison of CUDA-path outputs with the oracle.

Bar: |x_gpu - x_oracle| <= 1e-10 * max(|x_oracle|, 1e-20) + 64 * eps * scale, where scale is the
oracle's sum of the absolute values of the terms it added to form that entry. For an entry whose
condition number kappa = scale / |x| is below ~4500 the second term is below 1e-10 |x|, so the bar
is the plain 1e-10 relative error; above that the entry is a cancelled sum and both sides carry
rounding error of order eps * scale. The report also gives the paper's E_rel (Eq. e:error_norm,
over entries with |J| >= ||J||_F / 1e20) for the first state set.
"""
import numpy as np

EPS = 2.0 ** -52
REL = 1e-10
FLOOR = 1e-20
KAPPA_MULT = 64.0


def compare(gpu, ora, scale, rel=REL, floor=FLOOR, kappa_mult=KAPPA_MULT):
    gpu = np.asarray(gpu, dtype=np.float64)
    ora = np.asarray(ora, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    finite = np.isfinite(gpu) & np.isfinite(ora)
    err = np.abs(gpu - ora)
    bound = rel * np.maximum(np.abs(ora), floor) + kappa_mult * EPS * scale
    ok = finite & (err <= bound)
    strict = finite & (err <= rel * np.maximum(np.abs(ora), floor))
    rel_err = np.where(np.abs(ora) > floor, err / np.maximum(np.abs(ora), floor), 0.0)
    with np.errstate(over="ignore"):   # a huge scale over a tiny entry is an infinitely ill-conditioned entry
        kappa = np.where(np.abs(ora) > 0, scale / np.maximum(np.abs(ora), 1e-300), 0.0)
    well = (kappa <= 4500.0) & (np.abs(ora) >= floor)
    return {
        "n": int(ora.size),
        "n_bad": int((~ok).sum()),
        "n_nonfinite": int((~finite).sum()),
        "n_strict_fail": int((~strict).sum()),
        "max_rel_well_conditioned": float(rel_err[well].max()) if well.any() else 0.0,
        "max_kappa_of_strict_fail": float(kappa[~strict & finite].max()) if (~strict & finite).any() else 0.0,
    }


def e_rel(gpu_J, ora_J):
    """Paper's E_rel per state: Frobenius norm of elementwise relative errors over entries with
    |J| >= ||J||_F / 1e20 (Eq. e:error_norm); returns the per-state values."""
    out = []
    for g, o in zip(gpu_J, ora_J):
        thr = np.linalg.norm(o) / 1e20
        m = np.abs(o) >= thr
        m &= o != 0
        out.append(float(np.linalg.norm((g[m] - o[m]) / o[m])))
    return np.array(out)


def assert_parity(gpu, ora, scale, what=""):
    rep = compare(gpu, ora, scale)
    assert rep["n_nonfinite"] == 0, (what, rep)
    assert rep["n_bad"] == 0, (what, rep)
    assert rep["max_rel_well_conditioned"] <= REL, (what, rep)
    return rep
