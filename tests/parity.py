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


def rate_exponent_condition(model, T):
    """Largest sum of the absolute values of the terms of a rate exponent over the model's
    reactions at the temperatures T: ln k = ln A + beta ln T - Ta/T (every Arrhenius set of a
    reaction: k, k_0, k_inf, PLOG points, explicit reverse), ln(10) sum |eta| for Chebyshev, and
    for K_c reverse rates also |dnu ln(p_atm/R)| + sum_k |nu_k| (the absolute terms of B_k). Two
    correct evaluations of a rate differ by up to about this many ulps (relative), which the
    1e-10 relative bar absorbs except in entries that are themselves cancelled sums."""
    import math
    from paper_1605_03262_b300.synth import P_ATM, R_GAS
    worst = 0.0
    for t in np.atleast_1d(np.asarray(T, dtype=np.float64)):
        lt = math.log(t)
        bterm = []
        for sp in model.species:
            a = sp.a_low if t < sp.T_mid else sp.a_high
            bterm.append(abs((a[0] - 1.0) * lt) + abs(a[6] - a[0]) + abs(a[1] * t / 2) + abs(a[2] * t * t / 6)
                         + abs(a[3] * t ** 3 / 12) + abs(a[4] * t ** 4 / 20) + abs(a[5] / t))

        def arr(p):
            A, b, Ta = p
            return (abs(math.log(A)) if A > 0 else 0.0) + abs(b * lt) + abs(Ta / t)

        for r in model.reactions:
            sets = [r.arr, r.k0, r.kinf] + [g[1:] for g in r.plog]
            c = max(arr(p) for p in sets)
            if r.cheb_eta is not None:
                c = max(c, math.log(10.0) * float(np.abs(r.cheb_eta).sum()))
            if r.rev_mode == 1:
                dnu = sum(v for _, v in r.prod) - sum(v for _, v in r.reac)
                c += abs(dnu * math.log(P_ATM / R_GAS)) + sum(v * bterm[k] for k, v in r.reac + r.prod)
            elif r.rev_mode == 2 and r.rev_arr is not None:
                c = max(c, arr(r.rev_arr))
            worst = max(worst, c)
    return worst
