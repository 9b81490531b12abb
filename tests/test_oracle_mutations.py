"""The oracle's pins catch plausible mistakes.

Each case copies the oracle's C sources to a temporary directory, plants one mistake (a dropped
term, a flipped sign, a wrong index or operand), compiles the copy with gcc and runs a quick set of
pins against it: the analytical Jacobian against the complex-step derivative of the source terms,
mass / element / enthalpy conservation, thermodynamics against quadrature of c_p, and closed-form
rates. Every mutant must fail at least one pin; the unmodified copy must pass them all.
"""
import math
import os
import shutil

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1605_03262_b300 import synth
from paper_1605_03262_b300.synth import P_ATM, R_GAS
from tests import mechs

SRC = os.path.dirname(oracle.__file__)
FILES = ("pyjac_oracle.c", "source_terms.inc", "oracle_model.h")

# (file, text to replace, replacement)
MUTANTS = [
    ("pyjac_oracle.c", "dB[k] = (a[0] - 1.0 + a[5] / T) / T", "dB[k] = (a[0] - 1.0 - a[5] / T) / T"),
    ("pyjac_oracle.c", "(dAdPr * Bt - At * dBdPr)", "(dAdPr * Bt + At * dBdPr)"),
    ("pyjac_oracle.c", "dcdY = -Wm * c * Dl[j] + t2;", "dcdY = -Wm * c * Dl[j] - t2;"),
    ("pyjac_oracle.c", "(r->k0[2] - r->kinf[2]) / T - 1.0)", "(r->k0[2] - r->kinf[2]) / T + 1.0)"),
    ("source_terms.inc", "f[0] = -(hs + hsc) / (rho * cp);", "f[0] = (hs + hsc) / (rho * cp);"),
    ("source_terms.inc", "a[2] / 6.0", "a[2] / 3.0"),
    ("source_terms.inc", "(log(P) - log(a[0])) / (log(b[0]) - log(a[0]))",
     "(log(P) - log(b[0])) / (log(b[0]) - log(a[0]))"),
    ("source_terms.inc", "FN(chebT)(i, Tt) * FN(chebT)(j, pt)", "FN(chebT)(j, Tt) * FN(chebT)(i, pt)"),
    ("pyjac_oracle.c", "-(cpk[j] - cpk[L]) / (rho * cp) * HWO", "-(cpk[j] - cpk[0]) / (rho * cp) * HWO"),
    ("pyjac_oracle.c", "dkr = (dkf * Kc - dKc * kf) / (Kc * Kc);", "dkr = (dkf * Kc + dKc * kf) / (Kc * Kc);"),
    ("pyjac_oracle.c", "acc_d(&row[1 + j], &cmp[1 + j], om[k] * Wm * Dl[j]);",
     "acc_d(&row[1 + j], &cmp[1 + j], -om[k] * Wm * Dl[j]);"),
    ("pyjac_oracle.c", "double dl = (k == j ? 1.0 : 0.0) - (k == L ? 1.0 : 0.0);",
     "double dl = (k == j ? 1.0 : 0.0);"),
    ("pyjac_oracle.c", "*dFdT_Pr = Fv * (e / T + X", "*dFdT_Pr = Fv * (e * T + X"),
    ("pyjac_oracle.c", "else                        dcdY = c * (-1.0 / (1.0 + Pr) * dPrdY + dFdY / Fv);",
     "else                        dcdY = c * (1.0 / (1.0 + Pr) * dPrdY + dFdY / Fv);"),
    ("source_terms.inc", "f[1 + k] = m->W[k] * w / rho;\n        FN(acc)(&hs", "f[1 + k] = w / rho;\n        FN(acc)(&hs"),
    ("source_terms.inc", "pow(PJO_PATM / PJO_R, (double)dn)", "pow(PJO_R / PJO_PATM, (double)dn)"),
    ("source_terms.inc", "for (int s = 0; s < r->np; ++s) Prr *= FN(ipow)(C[r->psp[s]], r->pnu[s]);",
     "for (int s = 0; s < r->np; ++s) Prr *= C[r->psp[s]];"),
    ("pyjac_oracle.c", "cs_add(&s, hk[k] * J[(size_t)(1 + k) * ld + 0]);", "cs_add(&s, hk[k] * J[(size_t)(1 + k) * ld + 1]);"),
    ("source_terms.inc", "c = fPr * F; kf = ki;", "c = fPr * F; kf = k0;"),
    ("pyjac_oracle.c", "return kf / T * (r->kinf[1] + r->kinf[2] / T);", "return kf / T * (r->k0[1] + r->k0[2] / T);"),
    ("source_terms.inc", "cv_k[k] = (cpR - 1.0) * PJO_R / m->W[k];", "cv_k[k] = cpR * PJO_R / m->W[k];"),
    ("source_terms.inc", "u_k[k] = (HRT - 1.0) * PJO_R * T / m->W[k];", "u_k[k] = HRT * PJO_R * T / m->W[k];"),
    ("source_terms.inc", "SCALAR P = rho * (sYW + sYWc) * PJO_R * T;", "SCALAR P = rho * PJO_R * T;"),
    ("pyjac_oracle.c", "cimag(fz[row]) / h - (col == 0 ? 0.0 : dfN[row]);", "cimag(fz[row]) / h;"),
    ("source_terms.inc", "f[1] = V * (f[0] / T + PJO_R * T / P * (O + Oc));", "f[1] = V * (PJO_R * T / P * (O + Oc));"),
    ("source_terms.inc", "X[N - 1] = M - (s + sc);", "X[N - 1] = M + (s + sc);"),
    ("source_terms.inc", "H[k] = HRT * PJO_R * T;", "H[k] = HRT * PJO_R;"),
    ("source_terms.inc", "FN(acc)(&K, &Kc, X[k] * cpR * PJO_R);", "FN(acc)(&K, &Kc, cpR * PJO_R);"),
    ("source_terms.inc", "if (k < N - 1) f[2 + k] = V * wk_;", "if (k < N - 1) f[2 + k] = wk_;"),
    ("pyjac_oracle.c", "else { nz[col - 2] += I * h * Vs; dh = h * Vs; }", "else { nz[col - 2] += I * h * Vs; dh = h; }"),
    ("pyjac_oracle.c", "else if (col == 1) { Vz += I * h * Vs; dh = h * Vs; }", "else if (col == 1) { Vz += I * h; dh = h * Vs; }"),
    # the Troe and SRI blending values (pinned in the mid-range of log10 P_r)
    ("source_terms.inc", "SCALAR Bt = 0.806 - 1.1762 * lFc - 0.14 * lPr;", "SCALAR Bt = 0.8 - 1.1762 * lFc - 0.14 * lPr;"),
    ("source_terms.inc", "SCALAR Bt = 0.806 - 1.1762 * lFc - 0.14 * lPr;", "SCALAR Bt = 0.806 - 1.176 * lFc - 0.14 * lPr;"),
    ("source_terms.inc", "return pow(Fc, 1.0 / (1.0 + (At / Bt) * (At / Bt)));", "return pow(Fc, 1.0 / (1.0 + (At / Bt)));"),
    ("source_terms.inc", "SCALAR X = 1.0 / (1.0 + lPr * lPr);", "SCALAR X = 1.0 / (1.0 + lPr);"),
]

EPS = 2.0 ** -52


def _H_quad(a, T):
    v, _ = integrate.quad(lambda t: np.polynomial.polynomial.polyval(t, a[:5]), 0.0, T, epsabs=0.0, epsrel=1e-13)
    return a[5] + v


def _pins(lib) -> list:
    """Quick pins; returns the names of those that failed."""
    failed = []
    # 1. analytical Jacobian vs complex step, every reaction type (explicit and K_c reverse, chem.-act.)
    for seed in (3, 4):
        model = mechs.mixed_model(seed=seed, n_species=9, n_reactions=30)
        om = oracle.load_model(synth.to_bytes(model), lib=lib)
        T, P, Y = synth.generate_states(model.n_species, 6, seed=seed + 10)
        J, f, Js, fs = om.jacobian(T, P, Y, with_scale=True)
        Jc = om.jacobian_complex_step(T, P, Y)
        bad = ~(np.abs(J - Jc) <= 1e-10 * np.maximum(np.abs(Jc), 1e-20) + 64 * EPS * Js)
        if bad.any() or not np.all(np.isfinite(J)):
            failed.append("complex-step")
            break
    # 2. conservation: mass, elements, enthalpy
    model = synth.config_model(0)
    om = oracle.load_model(synth.to_bytes(model), lib=lib)
    T, P, Y = synth.config_states(0, 6)
    J, f, Js, fs = om.jacobian(T, P, Y, with_scale=True)
    W = np.array([s.W for s in model.species])
    E = np.array([s.elem for s in model.species], dtype=np.float64)
    if not np.all(np.abs(f[:, 1:].sum(1)) <= 1e-13 * fs[:, 1:].sum(1)):
        failed.append("mass")
    if not np.all(np.abs((f[:, 1:] / W) @ E) <= 1e-13 * ((fs[:, 1:] / W) @ E)):
        failed.append("elements")
    for s in range(2):
        a = [(sp.a_low if T[s] < sp.T_mid else sp.a_high) for sp in model.species]
        h = np.array([R_GAS / sp.W * _H_quad(a[i], T[s]) for i, sp in enumerate(model.species)])
        cpk = np.array([R_GAS / sp.W * np.polynomial.polynomial.polyval(T[s], a[i][:5])
                        for i, sp in enumerate(model.species)])
        if abs(np.sum(h * f[s, 1:]) + (Y[s] @ cpk) * f[s, 0]) > 1e-11 * np.abs(h * f[s, 1:]).sum():
            failed.append("enthalpy")
            break
    # 3. thermodynamics: B_k against quadrature-based S/R - H/(RT) - ln T
    th = om.species_thermo(1500.0)
    for k, sp in enumerate(model.species):
        a = sp.a_high
        S, _ = integrate.quad(lambda t: np.polynomial.polynomial.polyval(t, a[1:5]), 0.0, 1500.0, epsabs=0.0,
                              epsrel=1e-13)
        B = a[0] * math.log(1500.0) + a[6] + S - _H_quad(a, 1500.0) / 1500.0 - math.log(1500.0)
        if abs(th["B"][k] - B) > 1e-9 * max(1.0, abs(B)):
            failed.append("thermo")
            break
    # 4. rates at a PLOG interior pressure and a Chebyshev point against numpy
    grid = [(1.0 * P_ATM, 1.0e5, 0.5, 1000.0), (3.0 * P_ATM, 3.0e5, 0.2, 1500.0), (20.0 * P_ATM, 2.0e6, -0.4, 800.0)]
    r = synth.Reaction(kind=synth.KIND_PLOG, rev_mode=synth.REV_IRREVERSIBLE, reac=[(0, 1), (1, 1)], prod=[(2, 1)],
                       plog=grid)
    TWO = [(1, 0, 0), (0, 1, 0), (1, 1, 0)]
    om1 = oracle.load_model(synth.to_bytes(mechs.one_reaction_model(r, TWO)), lib=lib)
    Tq = 1300.0
    lk = [math.log(A * Tq ** b * math.exp(-Ta / Tq)) for _, A, b, Ta in grid]
    kf = om1.reaction_rates(Tq, 7.0 * P_ATM, np.array([0.3, 0.3, 0.4]))["kf"][0]
    if abs(kf - math.exp(np.interp(math.log(7.0 * P_ATM), [math.log(g[0]) for g in grid], lk))) > 1e-12 * kf:
        failed.append("plog")
    eta = np.arange(21, dtype=float).reshape(7, 3) * 0.05
    eta[0, 0] = 8.0
    rngs = (300.0, 3000.0, 0.1 * P_ATM, 100.0 * P_ATM)
    r = synth.Reaction(kind=synth.KIND_CHEB, rev_mode=synth.REV_IRREVERSIBLE, reac=[(0, 1), (1, 1)], prod=[(2, 1)],
                       cheb_shape=(7, 3), cheb_range=rngs, cheb_eta=eta)
    om2 = oracle.load_model(synth.to_bytes(mechs.one_reaction_model(r, TWO)), lib=lib)
    Pq = 5.0 * P_ATM
    Tt = (2 / Tq - 1 / rngs[0] - 1 / rngs[1]) / (1 / rngs[1] - 1 / rngs[0])
    pt = (2 * math.log10(Pq) - math.log10(rngs[2]) - math.log10(rngs[3])) / (math.log10(rngs[3]) - math.log10(rngs[2]))
    kf = om2.reaction_rates(Tq, Pq, np.array([0.3, 0.3, 0.4]))["kf"][0]
    if abs(math.log10(kf) - np.polynomial.chebyshev.chebval2d(Tt, pt, eta)) > 1e-12:
        failed.append("chebyshev")
    # 5. constant volume at the density of the same states: equal species rates, the energy
    #    identity c_v f0 + sum_k u_k f_k = 0, and two Jacobian columns against central differences
    #    (the rates on a model with every reaction type, so that pressure-dependent ones see p)
    mixed = mechs.mixed_model(seed=3, n_species=9, n_reactions=30)
    omm = oracle.load_model(synth.to_bytes(mixed), lib=lib)
    Tm, Pm, Ym = synth.generate_states(mixed.n_species, 6, seed=13)
    rm = Pm / (R_GAS * Tm * (Ym / np.array([s.W for s in mixed.species])).sum(axis=1))
    fcp, fcvm = omm.dydt(Tm, Pm, Ym), omm.dydt_cv(Tm, rm, Ym)
    if not np.all(np.abs(fcvm[:, 1:] - fcp[:, 1:]) <= 1e-13 * np.abs(fcp[:, 1:]).max(axis=1, keepdims=True)):
        failed.append("cv rates")
    Wk = np.array([s.W for s in model.species])
    rho = P / (R_GAS * T * (Y / Wk).sum(axis=1))
    fcv = om.dydt_cv(T, rho, Y)
    for s in range(2):
        a = [(sp.a_low if T[s] < sp.T_mid else sp.a_high) for sp in model.species]
        u = np.array([R_GAS / sp.W * (_H_quad(a[i], T[s]) - T[s]) for i, sp in enumerate(model.species)])
        cvk = np.array([R_GAS / sp.W * (np.polynomial.polynomial.polyval(T[s], a[i][:5]) - 1.0)
                        for i, sp in enumerate(model.species)])
        if abs(np.sum(u * fcv[s, 1:]) + (Y[s] @ cvk) * fcv[s, 0]) > 1e-11 * np.abs(u * fcv[s, 1:]).sum():
            failed.append("cv energy")
            break
    Jcv = om.jacobian_cv(T[:1], rho[:1], Y[:1])[0]
    N = model.n_species
    for col in (0, 1):
        h = 1e-3 * (T[0] if col == 0 else min(Y[0, 0], Y[0, N - 1]))
        fd = []
        for st in (-2, -1, 1, 2):
            Tp, Yp = T[:1].copy(), Y[:1].copy()
            if col == 0:
                Tp += st * h
            else:
                Yp[0, 0] += st * h
                Yp[0, N - 1] -= st * h
            fd.append(om.dydt_cv(Tp, rho[:1], Yp)[0])
        d = (fd[0] - 8 * fd[1] + 8 * fd[2] - fd[3]) / (12 * h)
        big = np.abs(Jcv[:, col]) > 1e-3 * np.abs(Jcv[:, col]).max()
        if not np.all(np.abs(d - Jcv[:, col])[big] <= 1e-5 * np.abs(Jcv[big, col])):
            failed.append("cv jacobian")
            break
    # 6. molar-concentration basis: one elementary reaction A + B -> C with D inert, in closed form
    #    (source terms, n_A and V columns); element conservation with the last species' rate implied
    #    by the ideal-gas law; the T and first n column against central differences
    A, beta, Ta = 3.0e5, 0.7, 4000.0
    r = synth.Reaction(kind=synth.KIND_ELEMENTARY, rev_mode=synth.REV_IRREVERSIBLE, reac=[(0, 1), (1, 1)],
                       prod=[(2, 1)], arr=(A, beta, Ta))
    om3 = oracle.load_model(synth.to_bytes(mechs.one_reaction_model(r, [(1, 0), (0, 1), (1, 1), (2, 0)])), lib=lib)
    Tc, Pc, Vc = np.array([1234.0]), np.array([3.0 * P_ATM]), np.array([2.5e-3])
    nc = np.array([[0.2, 0.3, 0.1]]) * Pc[0] * Vc[0] / (R_GAS * Tc[0])
    Jc, fc = om3.jacobian_conc(Tc, Pc, Vc, nc)
    k = A * Tc[0] ** beta * math.exp(-Ta / Tc[0])
    CA, CB = nc[0, 0] / Vc[0], nc[0, 1] / Vc[0]
    ok = (abs(fc[0, 2] + Vc[0] * k * CA * CB) <= 1e-12 * Vc[0] * k * CA * CB
          and abs(Jc[0, 2, 2] + k * CB) <= 1e-12 * k * CB and abs(Jc[0, 2, 1] - k * CA * CB) <= 1e-12 * k * CA * CB)
    if not ok:
        failed.append("conc closed form")
    Nm = mixed.n_species
    Tn, Pn, Vn, nn = synth.generate_conc_states(Nm, 3, seed=33, alpha=3.0)
    Jn, fn = omm.jacobian_conc(Tn, Pn, Vn, nn)
    Wm = np.array([sp.W for sp in mixed.species])
    Em = np.array([sp.elem for sp in mixed.species], dtype=np.float64)
    for s in range(3):
        dnN = Pn[s] * fn[s, 1] / (R_GAS * Tn[s]) - Pn[s] * Vn[s] * fn[s, 0] / (R_GAS * Tn[s] ** 2) - fn[s, 2:].sum()
        rates = np.concatenate([fn[s, 2:], [dnN]])
        if not np.all(np.abs(rates @ Em) <= 1e-12 * (np.abs(rates) @ Em + 1e-300)):
            failed.append("conc elements")
            break
        a = [(sp.a_low if Tn[s] < sp.T_mid else sp.a_high) for sp in mixed.species]
        H = np.array([R_GAS * _H_quad(a[i], Tn[s]) for i in range(Nm)])
        cpm = np.array([R_GAS * np.polynomial.polynomial.polyval(Tn[s], a[i][:5]) for i in range(Nm)])
        n_all = np.concatenate([nn[s], [Pn[s] * Vn[s] / (R_GAS * Tn[s]) - nn[s].sum()]])
        if abs(rates @ H + (n_all @ cpm) * fn[s, 0]) > 1e-11 * np.abs(rates * H).sum():
            failed.append("conc enthalpy")
            break
    x = np.concatenate([[Tn[0], Vn[0]], nn[0]])
    nN = Pn[0] * Vn[0] / (R_GAS * Tn[0]) - nn[0].sum()
    for col in (0, 1, 2):
        h = 1e-5 * (abs(x[col]) if col < 2 else min(abs(x[col]), nN))
        d = []
        for st in (-2, -1, 1, 2):
            xp = x.copy()
            xp[col] += st * h
            d.append(omm.dydt_conc(xp[:1], Pn[:1], xp[1:2], xp[2:][None])[0])
        fd = (d[0] - 8 * d[1] + 8 * d[2] - d[3]) / (12 * h)
        big = np.abs(Jn[0, :, col]) > 1e-3 * np.abs(Jn[0, :, col]).max()
        if not np.all(np.abs(fd - Jn[0, :, col])[big] <= 1e-6 * np.abs(Jn[0, big, col])):
            failed.append("conc jacobian")
            break
    # 7. Troe (with and without T**) and SRI blending values at mid-range log10 P_r, by hand
    from tests.test_oracle_pins import _pressure_for_Pr, _sri_F_by_hand, _troe_F_by_hand
    Tf, Yf = 1400.0, np.array([0.2, 0.2, 0.2, 0.2, 0.2])
    k0, kinf = (1.0e3, 0.0, 0.0), (1.0e4, 0.5, 100.0)
    FIVE = [(1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1)]
    cases = [(synth.F_TROE, (0.35, 180.0, 2500.0, 0.0, 0.0), 0, lambda Pr: _troe_F_by_hand(Tf, Pr, 0.35, 180.0, 2500.0)),
             (synth.F_TROE, (0.35, 180.0, 2500.0, 4200.0, 0.0), 1,
              lambda Pr: _troe_F_by_hand(Tf, Pr, 0.35, 180.0, 2500.0, 4200.0)),
             (synth.F_SRI, (0.7, 450.0, 1300.0, 1.2, 0.15), 0, lambda Pr: _sri_F_by_hand(Tf, Pr, 0.7, 450.0, 1300.0, 1.2, 0.15))]
    for ftype, fp, has, Fh in cases:
        r = synth.Reaction(kind=synth.KIND_FALLOFF, rev_mode=synth.REV_IRREVERSIBLE, reac=[(2, 1)],
                           prod=[(0, 1), (1, 1)], tb_mode=synth.TB_MIXTURE, k0=k0, kinf=kinf, ftype=ftype,
                           fparams=fp, troe_has_T2=has)
        omf = oracle.load_model(synth.to_bytes(mechs.one_reaction_model(r, FIVE)), lib=lib)
        bad = False
        for lpr in (-2.0, 0.5, 3.0):
            Pr = 10.0 ** lpr
            c = omf.reaction_rates(Tf, _pressure_for_Pr(Tf, Pr, k0, kinf), Yf)["c"][0]
            bad |= not abs(c - Pr / (1 + Pr) * Fh(Pr)) <= 1e-12 * abs(c)
        if bad:
            failed.append("falloff blending")
            break
    return failed


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


def _variant(workdir, tag, mutation=None):
    d = os.path.join(str(workdir), tag)
    os.makedirs(d, exist_ok=True)
    for fn in FILES:
        shutil.copy(os.path.join(SRC, fn), os.path.join(d, fn))
    if mutation is not None:
        fn, old, new = mutation
        p = os.path.join(d, fn)
        text = open(p).read()
        assert text.count(old) == 1, ("mutation anchor not found exactly once", fn, old)
        open(p, "w").write(text.replace(old, new))
    so = oracle.compile_variant(d, os.path.join(d, "liboracle_%s.so" % tag))
    return oracle.load_variant(so)


def test_unmodified_copy_passes_the_quick_pins(workdir):
    assert _pins(_variant(workdir, "clean")) == []


@pytest.mark.parametrize("idx", range(len(MUTANTS)))
def test_planted_mistake_is_caught(workdir, idx):
    failed = _pins(_variant(workdir, "m%02d" % idx, MUTANTS[idx]))
    assert failed, "mutation %d survived every pin: %r" % (idx, MUTANTS[idx])
