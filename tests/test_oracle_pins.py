"""Pins of the CPU oracle to things other than itself (no GPU).

Each test fixes one part of the oracle against the mathematics the paper states:
thermodynamic identities checked by quadrature, closed forms of special cases, library routines
(numpy Chebyshev / interpolation), conservation invariants, equilibrium, complex-step and finite
difference derivatives of the source terms, and a hand-derived Jacobian of a one-reaction model.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1605_03262_b300 import synth
from paper_1605_03262_b300.synth import (KIND_CHEB, KIND_ELEMENTARY, KIND_FALLOFF, KIND_PLOG,
                                         KIND_THIRD_BODY, F_LINDEMANN, F_SRI, F_TROE, P_ATM, R_GAS,
                                         REV_IRREVERSIBLE, REV_KC, TB_MIXTURE, Reaction)
from tests import mechs

EPS = 2.0 ** -52


def _om(model):
    return oracle.load_model(synth.to_bytes(model))


def _coeffs(sp, T):
    return sp.a_low if T < sp.T_mid else sp.a_high


# ---------------------------------------------------------------------------------------------
# thermodynamics (Eqs. e:cpk, e:hk, e:sk; B_k of Section 2.3.1)

def _H_over_R_by_quadrature(a, T):
    """H/R = a5 + integral_0^T cp/R dT' (the enthalpy constant a5 is H/R at T = 0)."""
    val, _ = integrate.quad(lambda t: np.polynomial.polynomial.polyval(t, a[:5]), 0.0, T,
                            epsabs=0.0, epsrel=1e-13, limit=200)
    return a[5] + val


def _S_over_R_by_quadrature(a, T):
    """S/R = a0 ln T + a6 + integral_0^T (cp/R - a0)/T' dT'."""
    val, _ = integrate.quad(lambda t: np.polynomial.polynomial.polyval(t, a[1:5]), 0.0, T,
                            epsabs=0.0, epsrel=1e-13, limit=200)
    return a[0] * math.log(T) + a[6] + val


@pytest.mark.parametrize("T", [350.0, 812.5, 999.0, 1000.0, 1733.0, 2950.0])
def test_nasa7_thermo_matches_quadrature_of_cp(T):
    model = synth.config_model(0)
    th = _om(model).species_thermo(T)
    for k, sp in enumerate(model.species):
        a = _coeffs(sp, T)
        cpR = np.polynomial.polynomial.polyval(T, a[:5])
        assert th["cpR"][k] == pytest.approx(cpR, rel=1e-14)
        assert th["HRT"][k] * T == pytest.approx(_H_over_R_by_quadrature(a, T), rel=1e-11, abs=1e-9)
        assert th["SR"][k] == pytest.approx(_S_over_R_by_quadrature(a, T), rel=1e-11)
        # B_k = S/R - H/(R T) - ln T (the species term of K_c)
        Bk = _S_over_R_by_quadrature(a, T) - _H_over_R_by_quadrature(a, T) / T - math.log(T)
        assert th["B"][k] == pytest.approx(Bk, rel=1e-10, abs=1e-9)


def test_nasa7_ranges_continuous_at_Tmid():
    model = synth.config_model(1)
    om = _om(model)
    lo, hi = om.species_thermo(1000.0 * (1 - 1e-12)), om.species_thermo(1000.0)
    for key in ("cpR", "HRT", "SR", "B"):
        np.testing.assert_allclose(lo[key], hi[key], rtol=1e-8, atol=1e-8)


# ---------------------------------------------------------------------------------------------
# rate coefficients (Section 2.3)

def _state(n_species, seed=1):
    T, P, Y = synth.generate_states(n_species, 1, seed=seed)
    return float(T[0]), float(P[0]), Y[0]


def _conc(model, T, P, Y):
    """[X_k] = rho Y_k / W_k with rho from the ideal-gas law (Eq. e:state)."""
    W = np.array([s.W for s in model.species])
    Wm = 1.0 / np.sum(Y / W)
    rho = P * Wm / (R_GAS * T)
    return rho * Y / W, rho


TWO = [(1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1)]   # A, B, AB, C, AC


def test_arrhenius_and_its_special_forms():
    for (A, beta, Ta) in [(3.0e4, 0.0, 0.0), (2.5e3, 2.0, 0.0), (7.0e5, -1.3, 0.0), (1.0e6, 0.0, 12000.0),
                          (4.2e2, 1.7, 8000.0)]:
        r = Reaction(kind=KIND_ELEMENTARY, rev_mode=REV_IRREVERSIBLE, reac=[(0, 1), (1, 1)], prod=[(2, 1)],
                     arr=(A, beta, Ta))
        model = mechs.one_reaction_model(r, TWO)
        T, P, Y = _state(5)
        kf = _om(model).reaction_rates(T, P, Y)["kf"][0]
        if beta == 0.0 and Ta == 0.0:
            assert kf == A
        elif Ta == 0.0 and float(beta).is_integer():
            assert kf == pytest.approx(A * T ** int(beta), rel=4 * EPS)
        else:
            assert kf == pytest.approx(A * T ** beta * math.exp(-Ta / T), rel=1e-14)


def test_production_rate_closed_form_bimolecular():
    """A + B -> AB irreversible: q = k [A][B], omega = (-q, -q, +q, 0, 0)."""
    r = Reaction(kind=KIND_ELEMENTARY, rev_mode=REV_IRREVERSIBLE, reac=[(0, 1), (1, 1)], prod=[(2, 1)],
                 arr=(1.0e5, 0.5, 3000.0))
    model = mechs.one_reaction_model(r, TWO)
    T, P, Y = _state(5)
    C, rho = _conc(model, T, P, Y)
    k = 1.0e5 * T ** 0.5 * math.exp(-3000.0 / T)
    q = k * C[0] * C[1]
    rates = _om(model).reaction_rates(T, P, Y)
    assert rates["q"][0] == pytest.approx(q, rel=1e-13)
    f = _om(model).dydt([T], [P], Y[None])[0]
    W = np.array([s.W for s in model.species])
    np.testing.assert_allclose(f[1:], W * np.array([-q, -q, q, 0, 0]) / rho, rtol=1e-13, atol=0)


def test_reverse_rate_from_gibbs_energy_by_quadrature():
    """k_r = k_f / K_c, K_c = (p_atm/(R T))^{sum nu} exp(sum nu (S/R - H/(R T)))."""
    model = mechs.typed_model("elementary", seed=3, rev_modes=(REV_KC,))
    om = _om(model)
    T, P, Y = _state(model.n_species, seed=4)
    rates = om.reaction_rates(T, P, Y)
    g = np.array([_S_over_R_by_quadrature(_coeffs(s, T), T) - _H_over_R_by_quadrature(_coeffs(s, T), T) / T
                  for s in model.species])
    for i, r in enumerate(model.reactions):
        dn = sum(nu for _, nu in r.prod) - sum(nu for _, nu in r.reac)
        sg = sum(nu * g[s] for s, nu in r.prod) - sum(nu * g[s] for s, nu in r.reac)
        Kc = (P_ATM / (R_GAS * T)) ** dn * math.exp(sg)
        assert rates["kr"][i] == pytest.approx(rates["kf"][i] / Kc, rel=1e-9)


def test_third_body_unity_efficiencies_equal_elementary_times_total_concentration():
    base = dict(rev_mode=REV_IRREVERSIBLE, reac=[(0, 1), (1, 1)], prod=[(2, 1)], arr=(2.0e4, 0.3, 900.0))
    m_tb = mechs.one_reaction_model(Reaction(kind=KIND_THIRD_BODY, tb_mode=TB_MIXTURE, **base), TWO)
    m_el = mechs.one_reaction_model(Reaction(kind=KIND_ELEMENTARY, **base), TWO)
    T, P, Y = _state(5)
    q_tb = _om(m_tb).reaction_rates(T, P, Y)["q"][0]
    q_el = _om(m_el).reaction_rates(T, P, Y)["q"][0]
    assert q_tb == pytest.approx(q_el * P / (R_GAS * T), rel=1e-13)


def _falloff(kind, ftype, fparams=(0.0,) * 5, has_T2=0, k0=(1.0e3, 0.0, 0.0), kinf=(1.0e4, 0.5, 100.0)):
    return Reaction(kind=kind, rev_mode=REV_IRREVERSIBLE, reac=[(2, 1)], prod=[(0, 1), (1, 1)],
                    tb_mode=TB_MIXTURE, k0=k0, kinf=kinf, ftype=ftype, fparams=fparams, troe_has_T2=has_T2)


def test_troe_with_unit_fcent_equals_lindemann():
    # a = 0, T*** -> infinity, no T** term: F_cent = exp(0) = 1, so F = 1.
    T, P, Y = _state(5)
    troe = _om(mechs.one_reaction_model(_falloff(KIND_FALLOFF, F_TROE, (0.0, 1e300, 500.0, 0.0, 0.0)), TWO))
    lind = _om(mechs.one_reaction_model(_falloff(KIND_FALLOFF, F_LINDEMANN), TWO))
    assert troe.reaction_rates(T, P, Y)["c"][0] == pytest.approx(lind.reaction_rates(T, P, Y)["c"][0], rel=1e-14)


def test_troe_blending_equals_fcent_where_A_vanishes():
    """When log10 P_r = 0.4 + 0.67 log10 F_cent, A_Troe = 0 and F = F_cent exactly."""
    a, T3, T1 = 0.6, 200.0, 3000.0
    T, _, Y = _state(5)
    Fc = (1 - a) * math.exp(-T / T3) + a * math.exp(-T / T1)
    target_Pr = 10.0 ** (0.4 + 0.67 * math.log10(Fc))
    model = mechs.one_reaction_model(_falloff(KIND_FALLOFF, F_TROE, (a, T3, T1, 0.0, 0.0)), TWO)
    # P_r = (k0/kinf) [M] with [M] = P/(R T); choose P to hit the target with k0 = 1e3, kinf = 1e4 T^0.5 e^{-100/T}
    ratio = 1.0e3 / (1.0e4 * T ** 0.5 * math.exp(-100.0 / T))
    P = target_Pr / ratio * R_GAS * T
    c = _om(model).reaction_rates(T, P, Y)["c"][0]
    assert c == pytest.approx(target_Pr / (1 + target_Pr) * Fc, rel=1e-10)


def _troe_F_by_hand(T, Pr, a, T3, T1, T2=None):
    """Troe blending factor of Section 2.3.3 written out: F_cent from its three (or two) terms,
    A_Troe and B_Troe from log10 P_r and log10 F_cent, and log10 F = log10 F_cent / (1 + (A/B)^2)."""
    Fc = (1.0 - a) * math.exp(-T / T3) + a * math.exp(-T / T1)
    if T2 is not None:
        Fc += math.exp(-T2 / T)
    lpr, lfc = math.log10(Pr), math.log10(Fc)
    A = lpr - 0.67 * lfc - 0.4
    B = 0.806 - 1.1762 * lfc - 0.14 * lpr
    return 10.0 ** (lfc / (1.0 + (A / B) ** 2))


def _sri_F_by_hand(T, Pr, a, b, c, d, e):
    """SRI blending factor of Section 2.3.3 written out: X = 1 / (1 + (log10 P_r)^2) and
    F = d T^e (a exp(-b/T) + exp(-T/c))^X."""
    X = 1.0 / (1.0 + math.log10(Pr) ** 2)
    return d * T ** e * (a * math.exp(-b / T) + math.exp(-T / c)) ** X


def _pressure_for_Pr(T, Pr, k0, kinf):
    """Pressure at which P_r = (k_0 / k_inf) [M] takes the value Pr, [M] = P / (R T) (unit efficiencies)."""
    k0v = k0[0] * T ** k0[1] * math.exp(-k0[2] / T)
    kiv = kinf[0] * T ** kinf[1] * math.exp(-kinf[2] / T)
    return Pr * kiv / k0v * R_GAS * T


@pytest.mark.parametrize("lpr", [-2.0, 0.5, 3.0])
@pytest.mark.parametrize("form", ["troe", "troe_T2", "sri"])
def test_troe_and_sri_blending_values_in_mid_range(form, lpr):
    """The pressure modifier c = P_r / (1 + P_r) F of a falloff reaction at log10 P_r of -2, 0.5 and 3,
    against F computed by hand from Section 2.3.3 (the exponent (A/B)^2 and the constants 0.67, 0.4,
    0.806, 1.1762, 0.14 of Troe; the squared log10 P_r in the SRI exponent X)."""
    T, _, Y = _state(5)
    k0, kinf = (1.0e3, 0.0, 0.0), (1.0e4, 0.5, 100.0)
    Pr = 10.0 ** lpr
    if form == "sri":
        fp = (0.7, 450.0, 1300.0, 1.2, 0.15)
        F = _sri_F_by_hand(T, Pr, *fp)
        r = _falloff(KIND_FALLOFF, F_SRI, fp, k0=k0, kinf=kinf)
    else:
        a, T3, T1, T2 = 0.35, 180.0, 2500.0, 4200.0
        has = form == "troe_T2"
        F = _troe_F_by_hand(T, Pr, a, T3, T1, T2 if has else None)
        r = _falloff(KIND_FALLOFF, F_TROE, (a, T3, T1, T2 if has else 0.0, 0.0), has_T2=int(has), k0=k0, kinf=kinf)
    c = _om(mechs.one_reaction_model(r, TWO)).reaction_rates(T, _pressure_for_Pr(T, Pr, k0, kinf), Y)["c"][0]
    assert c == pytest.approx(Pr / (1.0 + Pr) * F, rel=1e-12)
    assert abs(F - 1.0) > 1e-3                       # a point where the blending matters


def test_falloff_pressure_limits():
    T, _, Y = _state(5)
    k0, kinf = (1.0e3, 0.2, 500.0), (1.0e4, 0.5, 100.0)
    k0v = k0[0] * T ** k0[1] * math.exp(-k0[2] / T)
    kiv = kinf[0] * T ** kinf[1] * math.exp(-kinf[2] / T)
    om = _om(mechs.one_reaction_model(_falloff(KIND_FALLOFF, F_LINDEMANN, k0=k0, kinf=kinf), TWO))
    for P, expect in [(1e14, lambda M: kiv), (1e-9, lambda M: k0v * M)]:
        r = om.reaction_rates(T, P, Y)
        M = P / (R_GAS * T)
        assert r["c"][0] * r["kf"][0] == pytest.approx(expect(M), rel=1e-6)


def test_sri_special_cases():
    T, P, Y = _state(5)
    d, e = 1.3, 0.25
    # c -> infinity and a = 0: base = 1, F = d T^e at any P_r
    om = _om(mechs.one_reaction_model(_falloff(KIND_FALLOFF, F_SRI, (0.0, 300.0, 1e300, d, e)), TWO))
    lind = _om(mechs.one_reaction_model(_falloff(KIND_FALLOFF, F_LINDEMANN), TWO))
    c_sri, c_lind = om.reaction_rates(T, P, Y)["c"][0], lind.reaction_rates(T, P, Y)["c"][0]
    assert c_sri == pytest.approx(c_lind * d * T ** e, rel=1e-13)


def test_plog_grid_points_and_log_interpolation():
    grid = [(1.0 * P_ATM, 1.0e5, 0.5, 1000.0), (3.0 * P_ATM, 3.0e5, 0.2, 1500.0),
            (20.0 * P_ATM, 2.0e6, -0.4, 800.0), (100.0 * P_ATM, 4.0e6, 0.1, 2000.0)]
    r = Reaction(kind=KIND_PLOG, rev_mode=REV_IRREVERSIBLE, reac=[(0, 1), (1, 1)], prod=[(2, 1)], plog=grid)
    om = _om(mechs.one_reaction_model(r, TWO))
    T, _, Y = _state(5)
    lk = [math.log(A * T ** b * math.exp(-Ta / T)) for _, A, b, Ta in grid]
    lp = [math.log(p) for p, *_ in grid]
    for P in [p for p, *_ in grid] + [1.7 * P_ATM, 9.0 * P_ATM, 55.0 * P_ATM, 0.3 * P_ATM, 300.0 * P_ATM]:
        expect = math.exp(np.interp(math.log(P), lp, lk))
        assert om.reaction_rates(T, P, Y)["kf"][0] == pytest.approx(expect, rel=1e-12)


def test_chebyshev_matches_numpy_chebval2d():
    rng = np.random.default_rng(7)
    eta = rng.normal(0, 0.5, size=(7, 3))
    eta[0, 0] = 9.0
    rngs = (300.0, 3000.0, 0.1 * P_ATM, 100.0 * P_ATM)
    r = Reaction(kind=KIND_CHEB, rev_mode=REV_IRREVERSIBLE, reac=[(0, 1), (1, 1)], prod=[(2, 1)],
                 cheb_shape=(7, 3), cheb_range=rngs, cheb_eta=eta)
    om = _om(mechs.one_reaction_model(r, TWO))
    for T, P in [(800.0, 2 * P_ATM), (1500.0, 40 * P_ATM), (2499.0, 1.1 * P_ATM), (300.0, 0.1 * P_ATM)]:
        Tt = (2 / T - 1 / rngs[0] - 1 / rngs[1]) / (1 / rngs[1] - 1 / rngs[0])
        pt = (2 * math.log10(P) - math.log10(rngs[2]) - math.log10(rngs[3])) / (math.log10(rngs[3]) - math.log10(rngs[2]))
        expect = 10.0 ** np.polynomial.chebyshev.chebval2d(Tt, pt, eta)
        # and the paper's trigonometric definition T_n(x) = cos(n arccos x)
        trig = sum(eta[i, j] * math.cos(i * math.acos(Tt)) * math.cos(j * math.acos(pt))
                   for i in range(7) for j in range(3))
        kf = om.reaction_rates(T, P, _state(5)[2])["kf"][0]
        assert kf == pytest.approx(expect, rel=1e-12)
        assert math.log10(kf) == pytest.approx(trig, rel=1e-12, abs=1e-12)


# ---------------------------------------------------------------------------------------------
# source-term invariants

@pytest.mark.parametrize("cfg", [0, 1])
def test_mass_and_element_conservation(cfg):
    model = synth.config_model(cfg)
    T, P, Y = synth.config_states(cfg, 32)
    J, f, Js, fs = _om(model).jacobian(T, P, Y, with_scale=True)
    W = np.array([s.W for s in model.species])
    E = np.array([s.elem for s in model.species], dtype=np.float64)     # N x n_elements
    # sum_k dY_k/dt = 0
    assert np.all(np.abs(f[:, 1:].sum(1)) <= 1e-13 * fs[:, 1:].sum(1))
    # sum_k n_ke omega_k = 0  <=>  sum_k n_ke f_k / W_k = 0
    lhs = (f[:, 1:] / W) @ E
    bound = (fs[:, 1:] / W) @ E
    assert np.all(np.abs(lhs) <= 1e-13 * bound)


def test_energy_equation_conserves_enthalpy():
    """Constant-p adiabatic: sum_k h_k dY_k/dt + c_p dT/dt = 0, h_k by quadrature of cp."""
    model = synth.config_model(0)
    T, P, Y = synth.config_states(0, 6)
    f = _om(model).dydt(T, P, Y)
    W = np.array([s.W for s in model.species])
    for s in range(len(T)):
        h = np.array([R_GAS / sp.W * _H_over_R_by_quadrature(_coeffs(sp, T[s]), T[s]) for sp in model.species])
        cpk = np.array([R_GAS / sp.W * np.polynomial.polynomial.polyval(T[s], _coeffs(sp, T[s])[:5])
                        for sp in model.species])
        cp = np.sum(Y[s] * cpk)
        terms = h * f[s, 1:]
        assert abs(terms.sum() + cp * f[s, 0]) <= 1e-11 * np.abs(terms).sum()
    del W


def _equilibrium_state(model, om, T, lam):
    """ln[X_k] = ln(p_atm/(R T)) + S_k/R - H_k/(R T) + sum_e n_ke lambda_e: every balanced
    reaction then has sum_k nu_k ln[X_k] = ln K_c, so R_f = R_r."""
    th = om.species_thermo(T)
    E = np.array([s.elem for s in model.species], dtype=np.float64)
    lnC = math.log(P_ATM / (R_GAS * T)) + th["SR"] - th["HRT"] + E @ lam
    C = np.exp(lnC)
    W = np.array([s.W for s in model.species])
    P = R_GAS * T * C.sum()
    rho = np.sum(C * W)
    return P, C * W / rho


def test_equilibrium_gives_zero_net_rates():
    model = mechs.mixed_model(seed=21)
    for r in model.reactions:
        r.rev_mode = REV_KC
    om = _om(model)
    rng = np.random.default_rng(5)
    for T in (900.0, 1400.0, 2200.0):
        lam = rng.uniform(-1.5, 1.5, size=model.n_elements)
        P, Y = _equilibrium_state(model, om, T, lam)
        r = om.reaction_rates(T, P, Y)
        assert np.all(np.abs(r["Rf"] - r["Rr"]) <= 1e-11 * np.maximum(r["Rf"], r["Rr"]))
        f, fs = om.jacobian([T], [P], Y[None], with_scale=True)[1::2]
        assert np.all(np.abs(f) <= 1e-10 * fs + 1e-300)


# ---------------------------------------------------------------------------------------------
# the analytical Jacobian against derivatives of the source terms

def _check_against_reference(J, Js, Jref, tol_rel=1e-10, kappa_mult=64.0):
    err = np.abs(J - Jref)
    bound = tol_rel * np.maximum(np.abs(Jref), 1e-20) + kappa_mult * EPS * Js
    bad = err > bound
    return int(bad.sum()), err, bound


@pytest.mark.parametrize("case", range(len(mechs.TYPE_CASES)))
def test_jacobian_matches_complex_step_per_reaction_type(case):
    label, kw = mechs.TYPE_CASES[case]
    model = mechs.typed_model(label, seed=100 + case, **kw)
    om = _om(model)
    T, P, Y = synth.generate_states(model.n_species, 12, seed=200 + case)
    J, f, Js, fs = om.jacobian(T, P, Y, with_scale=True)
    Jc = om.jacobian_complex_step(T, P, Y)
    nbad, err, bound = _check_against_reference(J, Js, Jc)
    assert nbad == 0, (label, kw)
    # structural zeros: column N and the energy-row entry of column N
    assert np.all(J[:, :, -1] == 0.0)


@pytest.mark.parametrize("cfg", [0, 1])
def test_jacobian_matches_complex_step_configs(cfg):
    model = synth.config_model(cfg)
    om = _om(model)
    T, P, Y = synth.config_states(cfg, 8 if cfg == 0 else 3)
    J, f, Js, fs = om.jacobian(T, P, Y, with_scale=True)
    Jc = om.jacobian_complex_step(T, P, Y)
    nbad, err, bound = _check_against_reference(J, Js, Jc)
    assert nbad == 0
    well = (Js <= 4500.0 * np.abs(J)) & (np.abs(J) > 1e-20)
    assert np.max(err[well] / np.abs(J[well])) < 1e-11


def test_jacobian_matches_central_differences():
    model = mechs.mixed_model(seed=31)
    om = _om(model)
    T, P, Y = synth.generate_states(model.n_species, 6, seed=32)
    T = np.where(np.abs(T - 1000.0) < 50.0, T + 120.0, T)      # stay clear of the NASA7 T_mid switch
    J, f, Js, fs = om.jacobian(T, P, Y, with_scale=True)
    N = model.n_species
    for s in range(len(T)):
        Jfd = np.zeros((N + 1, N + 1))
        hT = 1e-3 * T[s]
        fT = [om.dydt([T[s] + a * hT], [P[s]], Y[s][None])[0] for a in (-2, -1, 1, 2)]
        Jfd[:, 0] = (fT[0] - 8 * fT[1] + 8 * fT[2] - fT[3]) / (12 * hT)
        for j in range(N - 1):
            h = 1e-3 * min(Y[s, j], Y[s, N - 1])
            fs_ = []
            for a in (-2, -1, 1, 2):
                Yp = Y[s].copy()
                Yp[j] += a * h
                Yp[N - 1] -= a * h
                fs_.append(om.dydt([T[s]], [P[s]], Yp[None])[0])
            Jfd[:, 1 + j] = (fs_[0] - 8 * fs_[1] + 8 * fs_[2] - fs_[3]) / (12 * h)
        well = (Js[s] <= 100.0 * np.abs(J[s])) & (np.abs(J[s]) > 1e-12 * np.abs(J[s]).max())
        rel = np.abs(J[s] - Jfd)[well] / np.abs(J[s])[well]
        assert np.median(rel) < 1e-8
        assert np.quantile(rel, 0.99) < 1e-5


@pytest.mark.parametrize("cfg", [0, 1])
def test_jacobian_row_invariants(cfg):
    """sum_k J_{k,j} = 0 (mass) and sum_k n_ke/W_k J_{k,j} = 0 (elements) for every column j."""
    model = synth.config_model(cfg)
    T, P, Y = synth.config_states(cfg, 8)
    J, f, Js, fs = _om(model).jacobian(T, P, Y, with_scale=True)
    W = np.array([s.W for s in model.species])
    E = np.array([s.elem for s in model.species], dtype=np.float64)
    assert np.all(np.abs(J[:, 1:, :].sum(1)) <= 1e-12 * Js[:, 1:, :].sum(1) + 1e-300)
    lhs = np.einsum("skj,ke->sje", J[:, 1:, :], E / W[:, None])
    bound = np.einsum("skj,ke->sje", Js[:, 1:, :], E / W[:, None])
    assert np.all(np.abs(lhs) <= 1e-12 * bound + 1e-300)


def test_jacobian_closed_form_recombination():
    """A + A -> B (B = A2), irreversible, N = 2: hand-derived f and J.

    f_A = -2 k rho Y_A^2 / W_A, f_B = -f_A; with D = d/dY_A - d/dY_B at fixed T, p:
    D rho = -rho W (1/W_A - 1/W_B), D f_A = -(2k/W_A)(Y_A^2 D rho + 2 rho Y_A),
    d f_A/dT = -(2/W_A) Y_A^2 (k' rho + k drho/dT), drho/dT = -rho/T,
    f_T = -(h_A f_A + h_B f_B)/c_p."""
    vecs = [(1, 0), (2, 0)]
    A, beta, Ta = 3.0e3, 0.7, 2500.0
    r = Reaction(kind=KIND_ELEMENTARY, rev_mode=REV_IRREVERSIBLE, reac=[(0, 2)], prod=[(1, 1)], arr=(A, beta, Ta))
    model = mechs.one_reaction_model(r, vecs, seed=3)
    om = _om(model)
    P = 5.0 * P_ATM
    for T, YA in [(900.0, 0.3), (1700.0, 0.85), (2400.0, 0.05)]:
        Y = np.array([YA, 1.0 - YA])
        WA, WB = model.species[0].W, model.species[1].W
        Wm = 1.0 / (Y[0] / WA + Y[1] / WB)
        rho = P * Wm / (R_GAS * T)
        k = A * T ** beta * math.exp(-Ta / T)
        kp = k * (beta + Ta / T) / T
        polyval = np.polynomial.polynomial.polyval
        a = [_coeffs(sp, T) for sp in model.species]
        h = np.array([R_GAS / sp.W * _H_over_R_by_quadrature(a[i], T) for i, sp in enumerate(model.species)])
        cpk = np.array([R_GAS / sp.W * polyval(T, a[i][:5]) for i, sp in enumerate(model.species)])
        dcpk = np.array([R_GAS / sp.W * polyval(T, np.polynomial.polynomial.polyder(a[i][:5]))
                         for i, sp in enumerate(model.species)])
        cp, dcp = Y @ cpk, Y @ dcpk
        fA = -2 * k * rho * YA ** 2 / WA
        fB = -fA
        fT = -(h[0] * fA + h[1] * fB) / cp
        Drho = -rho * Wm * (1 / WA - 1 / WB)
        DfA = -(2 * k / WA) * (YA ** 2 * Drho + 2 * rho * YA)
        dfA_dT = -(2 / WA) * YA ** 2 * (kp * rho + k * (-rho / T))
        # energy row: d/dT of -(h.f)/cp and D of the same (D cp = cp_A - cp_B, D h_k = 0)
        hf = h[0] * fA + h[1] * fB
        dfT_dT = -(cpk[0] * fA + cpk[1] * fB + h[0] * dfA_dT - h[1] * dfA_dT) / cp + hf * dcp / cp ** 2
        DfT = -(h[0] * DfA - h[1] * DfA) / cp + hf * (cpk[0] - cpk[1]) / cp ** 2
        J, f = om.jacobian([T], [P], Y[None])
        np.testing.assert_allclose(f[0], [fT, fA, fB], rtol=1e-12)
        expect = np.array([[dfT_dT, DfT, 0.0], [dfA_dT, DfA, 0.0], [-dfA_dT, -DfA, 0.0]])
        np.testing.assert_allclose(J[0], expect, rtol=1e-10, atol=0)


def test_load_rejects_corrupt_and_truncated_models():
    blob = synth.to_bytes(synth.config_model(0))
    with pytest.raises(ValueError):
        oracle.load_model(blob[:-3])
    with pytest.raises(ValueError):
        oracle.load_model(b"NOTAMODEL" + blob[9:])
    with pytest.raises(ValueError):
        oracle.load_model(blob + b"\0")


# ---------------------------------------------------------------------------------------------
# forward-difference Jacobian (the paper's finite-difference comparison)

@pytest.mark.parametrize("cfg", [0, 1])
def test_forward_difference_within_its_rounding_bound_of_complex_step(cfg):
    """The first-order forward difference converges to the exact (complex-step) Jacobian: every
    entry lies within the rounding bound 64 eps S / h that the oracle reports for it plus a
    truncation allowance of 1e-5 |J|. Perturbing Y_j without the opposite step in Y_N, a wrong
    increment or a shifted column gives errors of order |J| instead."""
    model = synth.config_model(cfg)
    om = _om(model)
    T, P, Y = synth.config_states(cfg, 6, seed_offset=77)
    Jfd, Jsc = om.jacobian_fd(T, P, Y, with_scale=True)
    Jcs = om.jacobian_complex_step(T, P, Y)
    err = np.abs(Jfd - Jcs)
    assert np.all(err <= 64 * EPS * Jsc + 1e-5 * np.abs(Jcs) + 1e-300)
    assert np.all(Jfd[:, :, -1] == 0.0)
    # the typical entry is accurate to far better than the allowance
    big = np.abs(Jcs) > 1e-6 * np.abs(Jcs).max()
    assert np.median(err[big] / np.abs(Jcs[big])) < 1e-5


def test_forward_difference_increment_rule():
    """Column c is (f(y + h_c d_c) - f(y)) / h_c with h_c = 2^-26 max(|y_c|, a_c), a = 1 K for T
    and 1e-10 for mass fractions, d_c = e_T or e_Yj - e_YN; checked on the source terms directly."""
    model = synth.config_model(0)
    om = _om(model)
    T, P, Y = synth.config_states(0, 1, seed_offset=5)
    Y = Y.copy()
    Y[0, 3] = 0.0                                              # takes the 1e-10 floor
    N = model.n_species
    Jfd, Jsc = om.jacobian_fd(T, P, Y, with_scale=True)
    f0 = om.dydt(T, P, Y)[0]
    for c in (0, 1, 4, N - 1):
        Tp, Yp = T.copy(), Y.copy()
        if c == 0:
            h = 2.0 ** -26 * max(abs(T[0]), 1.0)
            Tp[0] += h
        else:
            h = 2.0 ** -26 * max(abs(Y[0, c - 1]), 1e-10)
            Yp[0, c - 1] += h
            Yp[0, N - 1] -= h
        col = (om.dydt(Tp, P, Yp)[0] - f0) / h
        assert np.all(np.abs(col - Jfd[0, :, c]) <= 64 * EPS * Jsc[0, :, c] + 1e-300)


# ---------------------------------------------------------------------------------------------
# constant volume (Section 3.3)

def _rho(model, T, P, Y):
    W = 1.0 / (Y / np.array([s.W for s in model.species])).sum(axis=1)
    return P * W / (R_GAS * T)


@pytest.mark.parametrize("cfg", [0, 1])
def test_constant_volume_species_rates_equal_constant_pressure_rates(cfg):
    """At the density of the same state, dY_k/dt does not depend on which variable is held fixed
    (both are W_k omega_k / rho); the temperature rates are tied by c_p - c_v = R/W per species:
    c_v f0_cv + sum_k u_k f_k = 0 and c_p f0_cp + sum_k h_k f_k = 0 with h_k = u_k + R T / W_k."""
    model = synth.config_model(cfg)
    om = _om(model)
    T, P, Y = synth.config_states(cfg, 6, seed_offset=3)
    rho = _rho(model, T, P, Y)
    (fcv, fcv_s), fcp = om.dydt_cv(T, rho, Y, with_scale=True), om.dydt(T, P, Y)
    scale = np.abs(fcp[:, 1:]).max(axis=1, keepdims=True)
    assert np.all(np.abs(fcv[:, 1:] - fcp[:, 1:]) <= 1e-13 * scale)
    # rounding scales: bound the values; the species ones are the constant-pressure ones
    _, _, _, fcp_s = om.jacobian(T, P, Y, with_scale=True)
    assert np.all(np.abs(fcv) <= fcv_s * (1 + 1e-12))
    assert np.allclose(fcv_s[:, 1:], fcp_s[:, 1:], rtol=1e-12, atol=0)
    W = np.array([s.W for s in model.species])
    for s in range(len(T)):
        cpk = np.array([np.polynomial.polynomial.polyval(T[s], _coeffs(sp, T[s])[:5]) for sp in model.species]) * R_GAS / W
        cvk = cpk - R_GAS / W
        cp, cv = (Y[s] * cpk).sum(), (Y[s] * cvk).sum()
        sum_hf = -cp * fcp[s, 0]                                   # sum_k h_k f_k
        sum_uf = sum_hf - R_GAS * T[s] * (fcp[s, 1:] / W).sum()    # sum_k u_k f_k
        assert abs(cv * fcv[s, 0] + sum_uf) <= 1e-9 * (abs(sum_hf) + abs(cv * fcv[s, 0]))


def test_constant_volume_jacobian_matches_central_differences():
    """The complex-step constant-volume Jacobian against fourth-order central differences of the
    constant-volume source terms, on the entries the differences resolve: well-conditioned ones
    whose difference-quotient rounding (~30 eps S_f / h, S_f the source-term scale of the row,
    equal at constant pressure) is below 1e-7 |J|. There the two agree to ~1e-12 typically; a
    dropped or mis-signed term shows up as an O(1) relative error."""
    model = mechs.mixed_model(seed=33)
    om = _om(model)
    T, P, Y = synth.generate_states(model.n_species, 5, seed=34)
    T = np.where(np.abs(T - 1000.0) < 50.0, T + 120.0, T)
    rho = _rho(model, T, P, Y)
    J, Js = om.jacobian_cv(T, rho, Y, with_scale=True)
    _, _, _, fs = om.jacobian(T, P, Y, with_scale=True)
    N = model.n_species
    for s in range(len(T)):
        Jfd = np.zeros((N + 1, N + 1))
        steps = np.empty(N + 1)
        hT = 1e-3 * T[s]
        steps[0] = hT
        fT = [om.dydt_cv([T[s] + a * hT], [rho[s]], Y[s][None])[0] for a in (-2, -1, 1, 2)]
        Jfd[:, 0] = (fT[0] - 8 * fT[1] + 8 * fT[2] - fT[3]) / (12 * hT)
        for j in range(N - 1):
            h = 1e-3 * min(Y[s, j], Y[s, N - 1])
            steps[1 + j] = h
            fs_ = []
            for a in (-2, -1, 1, 2):
                Yp = Y[s].copy()
                Yp[j] += a * h
                Yp[N - 1] -= a * h
                fs_.append(om.dydt_cv([T[s]], [rho[s]], Yp[None])[0])
            Jfd[:, 1 + j] = (fs_[0] - 8 * fs_[1] + 8 * fs_[2] - fs_[3]) / (12 * h)
        steps[N] = np.inf
        fd_round = 30 * EPS * fs[s][:, None] / steps[None, :]
        well = (Js[s] <= 100.0 * np.abs(J[s])) & (np.abs(J[s]) > 1e-12 * np.abs(J[s]).max()) & \
            (fd_round <= 1e-7 * np.abs(J[s]))
        rel = np.abs(J[s] - Jfd)[well] / np.abs(J[s])[well]
        assert well.sum() >= 10 and well[:, 0].any() and well[0, :].any() and well[1:, 1:].any()
        assert np.median(rel) < 1e-10
        assert rel.max() < 1e-7
    assert np.all(J[:, :, -1] == 0.0)
    assert np.all(np.abs(J[:, 1:, :].sum(axis=1)) <= 1e-12 * np.abs(J[:, 1:, :]).sum(axis=1) + 1e-300)


def test_constant_volume_jacobian_is_sparse_for_elementary_reactions():
    """Section 3.3: with the density fixed, a species row k has entries only in the columns of the
    species it reacts with directly (columns move Y_j against Y_N, so those of N's partners too);
    the constant-pressure Jacobian of the same model is dense through d rho / d Y_j."""
    model = mechs.typed_model("elementary", seed=35, n_species=10, n_reactions=6, rev_modes=(1,))
    om = _om(model)
    N = model.n_species
    T, P, Y = synth.generate_states(N, 3, seed=36)
    Jcv = om.jacobian_cv(T, _rho(model, T, P, Y), Y)
    Jcp, _ = om.jacobian(T, P, Y)
    partners = [set() for _ in range(N)]
    for r in model.reactions:
        sps = {s for s, _ in r.reac} | {s for s, _ in r.prod}
        for k in sps:
            partners[k] |= sps
    zero = 0
    for k in range(N):
        for j in range(N - 1):
            if j not in partners[k] and (N - 1) not in partners[k]:
                assert np.all(Jcv[:, 1 + k, 1 + j] == 0.0)
                assert np.all(Jcp[:, 1 + k, 1 + j] != 0.0) or not any(partners[k])
                zero += 1
    assert zero > 0


@pytest.mark.parametrize("ftype", ["lindemann", "troe", "sri"])
def test_falloff_with_absent_third_body_species(ftype):
    """A falloff reaction whose single third-body species m is absent has P_r = 0, where the forms of
    dc/dT and dc/dY with 1/P_r are 0 * inf. With F constant below the P_r clamp (reading of the
    clamp), c = P_r F(clamp) / (1 + P_r) has dc/d[X_m] = (k_0/k_inf) F(clamp) and dc/dT = 0 there,
    so the only nonzero entries of the reaction's columns are
    d(dY_k/dt)/dY_m = (W_k / rho) nu_k (k_0/k_inf) F (rho / W_m) R, computed here independently.
    (The complex step is no check at this point: the sign of an O(h^2) real part of P_r decides
    whether its perturbed log P_r is clamped.)"""
    import math
    model = mechs.typed_model(ftype, seed=81, n_species=8, n_reactions=6, species_tb_fraction=1.0,
                              chem_fraction=0.0)
    N = model.n_species
    r = next(x for x in model.reactions if x.tb_species >= 0 and x.tb_species != N - 1)
    import copy
    sub = copy.deepcopy(model)
    sub.reactions = [r]
    om = _om(sub)
    T, P, Y = synth.generate_states(N, 3, seed=82)
    m = r.tb_species
    Y[:, m] = 0.0
    Y /= Y.sum(axis=1, keepdims=True)
    J, f = om.jacobian(T, P, Y)
    assert np.all(np.isfinite(J))
    W = np.array([sp.W for sp in model.species])
    for s in range(len(T)):
        t = T[s]
        rho = P[s] / (R_GAS * t * (Y[s] / W).sum())
        k0 = r.k0[0] * t ** r.k0[1] * math.exp(-r.k0[2] / t)
        ki = r.kinf[0] * t ** r.kinf[1] * math.exp(-r.kinf[2] / t)
        if ftype == "lindemann":
            F = 1.0
        elif ftype == "troe":
            a, T3, T1, T2 = r.fparams[:4]
            Fc = (1 - a) * math.exp(-t / T3) + a * math.exp(-t / T1) + (math.exp(-T2 / t) if r.troe_has_T2 else 0.0)
            lFc = math.log10(Fc)
            At, Bt = -300.0 - 0.67 * lFc - 0.4, 0.806 - 1.1762 * lFc + 0.14 * 300.0
            F = Fc ** (1.0 / (1.0 + (At / Bt) ** 2))
        else:
            a, b, c, d, e = r.fparams[:5]
            F = d * t ** e * (a * math.exp(-b / t) + math.exp(-t / c)) ** (1.0 / (1.0 + 300.0 ** 2))
        rates = om.reaction_rates(t, P[s], Y[s])
        R = rates["Rf"][0] - rates["Rr"][0]
        assert rates["c"][0] == 0.0
        dq = k0 / ki * F * rho / W[m] * R
        for k in range(N):
            nu = sum(v for x, v in r.prod if x == k) - sum(v for x, v in r.reac if x == k)
            want = W[k] / rho * nu * dq
            assert abs(J[s, 1 + k, 1 + m] - want) <= 1e-12 * abs(dq * W.max() / rho) + 1e-300
        assert np.all(J[s, 1:, 0] == 0.0)              # dc/dT = 0 and c = 0: no temperature column
