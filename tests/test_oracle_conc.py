"""Pins of the oracle's molar-concentration basis at constant pressure (state (T, V, n_1..n_{N-1}),
the formulation the paper names as future work in Sections 3.4 and 6), against what the
mathematics and the physics fix rather than against the oracle itself:

- closed forms for one elementary reaction A + B -> C with an inert last species;
- element, mass and enthalpy conservation, with the last species' rate implied by the ideal-gas law
  at constant pressure (so dV/dt and dT/dt both enter);
- the Jacobian columns against fourth-order central differences of the source terms;
- homogeneity: d f / d V = f / V - sum_l [X_l] d f / d n_l (rows with a V factor), since every rate
  depends on n and V only through [X] = n / V;
- structural zeros: entries outside the sparsity pattern of the formulation are zero to rounding.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1605_03262_b300 import synth
from paper_1605_03262_b300.synth import P_ATM, R_GAS
from tests import mechs

EPS = 2.0 ** -52


def _H_quad(a, T):
    v, _ = integrate.quad(lambda t: np.polynomial.polynomial.polyval(t, a[:5]), 0.0, T, epsabs=0.0, epsrel=1e-13)
    return a[5] + v


def _implied_dnN(T, P, V, f):
    """dn_N/dt from n_N = P V / (R T) - sum_{k<N} n_k at constant P."""
    return P * f[1] / (R_GAS * T) - P * V * f[0] / (R_GAS * T * T) - f[2:].sum()


def test_closed_form_single_elementary_reaction():
    # A + B -> C (irreversible), D inert and last
    A, beta, Ta = 3.0e5, 0.7, 4000.0
    r = synth.Reaction(kind=synth.KIND_ELEMENTARY, rev_mode=synth.REV_IRREVERSIBLE, reac=[(0, 1), (1, 1)],
                       prod=[(2, 1)], arr=(A, beta, Ta))
    model = mechs.one_reaction_model(r, [(1, 0), (0, 1), (1, 1), (2, 0)])
    om = oracle.load_model(synth.to_bytes(model))
    T, P, V = np.array([1234.0]), np.array([3.0 * P_ATM]), np.array([2.5e-3])
    ntot = P[0] * V[0] / (R_GAS * T[0])
    nmol = np.array([[0.2, 0.3, 0.1]]) * ntot
    J, f = om.jacobian_conc(T, P, V, nmol)
    J, f = J[0], f[0]
    k = A * T[0] ** beta * math.exp(-Ta / T[0])
    dk = k * (beta + Ta / T[0]) / T[0]
    CA, CB = nmol[0, 0] / V[0], nmol[0, 1] / V[0]
    q = k * CA * CB
    # species rows (state order T, V, n_A, n_B, n_C): f = V nu q
    assert f[2:] == pytest.approx([-V[0] * q, -V[0] * q, V[0] * q], rel=1e-13)
    for row, nu in ((2, -1.0), (3, -1.0), (4, 1.0)):
        assert J[row, 0] == pytest.approx(nu * V[0] * dk * CA * CB, rel=1e-12)   # d/dT at fixed n, V
        assert J[row, 1] == pytest.approx(-nu * q, rel=1e-12)                     # d(V nu k n_A n_B / V^2)/dV
        assert J[row, 2] == pytest.approx(nu * k * CB, rel=1e-12)
        assert J[row, 3] == pytest.approx(nu * k * CA, rel=1e-12)
        assert abs(J[row, 4]) <= 1e-14 * k * (CA + CB)
    # dV/dt: the reaction removes one mole per event, so at constant T the volume shrinks by
    # V (R T / P) q; plus the thermal expansion V f_T / T
    assert f[1] == pytest.approx(V[0] * (f[0] / T[0] - R_GAS * T[0] / P[0] * q), rel=1e-12)


@pytest.mark.parametrize("which", ["mixed", "cfg0"])
def test_conservation_with_implied_last_species(which):
    model = mechs.mixed_model(seed=3, n_species=9, n_reactions=30) if which == "mixed" else synth.config_model(0)
    om = oracle.load_model(synth.to_bytes(model))
    N = model.n_species
    T, P, V, nmol = synth.generate_conc_states(N, 6, seed=21)
    f = om.dydt_conc(T, P, V, nmol)
    W = np.array([s.W for s in model.species])
    E = np.array([s.elem for s in model.species], dtype=np.float64)
    for s in range(len(T)):
        rates = np.concatenate([f[s, 2:], [_implied_dnN(T[s], P[s], V[s], f[s])]])
        assert abs(rates @ W) <= 1e-12 * (np.abs(rates) @ W)
        assert np.all(np.abs(rates @ E) <= 1e-12 * (np.abs(rates) @ E + 1e-300))
        # total enthalpy sum_k n_k H_k(T) is constant at constant pressure
        a = [(sp.a_low if T[s] < sp.T_mid else sp.a_high) for sp in model.species]
        H = np.array([R_GAS * _H_quad(a[i], T[s]) for i in range(N)])
        cp = np.array([R_GAS * np.polynomial.polynomial.polyval(T[s], a[i][:5]) for i in range(N)])
        n_all = np.concatenate([nmol[s], [P[s] * V[s] / (R_GAS * T[s]) - nmol[s].sum()]])
        dH = rates @ H + (n_all @ cp) * f[s, 0]
        assert abs(dH) <= 1e-11 * np.abs(rates * H).sum()


@pytest.mark.parametrize("seed", [3, 4])
def test_columns_against_central_differences(seed):
    model = mechs.mixed_model(seed=seed, n_species=9, n_reactions=30)
    om = oracle.load_model(synth.to_bytes(model))
    N = model.n_species
    T, P, V, nmol = synth.generate_conc_states(N, 3, seed=30 + seed, alpha=3.0)
    J, f = om.jacobian_conc(T, P, V, nmol)
    for s in range(len(T)):
        nN = P[s] * V[s] / (R_GAS * T[s]) - nmol[s].sum()
        x = np.concatenate([[T[s], V[s]], nmol[s]])
        for col in range(N + 1):
            h = 1e-5 * (abs(x[col]) if col < 2 else min(abs(x[col]), nN))
            d = []
            for st in (-2, -1, 1, 2):
                xp = x.copy()
                xp[col] += st * h
                d.append(om.dydt_conc(xp[:1], P[s:s + 1], xp[1:2], xp[2:][None])[0])
            fd = (d[0] - 8 * d[1] + 8 * d[2] - d[3]) / (12 * h)
            big = np.abs(J[s, :, col]) > 1e-3 * np.abs(J[s, :, col]).max()
            assert np.all(np.abs(fd - J[s, :, col])[big] <= 1e-6 * np.abs(J[s, big, col])), (s, col)


@pytest.mark.parametrize("cfg", [0, 1])
def test_homogeneity_and_structural_zeros(cfg):
    model = synth.config_model(cfg)
    om = oracle.load_model(synth.to_bytes(model))
    N = model.n_species
    T, P, V, nmol = synth.config_conc_states(cfg, 3)
    J, f, Js, fs = om.jacobian_conc(T, P, V, nmol, with_scale=True)
    assert np.all(np.isfinite(J)) and np.all(Js >= 0)
    # the scales bound the entries (structural zeros carry rounding noise of the row's size)
    rowmax = np.abs(J).max(axis=2, keepdims=True)
    assert np.all(np.abs(J) <= Js * (1 + 1e-6) + 1e-13 * rowmax)
    for s in range(len(T)):
        X = nmol[s] / V[s]
        lhs = J[s, :, 1]
        rhs = np.where(np.arange(N + 1) >= 1, f[s] / V[s], 0.0) - J[s, :, 2:] @ X
        scale = Js[s, :, 1] + np.abs(Js[s, :, 2:]) @ X
        assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale)
    # structural pattern: species k couples to n_j only through the reactions both take part in
    # (as participant, non-unity efficiency or third-body species), or to every n_j when species N
    # takes part in one of k's reactions
    pat = np.zeros((N, N), bool)
    for r in model.reactions:
        net = {}
        for sp, nu in r.reac:
            net[sp] = net.get(sp, 0) - nu
        for sp, nu in r.prod:
            net[sp] = net.get(sp, 0) + nu
        dep = {sp for sp, _ in r.reac} | {sp for sp, _ in r.prod}
        if r.tb_species >= 0:
            dep.add(r.tb_species)
        dep |= {sp for sp, a in r.eff if a != 1.0}
        for k, nu in net.items():
            if nu == 0:
                continue
            for j in dep:
                pat[k, j] = True
            if N - 1 in dep:
                pat[k, :] = True
    off = ~pat[: N - 1, : N - 1]
    blk, blks = J[:, 2:, 2:], Js[:, 2:, 2:]
    ref = np.abs(J[:, 2:, :]).max(axis=2)[:, :, None]
    assert np.all(np.abs(blk[:, off]) <= 1e-13 * np.broadcast_to(ref, blk.shape)[:, off] + 64 * EPS * blks[:, off])
