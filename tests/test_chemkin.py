"""Chemkin reader and writer (no GPU): unit and reaction-order conversions against hand-converted
values, molecular weights from element composition, every supported keyword, errors, and round
trips of the synthetic models through Chemkin text evaluated by the oracle."""
import os

import numpy as np
import pytest

import oracle
from paper_1605_03262_b300 import chemkin, synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "chemkin_features.inp")
R = 8.31446261815324
CAL = 4.184


def _fixture():
    with open(GOLDEN) as f:
        return chemkin.parse(f.read())


def _close(a, b, rel=1e-14):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    assert np.all(np.abs(a - b) <= rel * np.maximum(np.abs(b), 1e-300)), (a, b)


def test_fixture_parameters_in_si():
    """Each reaction's parameters, converted by hand: A (cm^3/mol)^(order-1)/s -> SI by
    1e-6^(order-1), the order counting a third body for +M and for k_0; Ta = Ea cal/mol / R."""
    m = _fixture()
    r = m.reactions
    assert (m.n_species, m.n_reactions, m.n_elements) == (10, 11, 4)
    _close(r[0].arr, (3.1e14 * 1e-6, -0.2, 1.52e4 * CAL / R))
    assert r[0].kind == synth.KIND_ELEMENTARY and r[0].rev_mode == synth.REV_KC
    _close(r[1].arr, (2.4e17 * 1e-12, -1.1, 0.0))
    assert r[1].kind == synth.KIND_THIRD_BODY and r[1].tb_mode == synth.TB_MIXTURE
    assert r[1].eff == [(0, 2.5), (5, 11.0), (8, 0.7)]                  # N2/1.0/ is the default
    assert r[2].kind == synth.KIND_FALLOFF and r[2].ftype == synth.F_TROE and r[2].troe_has_T2 == 1
    _close(r[2].kinf, (5.0e12 * 1e-6, 0.4, 0.0))
    _close(r[2].k0, (7.2e19 * 1e-12, -1.3, 0.0))
    _close(r[2].fparams[:4], (0.55, 1e-30, 1e30, 8e3))
    assert r[3].kind == synth.KIND_CHEM and r[3].ftype == synth.F_SRI
    assert (r[3].tb_mode, r[3].tb_species) == (synth.TB_SPECIES, 8)
    _close(r[3].k0, (3.0e16 * 1e-12, 0.0, 0.0))
    _close(r[3].kinf, (1.6e12 * 1e-6, 0.15, 120.0 * CAL / R))
    _close(r[3].fparams, (0.45, 210.0, 1100.0, 0.9, 0.05))
    assert r[4].kind == synth.KIND_FALLOFF and r[4].ftype == synth.F_LINDEMANN and r[4].reac == [(4, 2)]
    _close(r[4].k0, (2.3e18 * 1e-12, -0.9, -1700.0 * CAL / R))
    assert r[5].kind == synth.KIND_PLOG
    _close(np.array(r[5].plog), [(0.1 * 101325.0, 4.0e12 * 1e-6, 0.5, 6000.0 * CAL / R),
                                 (1.0 * 101325.0, 6.0e12 * 1e-6, 0.45, 6200.0 * CAL / R),
                                 (10.0 * 101325.0, 9.0e12 * 1e-6, 0.4, 6500.0 * CAL / R)])
    assert r[6].kind == synth.KIND_CHEB and r[6].rev_mode == synth.REV_IRREVERSIBLE
    eta = np.array([[13.1, 0.2], [-0.25, 0.03], [0.07, -0.01]])
    eta[0, 0] += np.log10(1e-6)                                        # log10 k to SI, order 2
    _close(r[6].cheb_eta, eta)
    _close(r[6].cheb_range, (300.0, 2500.0, 0.01 * 101325.0, 100.0 * 101325.0))
    assert r[7].rev_mode == synth.REV_EXPLICIT
    _close(r[7].rev_arr, (3.1e13 * 1e-6, 0.05, 5.6e4 * CAL / R))
    assert r[8].rev_mode == synth.REV_IRREVERSIBLE
    assert r[9].reac == r[10].reac and r[9].prod == r[10].prod        # duplicates kept apart


def test_molecular_weights_from_elements():
    m = _fixture()
    W = {n: s.W for n, s in zip("H2 O2 H O OH H2O HO2 H2O2 AR N2".split(), m.species)}
    _close(W["H2O"], (2 * 1.00794 + 15.9994) * 1e-3)
    _close(W["AR"], 39.948e-3)
    _close(W["N2"], 2 * 14.0067e-3)


@pytest.mark.parametrize("unit,scale", [("KCAL/MOLE", 1e3 * CAL / R), ("KELVINS", 1.0), ("JOULES/MOLE", 1.0 / R),
                                        ("KJOULES/MOLE", 1e3 / R), ("CAL/MOLE", CAL / R)])
def test_energy_units(unit, scale):
    text = open(GOLDEN).read().replace("REACTIONS\n", "REACTIONS %s\n" % unit)
    m = chemkin.parse(text)
    _close(m.reactions[0].arr[2], 1.52e4 * scale)


def test_molecule_units():
    text = open(GOLDEN).read().replace("REACTIONS\n", "REACTIONS MOLECULES\n")
    m = chemkin.parse(text)
    _close(m.reactions[0].arr[0], 3.1e14 * 6.02214076e23 * 1e-6)            # per molecule -> per mol
    _close(m.reactions[1].arr[0], 2.4e17 * 6.02214076e23 ** 2 * 1e-12)


@pytest.mark.parametrize("bad,what", [
    ("H + O2 <=> O + OH                 3.10E+14   -0.20   1.52E+04",
     "H + XX <=> O + OH                 3.10E+14   -0.20   1.52E+04"),
    ("   TROE / 0.55  1.0E-30  1.0E+30  8.0E+03 /", "   FORD / H 1.0 /"),
    ("2OH <=> O + H2O                   1.0E+10    0.0     0.0",
     "1.5OH <=> O + H2O                 1.0E+10    0.0     0.0"),
])
def test_unsupported_input_is_an_error(bad, what):
    text = open(GOLDEN).read().replace(bad, what)
    with pytest.raises(chemkin.ChemkinError):
        chemkin.parse(text)


def test_missing_thermo_is_an_error():
    text = open(GOLDEN).read().replace("SPECIES\nH2 ", "SPECIES\nCH4 H2 ")
    with pytest.raises(chemkin.ChemkinError):
        chemkin.parse(text)


def test_fixture_source_terms_conserve_mass():
    m = _fixture()
    om = oracle.load_model(synth.to_bytes(m))
    T, P, Y = synth.generate_states(m.n_species, 16, seed=8)
    f = om.dydt(T, P, Y)
    assert np.all(np.isfinite(f))
    assert np.all(np.abs(f[:, 1:].sum(axis=1)) <= 1e-12 * np.abs(f[:, 1:]).sum(axis=1))


def _merged(side, sp):
    d = dict(side)
    d[sp] = d.get(sp, 0) + 1
    return sorted(d.items())


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_round_trip_of_synthetic_models(cfg):
    """write -> parse keeps every reaction; a third-body reaction with one collider comes back as
    the equivalent elementary reaction with the collider on both sides (Chemkin has no other
    syntax for it). The oracle's source terms and Jacobian agree to the 9 digits of the thermo
    format."""
    m = synth.config_model(cfg)
    m2 = chemkin.parse(chemkin.write(m))
    assert (m2.n_species, m2.n_reactions) == (m.n_species, m.n_reactions)
    for a, b in zip(m.reactions, m2.reactions):
        if a.kind == synth.KIND_THIRD_BODY and a.tb_mode == synth.TB_SPECIES:
            assert b.kind == synth.KIND_ELEMENTARY
            assert b.reac == _merged(a.reac, a.tb_species) and b.prod == _merged(a.prod, a.tb_species)
            continue
        assert (a.kind, a.rev_mode, a.reac, a.prod, a.tb_mode, a.tb_species, a.ftype) == \
            (b.kind, b.rev_mode, b.reac, b.prod, b.tb_mode, b.tb_species, b.ftype)
    T, P, Y = synth.config_states(cfg, 4)
    J1, f1 = oracle.load_model(synth.to_bytes(m)).jacobian(T, P, Y)
    J2, f2 = oracle.load_model(synth.to_bytes(m2)).jacobian(T, P, Y)
    assert np.linalg.norm(f1 - f2) <= 1e-6 * np.linalg.norm(f1)
    assert np.linalg.norm(J1 - J2) <= 1e-6 * np.linalg.norm(J1)
