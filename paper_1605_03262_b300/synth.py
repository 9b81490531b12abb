"""Seeded synthetic chemical kinetic models and thermochemical states.

This module is the single source of inputs for both the CPU oracle (``oracle/``) and the CUDA
path: it draws model parameters and states from fixed seeds and serialises models to the binary
model format that both sides parse with their own, independent readers. It evaluates none of the
source-term or Jacobian arithmetic: no thermodynamic property, rate coefficient, production rate
or derivative is computed here. Parameter design uses only unit conversions, integer element
bookkeeping and least-squares polynomial fits of a heat-capacity curve (numpy routines).

Model content follows the paper's formulation (Section 2): species carry a molecular weight, an
element composition and two-range NASA seven-coefficient polynomials (Eqs. e:cpk, e:hk, e:sk);
reactions carry integer stoichiometry, a pressure-dependence kind (elementary, third-body,
falloff, chemically activated, PLOG, Chebyshev; Eq. e:rxn_pressure and Section 2.3), a
reversibility mode (irreversible, equilibrium constant or explicit reverse Arrhenius; Section
2.3.1), third-body efficiencies and falloff blending parameters (Lindemann/Troe/SRI).

Units of the stored model are SI throughout: W in kg/mol, A in (m^3/mol)^(order-1)/s, activation
temperatures in K, pressures in Pa. Arrhenius prefactors are drawn in cm^3-mol-s units and
converted by (1e-6)^(order-1).

Binary model format (little endian), written by :func:`to_bytes`::

    char[8]  magic "PYJACMEC"
    u32      version (=1)
    u32      n_elements, n_species, n_reactions
    species (n_species records):
        f64  W
        f64  T_low, T_mid, T_high
        f64  a_low[7], a_high[7]
        i32  elem[n_elements]
    reactions (n_reactions records):
        i32  kind      0 elementary, 1 third-body, 2 falloff, 3 chemically activated, 4 PLOG, 5 Chebyshev
        i32  rev_mode  0 irreversible, 1 via equilibrium constant, 2 explicit reverse Arrhenius
        i32  n_reac, then n_reac x (i32 species, i32 nu')
        i32  n_prod, then n_prod x (i32 species, i32 nu'')
        f64  A, beta, Ta                 (forward Arrhenius; unused for kinds 2, 3, 4, 5)
        if rev_mode == 2:  f64 Ar, beta_r, Ta_r
        if kind in (1, 2, 3):
            i32 tb_mode (1 mixture, 2 single species), i32 tb_species (-1 for mixture),
            i32 n_eff, then n_eff x (i32 species, f64 alpha)    (mixture only; default alpha = 1)
        if kind in (2, 3):
            f64 A0, beta0, Ta0, Ainf, betainf, Tainf             (low- and high-pressure limits)
            i32 ftype (0 Lindemann, 1 Troe, 2 SRI)
            f64 params[5]  Troe: a, T***, T*, T**, unused; SRI: a, b, c, d, e
            i32 troe_has_T2 (1 if the T** term is present)
        if kind == 4:  i32 n_p, then n_p x (f64 p, A, beta, Ta), p strictly increasing
        if kind == 5:  i32 NT, NP; f64 Tmin, Tmax, Pmin, Pmax; f64 eta[NT*NP] (row-major [t][p], log10 k in SI)
"""
from __future__ import annotations

import dataclasses
import math
import struct
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Species", "Reaction", "Model", "generate_model", "generate_states", "to_bytes",
    "CONFIGS", "config_model", "config_states", "P_ATM", "R_GAS",
    "KIND_ELEMENTARY", "KIND_THIRD_BODY", "KIND_FALLOFF", "KIND_CHEM", "KIND_PLOG", "KIND_CHEB",
    "REV_IRREVERSIBLE", "REV_KC", "REV_EXPLICIT", "F_LINDEMANN", "F_TROE", "F_SRI",
    "TB_MIXTURE", "TB_SPECIES",
]

# Unit-conversion constants (SI). R_GAS converts kcal/mol activation energies to temperatures.
R_GAS = 8.31446261815324       # J/(mol K)
P_ATM = 101325.0               # Pa
CAL = 4.184                    # J/cal

KIND_ELEMENTARY, KIND_THIRD_BODY, KIND_FALLOFF, KIND_CHEM, KIND_PLOG, KIND_CHEB = range(6)
REV_IRREVERSIBLE, REV_KC, REV_EXPLICIT = range(3)
F_LINDEMANN, F_TROE, F_SRI = range(3)
TB_MIXTURE, TB_SPECIES = 1, 2

# Element molar masses (kg/mol) used to give synthetic species a molecular weight.
_ELEMENT_MASS = (1.008e-3, 12.011e-3, 15.999e-3, 14.007e-3, 39.948e-3, 32.06e-3)

MAGIC = b"PYJACMEC"
VERSION = 1


@dataclasses.dataclass
class Species:
    W: float
    T_low: float
    T_mid: float
    T_high: float
    a_low: np.ndarray     # 7 NASA coefficients, T < T_mid
    a_high: np.ndarray    # 7 NASA coefficients, T >= T_mid
    elem: np.ndarray      # element counts


@dataclasses.dataclass
class Reaction:
    kind: int
    rev_mode: int
    reac: List[Tuple[int, int]]            # (species, nu')
    prod: List[Tuple[int, int]]            # (species, nu'')
    arr: Tuple[float, float, float] = (0.0, 0.0, 0.0)      # A, beta, Ta
    rev_arr: Optional[Tuple[float, float, float]] = None
    tb_mode: int = 0
    tb_species: int = -1
    eff: List[Tuple[int, float]] = dataclasses.field(default_factory=list)
    k0: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    kinf: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    ftype: int = F_LINDEMANN
    fparams: Tuple[float, ...] = (0.0, 0.0, 0.0, 0.0, 0.0)
    troe_has_T2: int = 0
    plog: List[Tuple[float, float, float, float]] = dataclasses.field(default_factory=list)
    cheb_shape: Tuple[int, int] = (0, 0)
    cheb_range: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)
    cheb_eta: Optional[np.ndarray] = None


@dataclasses.dataclass
class Model:
    n_elements: int
    species: List[Species]
    reactions: List[Reaction]
    name: str = "synthetic"
    seed: int = 0

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return len(self.reactions)


# ----------------------------------------------------------------------------------------------
# serialisation


def to_bytes(model: Model) -> bytes:
    """Serialise ``model`` to the binary model format described in the module docstring."""
    out = bytearray()
    out += MAGIC
    out += struct.pack("<IIII", VERSION, model.n_elements, model.n_species, model.n_reactions)
    for sp in model.species:
        out += struct.pack("<4d", sp.W, sp.T_low, sp.T_mid, sp.T_high)
        out += struct.pack("<7d", *[float(x) for x in sp.a_low])
        out += struct.pack("<7d", *[float(x) for x in sp.a_high])
        out += struct.pack("<%di" % model.n_elements, *[int(x) for x in sp.elem])
    for r in model.reactions:
        out += struct.pack("<ii", r.kind, r.rev_mode)
        out += struct.pack("<i", len(r.reac))
        for s, nu in r.reac:
            out += struct.pack("<ii", s, nu)
        out += struct.pack("<i", len(r.prod))
        for s, nu in r.prod:
            out += struct.pack("<ii", s, nu)
        out += struct.pack("<3d", *r.arr)
        if r.rev_mode == REV_EXPLICIT:
            out += struct.pack("<3d", *r.rev_arr)
        if r.kind in (KIND_THIRD_BODY, KIND_FALLOFF, KIND_CHEM):
            out += struct.pack("<iii", r.tb_mode, r.tb_species, len(r.eff))
            for s, a in r.eff:
                out += struct.pack("<id", s, a)
        if r.kind in (KIND_FALLOFF, KIND_CHEM):
            out += struct.pack("<6d", *r.k0, *r.kinf)
            out += struct.pack("<i", r.ftype)
            fp = list(r.fparams) + [0.0] * (5 - len(r.fparams))
            out += struct.pack("<5d", *fp[:5])
            out += struct.pack("<i", r.troe_has_T2)
        if r.kind == KIND_PLOG:
            out += struct.pack("<i", len(r.plog))
            for p, A, b, Ta in r.plog:
                out += struct.pack("<4d", p, A, b, Ta)
        if r.kind == KIND_CHEB:
            nt, npr = r.cheb_shape
            out += struct.pack("<ii", nt, npr)
            out += struct.pack("<4d", *r.cheb_range)
            out += struct.pack("<%dd" % (nt * npr), *[float(x) for x in np.asarray(r.cheb_eta).ravel()])
    return bytes(out)


# ----------------------------------------------------------------------------------------------
# thermodynamic data: two-range NASA7 fits of a smooth random heat-capacity curve


def _fit_nasa7(rng: np.random.Generator, T_low: float, T_mid: float, T_high: float
               ) -> Tuple[np.ndarray, np.ndarray]:
    """Fit two quartic cp/R polynomials to a smooth random sigmoid cp/R curve in [3, 8].

    Both ranges are fitted jointly with cp/R and d(cp/R)/dT equal at T_mid; the enthalpy and
    entropy integration constants (a5, a6) are then set from a drawn formation enthalpy and
    standard entropy at 298.15 K and carried across T_mid so that H and S are continuous.
    Integration uses numpy's polynomial antiderivatives.
    """
    c_lo = rng.uniform(3.0, 5.0)
    c_hi = rng.uniform(c_lo + 0.5, 8.0)
    Tc = rng.uniform(500.0, 2000.0)
    width = rng.uniform(300.0, 1000.0)

    def cp_curve(T):
        return c_lo + (c_hi - c_lo) / (1.0 + np.exp(-(T - Tc) / width))

    s = 1000.0                                   # fit in tau = T / 1000 for conditioning
    Tl = np.linspace(T_low, T_mid, 60)
    Th = np.linspace(T_mid, T_high, 120)
    Vl = np.vander(Tl / s, 5, increasing=True)
    Vh = np.vander(Th / s, 5, increasing=True)
    M = np.zeros((len(Tl) + len(Th), 10))
    M[:len(Tl), :5] = Vl
    M[len(Tl):, 5:] = Vh
    y = np.concatenate([cp_curve(Tl), cp_curve(Th)])
    tm = T_mid / s
    v0 = np.array([1.0, tm, tm ** 2, tm ** 3, tm ** 4])
    v1 = np.array([0.0, 1.0, 2 * tm, 3 * tm ** 2, 4 * tm ** 3])
    Cst = np.zeros((2, 10))
    Cst[0, :5], Cst[0, 5:] = v0, -v0
    Cst[1, :5], Cst[1, 5:] = v1, -v1
    K = np.zeros((12, 12))
    K[:10, :10] = 2.0 * M.T @ M
    K[:10, 10:] = Cst.T
    K[10:, :10] = Cst
    rhs = np.concatenate([2.0 * M.T @ y, np.zeros(2)])
    sol = np.linalg.solve(K, rhs)
    scale = np.array([1.0, s, s ** 2, s ** 3, s ** 4])
    b_lo = sol[:5] / scale
    b_hi = sol[5:10] / scale

    h298 = rng.uniform(-1.0e4, 1.0e4)            # H/R at 298.15 K, in K
    s298 = rng.uniform(20.0, 40.0)               # S/R at 298.15 K
    P = np.polynomial.polynomial
    Hl = P.polyint(b_lo)                         # antiderivative of cp/R: H/R without constant
    Hh = P.polyint(b_hi)
    Sl = P.polyint(b_lo[1:])                     # antiderivative of (cp/R - a0)/T
    Sh = P.polyint(b_hi[1:])
    a5_lo = h298 - P.polyval(298.15, Hl)
    a5_hi = a5_lo + P.polyval(T_mid, Hl) - P.polyval(T_mid, Hh)
    a6_lo = s298 - (b_lo[0] * math.log(298.15) + P.polyval(298.15, Sl))
    a6_hi = a6_lo + (b_lo[0] - b_hi[0]) * math.log(T_mid) + P.polyval(T_mid, Sl) - P.polyval(T_mid, Sh)
    a_low = np.concatenate([b_lo, [a5_lo, a6_lo]])
    a_high = np.concatenate([b_hi, [a5_hi, a6_hi]])
    return a_low, a_high


# ----------------------------------------------------------------------------------------------
# species and element-balanced reactions


def _species_vectors(rng: np.random.Generator, n_species: int, n_elements: int) -> List[Tuple[int, ...]]:
    """Distinct element-count vectors: all atoms and diatomics first, then random small molecules."""
    base: List[Tuple[int, ...]] = []
    for e in range(n_elements):
        v = [0] * n_elements
        v[e] = 1
        base.append(tuple(v))
    for e in range(n_elements):
        for f in range(e, n_elements):
            v = [0] * n_elements
            v[e] += 1
            v[f] += 1
            base.append(tuple(v))
    if n_species <= len(base):
        # keep every atom, then a random subset of the diatomics
        atoms, di = base[:n_elements], base[n_elements:]
        idx = rng.permutation(len(di))[: n_species - n_elements]
        vecs = atoms + [di[i] for i in sorted(idx)]
    else:
        vecs = list(base)
        seen = set(vecs)
        maxc = 2 if n_species <= 64 else 3
        tries = 0
        while len(vecs) < n_species:
            tries += 1
            if tries > 10_000_000:
                raise RuntimeError("could not draw enough distinct species")
            v = tuple(int(x) for x in rng.integers(0, maxc + 1, size=n_elements))
            if sum(v) < 3 or sum(v) > 8 or v in seen:
                continue
            seen.add(v)
            vecs.append(v)
    order = rng.permutation(len(vecs))
    return [vecs[i] for i in order]


class _Balancer:
    """Finds element-balanced product multisets for a drawn reactant multiset."""

    def __init__(self, vecs: Sequence[Tuple[int, ...]]):
        self.vecs = [np.array(v, dtype=np.int64) for v in vecs]
        self.n = len(vecs)
        self.singles: Dict[Tuple[int, ...], List[int]] = {}
        for i, v in enumerate(vecs):
            self.singles.setdefault(tuple(v), []).append(i)
        self.pairs: Dict[Tuple[int, ...], List[Tuple[int, int]]] = {}
        for i in range(self.n):
            for j in range(i, self.n):
                key = tuple(int(x) for x in self.vecs[i] + self.vecs[j])
                self.pairs.setdefault(key, []).append((i, j))

    def products(self, rng, total: np.ndarray, n_prod: int) -> List[Tuple[int, ...]]:
        key = tuple(int(x) for x in total)
        if n_prod == 1:
            return [(i,) for i in self.singles.get(key, [])]
        if n_prod == 2:
            return list(self.pairs.get(key, []))
        out = []
        cand = rng.permutation(self.n)[:64]
        for c in cand:
            rest = total - self.vecs[c]
            if (rest < 0).any():
                continue
            for (a, b) in self.pairs.get(tuple(int(x) for x in rest), []):
                out.append(tuple(sorted((int(c), a, b))))
        return out


def _to_stoich(ms: Sequence[int]) -> List[Tuple[int, int]]:
    d: Dict[int, int] = {}
    for s in ms:
        d[int(s)] = d.get(int(s), 0) + 1
    return sorted(d.items())


def _draw_balanced(rng, bal: _Balancer, n_reac: int, n_prod: int, allow_repeat: bool = True
                   ) -> Optional[Tuple[List[Tuple[int, int]], List[Tuple[int, int]]]]:
    for _ in range(400):
        reac = [int(x) for x in rng.integers(0, bal.n, size=n_reac)]
        if not allow_repeat and len(set(reac)) < len(reac):
            continue
        total = sum(bal.vecs[s] for s in reac)
        cands = bal.products(rng, total, n_prod)
        rs = tuple(sorted(reac))
        cands = [c for c in cands if tuple(sorted(c)) != rs and not (set(c) & set(reac))]
        if not cands:
            continue
        prod = cands[int(rng.integers(0, len(cands)))]
        return _to_stoich(reac), _to_stoich(prod)
    return None


# ----------------------------------------------------------------------------------------------
# rate parameters


def _arrhenius(rng, order: int) -> Tuple[float, float, float]:
    """A log-uniform 1e6..1e14 (cm^3-mol-s), beta U(-2, 2), Ea U(0, 50) kcal/mol -> SI."""
    A_cgs = 10.0 ** rng.uniform(6.0, 14.0)
    A = A_cgs * (1.0e-6) ** (order - 1)
    beta = rng.uniform(-2.0, 2.0)
    Ea = rng.uniform(0.0, 50.0) * 1000.0 * CAL            # J/mol
    return (A, beta, Ea / R_GAS)


def _order(st: List[Tuple[int, int]]) -> int:
    return sum(nu for _, nu in st)


# typical third-body concentration p/(R T) at 10 atm and 1500 K (mol/m^3), for sizing k0 vs kinf
_M_TYP = 10.0 * P_ATM / (R_GAS * 1500.0)
_T_TYP = 1500.0


def _falloff_pair(rng, order_inf: int, chem: bool):
    """Low/high-pressure Arrhenius pair with log10 P_r near U(-4, 4) at 10 atm, 1500 K."""
    target = rng.uniform(-4.0, 4.0)
    if not chem:
        kinf = _arrhenius(rng, order_inf)
        beta0 = rng.uniform(-2.0, 2.0)
        Ta0 = rng.uniform(0.0, 30.0) * 1000.0 * CAL / R_GAS
        # choose A0 so that log10(k0/kinf * M) ~ target at the typical state
        lg = (target - math.log10(_M_TYP) + math.log10(kinf[0])
              + (kinf[1] - beta0) * math.log10(_T_TYP) - (kinf[2] - Ta0) / (_T_TYP * math.log(10.0)))
        k0 = (10.0 ** lg, beta0, Ta0)
    else:
        k0 = _arrhenius(rng, order_inf + 1)
        betai = rng.uniform(-2.0, 2.0)
        Tai = rng.uniform(0.0, 30.0) * 1000.0 * CAL / R_GAS
        lg = (math.log10(k0[0]) + math.log10(_M_TYP) - target
              + (k0[1] - betai) * math.log10(_T_TYP) - (k0[2] - Tai) / (_T_TYP * math.log(10.0)))
        kinf = (10.0 ** lg, betai, Tai)
    return k0, kinf


def _efficiencies(rng, n_species: int, exclude: Sequence[int]) -> List[Tuple[int, float]]:
    k = int(rng.integers(3, 7))
    pool = [s for s in range(n_species) if s not in exclude]
    k = min(k, len(pool))
    chosen = sorted(int(x) for x in rng.choice(pool, size=k, replace=False))
    out = []
    for s in chosen:
        a = float(rng.uniform(0.0, 6.0))
        if abs(a - 1.0) < 1e-3:
            a = 1.5
        out.append((s, a))
    return out


# ----------------------------------------------------------------------------------------------
# model generation

# reaction type mix: fraction of reactions per (kind, ftype) label
MIX_SMALL = {"elementary": 20 / 27, "third_body": 5 / 27, "troe": 2 / 27}
MIX_MEDIUM = {"elementary": 0.70, "third_body": 0.15, "troe": 0.08, "lindemann": 0.04, "sri": 0.03}
MIX_LARGE = {"elementary": 0.67, "third_body": 0.15, "troe": 0.08, "lindemann": 0.04, "sri": 0.03,
             "plog": 0.02, "cheb": 0.01}


def _counts(n: int, mix: Dict[str, float]) -> Dict[str, int]:
    raw = {k: v * n for k, v in mix.items()}
    cnt = {k: int(math.floor(v)) for k, v in raw.items()}
    rest = n - sum(cnt.values())
    for k in sorted(raw, key=lambda k: raw[k] - cnt[k], reverse=True)[:rest]:
        cnt[k] += 1
    return cnt


def generate_model(n_species: int, n_reactions: int, n_elements: int, mix: Dict[str, float],
                   seed: int, rev_modes: Sequence[int] = (REV_KC,), chem_fraction: float = 0.1,
                   species_tb_fraction: float = 0.1, eff_fraction: float = 0.7,
                   name: str = "synthetic") -> Model:
    """Draw an element-balanced synthetic model.

    ``mix`` maps labels (elementary, third_body, troe, lindemann, sri, plog, cheb) to fractions.
    Falloff labels become chemically activated with probability ``chem_fraction``; third-body and
    falloff reactions use a single third-body species with probability ``species_tb_fraction``
    and otherwise carry 3-6 non-unity efficiencies with probability ``eff_fraction``.
    ``rev_modes`` lists the reversibility modes drawn uniformly per reaction.
    """
    rng = np.random.default_rng(seed)
    vecs = _species_vectors(rng, n_species, n_elements)
    species = []
    for v in vecs:
        W = float(sum(c * _ELEMENT_MASS[e] for e, c in enumerate(v)))
        a_low, a_high = _fit_nasa7(rng, 300.0, 1000.0, 3000.0)
        species.append(Species(W, 300.0, 1000.0, 3000.0, a_low, a_high, np.array(v, dtype=np.int32)))
    bal = _Balancer(vecs)

    labels: List[str] = []
    for k, c in _counts(n_reactions, mix).items():
        labels += [k] * c
    labels = [labels[i] for i in rng.permutation(len(labels))]

    reactions: List[Reaction] = []
    for lab in labels:
        rev = int(rev_modes[int(rng.integers(0, len(rev_modes)))])
        if lab == "elementary":
            shape = [(2, 2)] * 6 + [(2, 1), (1, 2), (3, 2), (2, 3)]
        elif lab == "third_body":
            shape = [(2, 1), (1, 2)]
        elif lab in ("troe", "lindemann", "sri"):
            shape = [(1, 2), (2, 1)]
        else:
            shape = [(2, 2), (1, 2)]
        drawn = None
        for _ in range(50):
            nr, npd = shape[int(rng.integers(0, len(shape)))]
            drawn = _draw_balanced(rng, bal, nr, npd)
            if drawn is not None:
                break
        if drawn is None:
            raise RuntimeError("could not draw a balanced reaction for %s" % lab)
        reac, prod = drawn
        r = Reaction(kind=KIND_ELEMENTARY, rev_mode=rev, reac=reac, prod=prod)
        order = _order(reac)
        if lab == "elementary":
            r.arr = _arrhenius(rng, order)
        elif lab == "third_body":
            r.kind = KIND_THIRD_BODY
            r.arr = _arrhenius(rng, order + 1)
        elif lab in ("troe", "lindemann", "sri"):
            chem = rng.uniform() < chem_fraction
            r.kind = KIND_CHEM if chem else KIND_FALLOFF
            r.k0, r.kinf = _falloff_pair(rng, order if not chem else order - 1, chem)
            if lab == "lindemann":
                r.ftype = F_LINDEMANN
            elif lab == "troe":
                r.ftype = F_TROE
                has2 = int(rng.uniform() < 0.6)
                r.fparams = (rng.uniform(0.1, 0.9), rng.uniform(50.0, 500.0), rng.uniform(1000.0, 5000.0),
                             rng.uniform(2000.0, 8000.0) if has2 else 0.0, 0.0)
                r.troe_has_T2 = has2
            else:
                r.ftype = F_SRI
                r.fparams = (rng.uniform(0.1, 2.0), rng.uniform(100.0, 1000.0), rng.uniform(200.0, 2000.0),
                             rng.uniform(0.5, 1.5), rng.uniform(-0.5, 0.5))
        elif lab == "plog":
            r.kind = KIND_PLOG
            base = _arrhenius(rng, order)
            ps = np.sort(np.concatenate([[1.0, 100.0], 10.0 ** rng.uniform(0.15, 1.85, size=2)])) * P_ATM
            r.plog = []
            for p in ps:
                A = base[0] * 10.0 ** rng.uniform(-1.0, 1.0)
                b = base[1] + rng.uniform(-0.3, 0.3)
                Ta = max(0.0, base[2] + rng.uniform(-1000.0, 1000.0))
                r.plog.append((float(p), float(A), float(b), float(Ta)))
        elif lab == "cheb":
            r.kind = KIND_CHEB
            nt, npr = 7, 3
            eta = rng.normal(0.0, 1.0, size=(nt, npr)) * (0.4 / (1.0 + np.add.outer(np.arange(nt), np.arange(npr))))
            eta[0, 0] = rng.uniform(6.0, 14.0) - 6.0 * (order - 1)
            r.cheb_shape = (nt, npr)
            r.cheb_range = (300.0, 3000.0, 0.1 * P_ATM, 100.0 * P_ATM)
            r.cheb_eta = eta
        if r.kind in (KIND_PLOG, KIND_CHEB) and r.rev_mode == REV_EXPLICIT:
            r.rev_mode = REV_KC
        if r.rev_mode == REV_EXPLICIT:
            r.rev_arr = _arrhenius(rng, _order(prod) + (1 if r.kind == KIND_THIRD_BODY else 0))
        if r.kind in (KIND_THIRD_BODY, KIND_FALLOFF, KIND_CHEM):
            if rng.uniform() < species_tb_fraction:
                r.tb_mode = TB_SPECIES
                r.tb_species = int(rng.integers(0, n_species))
            else:
                r.tb_mode = TB_MIXTURE
                if rng.uniform() < eff_fraction:
                    r.eff = _efficiencies(rng, n_species, [])
        reactions.append(r)
    return Model(n_elements=n_elements, species=species, reactions=reactions, name=name, seed=seed)


def generate_states(n_species: int, n_states: int, seed: int, T_range=(800.0, 2500.0),
                    P_range_atm=(1.0, 50.0), alpha: float = 0.5):
    """T uniform, P log-uniform (Pa), Y ~ Dirichlet(alpha) over all species. Returns (T, P, Y)."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(T_range[0], T_range[1], size=n_states)
    P = P_ATM * 10.0 ** rng.uniform(math.log10(P_range_atm[0]), math.log10(P_range_atm[1]), size=n_states)
    Y = rng.dirichlet(np.full(n_species, alpha), size=n_states)
    return T.astype(np.float64), P.astype(np.float64), np.ascontiguousarray(Y, dtype=np.float64)


def generate_conc_states(n_species: int, n_states: int, seed: int, T_range=(800.0, 2500.0),
                         P_range_atm=(1.0, 50.0), alpha: float = 0.5, V_range=(1e-6, 1e-2)):
    """States of the molar-concentration basis: T uniform, P log-uniform (Pa), V log-uniform (m^3),
    mole fractions x ~ Dirichlet(alpha) over all species and n_k = x_k P V / (R T) for the first
    N - 1 species (the last one is implied). Returns (T, P, V, n) with n of shape (n_states, N-1)."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(T_range[0], T_range[1], size=n_states)
    P = P_ATM * 10.0 ** rng.uniform(math.log10(P_range_atm[0]), math.log10(P_range_atm[1]), size=n_states)
    V = 10.0 ** rng.uniform(math.log10(V_range[0]), math.log10(V_range[1]), size=n_states)
    x = rng.dirichlet(np.full(n_species, alpha), size=n_states)
    ntot = P * V / (R_GAS * T)
    nmol = x[:, : n_species - 1] * ntot[:, None]
    return (T.astype(np.float64), P.astype(np.float64), V.astype(np.float64),
            np.ascontiguousarray(nmol, dtype=np.float64))


def config_conc_states(cfg: int, n_states: Optional[int] = None, seed_offset: int = 2000):
    c = CONFIGS[cfg]
    n = c["n_states"] if n_states is None else n_states
    return generate_conc_states(c["n_species"], n, seed=SEED_BASE + cfg + seed_offset)


# ----------------------------------------------------------------------------------------------
# the benchmark workloads (synthetic stand-ins for the paper's four kinetic models, Table T:models)

SEED_BASE = 160503262

CONFIGS = {
    0: dict(name="small-13sp-27rxn", n_species=13, n_reactions=27, n_elements=4, mix=MIX_SMALL,
            n_states=1024, chem_fraction=0.0),
    1: dict(name="medium-53sp-325rxn", n_species=53, n_reactions=325, n_elements=5, mix=MIX_MEDIUM,
            n_states=65536, chem_fraction=0.1),
    2: dict(name="large-111sp-784rxn", n_species=111, n_reactions=784, n_elements=5, mix=MIX_LARGE,
            n_states=262144, chem_fraction=0.1),
    3: dict(name="xl-360sp-2172rxn", n_species=360, n_reactions=2172, n_elements=5, mix=MIX_LARGE,
            n_states=16384, chem_fraction=0.1),
}


def config_model(cfg: int) -> Model:
    c = CONFIGS[cfg]
    return generate_model(c["n_species"], c["n_reactions"], c["n_elements"], c["mix"],
                          seed=SEED_BASE + cfg, chem_fraction=c["chem_fraction"], name=c["name"])


def config_states(cfg: int, n_states: Optional[int] = None, seed_offset: int = 1000):
    c = CONFIGS[cfg]
    n = c["n_states"] if n_states is None else n_states
    return generate_states(c["n_species"], n, seed=SEED_BASE + cfg + seed_offset)
