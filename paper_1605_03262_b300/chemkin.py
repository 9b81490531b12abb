"""Chemkin-format mechanism reader and writer.

:func:`parse` reads a Chemkin-II mechanism (ELEMENTS, SPECIES, THERMO and REACTIONS blocks, thermo
either inline or from a separate file) into the in-memory model of :mod:`synth`, which
``synth.to_bytes`` turns into the library's binary model format. :func:`write` does the reverse,
so that any model can be exported and read back.

Supported, with the paper's rate formulations (Section 2.3): Arrhenius reactions, reversible
(``<=>`` or ``=``) through the equilibrium constant, irreversible (``=>``) or with an explicit
``REV``; third-body reactions (``+M``) with ``name/alpha/`` efficiencies; pressure-dependent
reactions ``(+M)`` or ``(+species)`` with ``LOW`` (falloff) or ``HIGH`` (chemically activated) and
Lindemann, ``TROE`` (3 or 4 parameters) or ``SRI`` (3 or 5 parameters) blending; ``PLOG``; and
Chebyshev (``TCHEB``/``PCHEB``/``CHEB``). ``DUPLICATE`` reactions are kept as separate reactions.
Other auxiliary keywords (FORD, RORD, LT, TDEP, ...) and non-integer stoichiometric coefficients
raise :class:`ChemkinError`.

Units: the REACTIONS line may give the activation-energy unit (CAL/MOLE default, KCAL/MOLE,
JOULES/MOLE, KJOULES/MOLE, KELVINS, EVOLTS) and the quantity unit (MOLES default, MOLECULES).
Pre-exponential factors are in cm^3, mol and s with the reaction order of their rate expression
(the reactant coefficients, plus one for a third body in +M reactions and in k_0 of a falloff
reaction, k_inf of a chemically activated one); PLOG pressures are in atm; Chebyshev coefficients
give log10 k in those units. The model stores SI units (A in (m^3/mol)^(order-1)/s, activation
temperatures in K, pressures in Pa).
"""
from __future__ import annotations

import math
import re
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import synth
from .synth import (F_LINDEMANN, F_SRI, F_TROE, KIND_CHEB, KIND_CHEM, KIND_ELEMENTARY, KIND_FALLOFF,
                    KIND_PLOG, KIND_THIRD_BODY, P_ATM, R_GAS, REV_EXPLICIT, REV_IRREVERSIBLE, REV_KC,
                    TB_MIXTURE, TB_SPECIES, Model, Reaction, Species)

__all__ = ["parse", "parse_file", "write", "ChemkinError", "ATOMIC_WEIGHTS"]

# Standard atomic weights (g/mol) of the elements a combustion mechanism uses; an ELEMENTS entry
# may override one with "X/weight/".
ATOMIC_WEIGHTS = {
    "H": 1.00794, "D": 2.014102, "T": 3.016049, "C": 12.0107, "O": 15.9994, "N": 14.0067,
    "AR": 39.948, "HE": 4.002602, "NE": 20.1797, "KR": 83.798, "XE": 131.293, "S": 32.065,
    "CL": 35.453, "F": 18.9984032, "BR": 79.904, "I": 126.90447, "SI": 28.0855, "P": 30.973762,
    "NA": 22.98977, "K": 39.0983, "FE": 55.845, "E": 5.4858e-4,
}

N_AVOGADRO = 6.02214076e23
EV = 1.602176634e-19           # J
_EA_UNITS = {"CAL/MOLE": synth.CAL / R_GAS, "KCAL/MOLE": 1e3 * synth.CAL / R_GAS, "JOULES/MOLE": 1.0 / R_GAS,
             "KJOULES/MOLE": 1e3 / R_GAS, "KELVINS": 1.0, "EVOLTS": EV * N_AVOGADRO / R_GAS}


class ChemkinError(ValueError):
    """A mechanism the reader cannot represent, with the line it came from."""


# ----------------------------------------------------------------------------------------------
# reading

def _strip(line: str) -> str:
    i = line.find("!")
    return (line if i < 0 else line[:i]).rstrip()


def _blocks(text: str):
    """Split the text into (keyword, header tokens, body lines) blocks; END closes a block."""
    blocks, cur = [], None
    for raw in text.splitlines():
        line = _strip(raw)
        if not line.strip():
            continue
        tok = line.split()
        key = tok[0].upper()
        key4 = key[:4]
        if cur is None or cur[0] in ("ELEM", "SPEC"):
            if key4 in ("ELEM", "SPEC", "THER", "REAC"):
                if cur is not None:
                    blocks.append(cur)
                cur = (key4, tok[1:], [])
                continue
        if cur is not None and key == "END":
            blocks.append(cur)
            cur = None
            continue
        if cur is None:
            if key4 in ("THER", "REAC"):
                cur = (key4, tok[1:], [])
                continue
            raise ChemkinError("text outside a block: %r" % raw)
        cur[2].append(raw if cur[0] == "THER" else line)
    if cur is not None:
        blocks.append(cur)
    return blocks


def _parse_thermo(lines: List[str], header: Sequence[str], names: Optional[set]) -> Dict[str, dict]:
    """NASA7 entries in the fixed-column format: 4 lines per species."""
    out = {}
    i = 0
    defaults = None
    body = [ln for ln in lines if ln.strip()]
    if body and not body[0].rstrip().endswith("1") and len(body[0].split()) in (3, 4):
        try:
            defaults = [float(x) for x in body[0].split()[:3]]
            body = body[1:]
        except ValueError:
            defaults = None
    while i < len(body):
        l1 = body[i].ljust(80)
        if i + 3 >= len(body):
            raise ChemkinError("incomplete thermo entry: %r" % body[i])
        name = l1[:18].split()[0] if l1[:18].split() else ""
        comp = {}
        for k in range(4):
            el, cnt = l1[24 + 5 * k: 26 + 5 * k].strip(), l1[26 + 5 * k: 29 + 5 * k].strip()
            if el and el != "0" and cnt:
                n = int(float(cnt))
                if n:
                    comp[el.upper()] = comp.get(el.upper(), 0) + n
        extra = l1[73:78]
        if extra.strip():
            el, cnt = extra[:2].strip(), extra[2:].strip()
            if el and cnt and int(float(cnt)):
                comp[el.upper()] = comp.get(el.upper(), 0) + int(float(cnt))
        try:
            T_low, T_high = float(l1[45:55]), float(l1[55:65])
            T_mid = float(l1[65:73]) if l1[65:73].strip() else (defaults[1] if defaults else 1000.0)
        except ValueError:
            raise ChemkinError("bad temperature ranges in thermo entry of %s" % name)
        coeffs = []
        for ln in body[i + 1: i + 4]:
            ln = ln.ljust(80)
            for k in range(5):
                f = ln[15 * k: 15 * (k + 1)].strip()
                if f:
                    coeffs.append(float(f.replace("D", "E").replace("d", "e")))
        if len(coeffs) < 14:
            raise ChemkinError("thermo entry of %s has %d coefficients, expected 14" % (name, len(coeffs)))
        high, low = coeffs[:7], coeffs[7:14]
        if names is None or name in names:
            out.setdefault(name, dict(comp=comp, T_low=T_low, T_mid=T_mid, T_high=T_high,
                                      a_low=np.array(low), a_high=np.array(high)))
        i += 4
    return out


_NUM = r"[+-]?(?:\d+\.?\d*|\.\d+)(?:[eEdD][+-]?\d+)?"


def _float(s: str) -> float:
    return float(s.replace("D", "E").replace("d", "e"))


def _side(text: str, species: Dict[str, int], lineno: int):
    """Species and coefficients of one side, its third-body marker and pressure-dependence marker."""
    third = None           # "M" or species name for +M / (+X)
    falloff = False
    m = re.search(r"\(\+\s*([^)]+?)\s*\)", text)
    if m:
        falloff = True
        third = m.group(1).strip()
        text = text[:m.start()] + text[m.end():]
    terms, out = [t.strip() for t in text.split("+")], {}
    for t in terms:
        if not t:
            continue
        if t.upper() == "M":
            if third not in (None, "M"):
                raise ChemkinError("line %d: two third bodies" % lineno)
            third = "M"
            continue
        if t in species:
            name, nu = t, 1
        else:
            name = None
            digits = re.match(r"^\d+", t)
            for i in range(1, (len(digits.group(0)) if digits else 0) + 1):   # "21-C4H8" may be 2 x "1-C4H8"
                if t[i:].strip() in species:
                    name, nu = t[i:].strip(), int(t[:i])
                    break
            if name is None:
                if re.match(r"^\d*\.\d*\s*\S", t):
                    raise ChemkinError("line %d: non-integer stoichiometric coefficient in %r" % (lineno, t))
                raise ChemkinError("line %d: unknown species %r" % (lineno, t))
        out[species[name]] = out.get(species[name], 0) + nu
    return out, third, falloff


def _order(side: Dict[int, int]) -> int:
    return sum(side.values())


def _arr(A: float, beta: float, Ea: float, order: int, ea_to_K: float, molecules: bool):
    """Arrhenius parameters to SI: A in (m^3/mol)^(order-1)/s, activation temperature in K."""
    if molecules:
        A = A * N_AVOGADRO ** (order - 1)
    return (A * 1e-6 ** (order - 1), beta, Ea * ea_to_K)


def parse(text: str, thermo_text: Optional[str] = None, name: str = "chemkin") -> Model:
    """Parse a Chemkin mechanism (and optionally a separate thermo file) into a synth.Model."""
    blocks = _blocks(text)
    elements: List[str] = []
    weights: Dict[str, float] = {}
    species_names: List[str] = []
    thermo_lines, thermo_header = [], []
    reac_lines, reac_header = [], []
    for key, header, body in blocks:
        if key == "ELEM":
            for tok in " ".join(header + body).split():
                mm = re.match(r"^([A-Za-z][A-Za-z0-9]*)(?:/\s*(" + _NUM + r")\s*/)?$", tok)
                if not mm:
                    raise ChemkinError("bad element entry %r" % tok)
                el = mm.group(1).upper()
                elements.append(el)
                if mm.group(2):
                    weights[el] = _float(mm.group(2))
        elif key == "SPEC":
            species_names += " ".join(header + body).split()
        elif key == "THER":
            thermo_lines += body
            thermo_header = header
        elif key == "REAC":
            reac_lines += body
            reac_header = header
    if len(set(species_names)) != len(species_names):
        raise ChemkinError("duplicate species names")
    thermo = {}
    if thermo_text is not None:
        for key, header, body in _blocks(thermo_text):
            if key == "THER":
                thermo.update(_parse_thermo(body, header, set(species_names)))
    thermo.update(_parse_thermo(thermo_lines, thermo_header, set(species_names)))
    missing = [s for s in species_names if s not in thermo]
    if missing:
        raise ChemkinError("no thermo data for %s" % ", ".join(missing))
    el_index = {e: i for i, e in enumerate(elements)}
    sp = []
    for s in species_names:
        t = thermo[s]
        elem = np.zeros(len(elements), dtype=np.int64)
        W = 0.0
        for e, n in t["comp"].items():
            if e not in el_index:
                raise ChemkinError("species %s uses undeclared element %s" % (s, e))
            elem[el_index[e]] = n
            w = weights.get(e, ATOMIC_WEIGHTS.get(e))
            if w is None:
                raise ChemkinError("no atomic weight for element %s" % e)
            W += n * w
        sp.append(Species(W=W * 1e-3, T_low=t["T_low"], T_mid=t["T_mid"], T_high=t["T_high"],
                          a_low=t["a_low"], a_high=t["a_high"], elem=elem))
    sidx = {s: i for i, s in enumerate(species_names)}
    ea_to_K, molecules = _EA_UNITS["CAL/MOLE"], False
    for tok in reac_header:
        u = tok.upper()
        if u in _EA_UNITS:
            ea_to_K = _EA_UNITS[u]
        elif u == "MOLECULES":
            molecules = True
        elif u != "MOLES":
            raise ChemkinError("unsupported REACTIONS unit %s" % tok)
    reactions = _parse_reactions(reac_lines, sidx, ea_to_K, molecules)
    return Model(n_elements=len(elements), species=sp, reactions=reactions, name=name)


_REACTION_LINE = re.compile(r"^(?P<eq>.*?(?:<=>|=>|=).*?)\s+(?P<A>" + _NUM + r")\s+(?P<b>" + _NUM + r")\s+(?P<E>"
                            + _NUM + r")\s*$")


def _parse_reactions(lines: List[str], sidx: Dict[str, int], ea_to_K: float, molecules: bool) -> List[Reaction]:
    """Reaction lines and their auxiliary lines into Reactions (SI units)."""
    raw = []                                                   # (lineno, equation, A, b, E, aux tokens)
    for n, line in enumerate(lines, 1):
        m = _REACTION_LINE.match(line.strip())
        if m and ("=" in m.group("eq")):
            raw.append([n, m.group("eq"), _float(m.group("A")), _float(m.group("b")), _float(m.group("E")), []])
        else:
            if not raw:
                raise ChemkinError("line %d: auxiliary data before the first reaction: %r" % (n, line))
            raw[-1][5].append((n, line))
    out = []
    for n, eq, A, b, E, aux in raw:
        if "<=>" in eq:
            lhs, rhs, rev = *eq.split("<=>", 1), True
        elif "=>" in eq:
            lhs, rhs, rev = *eq.split("=>", 1), False
        else:
            lhs, rhs, rev = *eq.split("=", 1), True
        reac, tb_l, fo_l = _side(lhs, sidx, n)
        prod, tb_r, fo_r = _side(rhs, sidx, n)
        if (tb_l is None) != (tb_r is None) or fo_l != fo_r or (tb_l != tb_r):
            raise ChemkinError("line %d: third body on one side only" % n)
        third, pdep = tb_l, fo_l
        kw = _aux(aux, sidx, n)
        r = Reaction(kind=KIND_ELEMENTARY, rev_mode=REV_KC if rev else REV_IRREVERSIBLE,
                     reac=sorted(reac.items()), prod=sorted(prod.items()))
        order = _order(reac)
        if "REV" in kw:
            if not rev:
                raise ChemkinError("line %d: REV on an irreversible reaction" % n)
            r.rev_mode = REV_EXPLICIT
            Ar, br, Er = kw["REV"]
            r.rev_arr = _arr(Ar, br, Er, _order(prod) + (1 if third is not None and not pdep else 0), ea_to_K,
                             molecules)
        if third is not None:
            if third == "M":
                r.tb_mode = TB_MIXTURE
                r.eff = [(s, a) for s, a in kw.get("EFF", []) if a != 1.0]
            else:
                if third not in sidx:
                    raise ChemkinError("line %d: unknown third body %s" % (n, third))
                r.tb_mode, r.tb_species = TB_SPECIES, sidx[third]
                if kw.get("EFF"):
                    raise ChemkinError("line %d: efficiencies with a specific third body" % n)
        if pdep:
            if "LOW" in kw and "HIGH" in kw:
                raise ChemkinError("line %d: both LOW and HIGH" % n)
            if "LOW" in kw:
                r.kind = KIND_FALLOFF
                r.kinf = _arr(A, b, E, order, ea_to_K, molecules)
                r.k0 = _arr(*kw["LOW"], order + 1, ea_to_K, molecules)
            elif "HIGH" in kw:
                r.kind = KIND_CHEM
                r.k0 = _arr(A, b, E, order + 1, ea_to_K, molecules)
                r.kinf = _arr(*kw["HIGH"], order, ea_to_K, molecules)
            else:
                raise ChemkinError("line %d: (+M) reaction without LOW or HIGH" % n)
            if "TROE" in kw:
                p = kw["TROE"]
                if len(p) not in (3, 4):
                    raise ChemkinError("line %d: TROE takes 3 or 4 parameters" % n)
                r.ftype, r.troe_has_T2 = F_TROE, 1 if len(p) == 4 else 0
                r.fparams = tuple(list(p) + [0.0] * (5 - len(p)))
            elif "SRI" in kw:
                p = kw["SRI"]
                if len(p) not in (3, 5):
                    raise ChemkinError("line %d: SRI takes 3 or 5 parameters" % n)
                r.ftype = F_SRI
                r.fparams = tuple(p) if len(p) == 5 else (p[0], p[1], p[2], 1.0, 0.0)
            else:
                r.ftype = F_LINDEMANN
        elif third is not None:
            r.kind = KIND_THIRD_BODY
            r.arr = _arr(A, b, E, order + 1, ea_to_K, molecules)
        elif "PLOG" in kw:
            r.kind = KIND_PLOG
            r.plog = sorted((p * P_ATM, *_arr(Ap, bp, Ep, order, ea_to_K, molecules)) for p, Ap, bp, Ep in kw["PLOG"])
            if len({p for p, *_ in r.plog}) != len(r.plog):
                raise ChemkinError("line %d: PLOG pressures must differ (one rate per pressure)" % n)
        elif "CHEB" in kw:
            r.kind = KIND_CHEB
            nt, npr, eta = kw["CHEB"]
            tr, pr = kw.get("TCHEB", (300.0, 2500.0)), kw.get("PCHEB", (0.001, 100.0))
            e = np.array(eta, dtype=np.float64).reshape(nt, npr)
            scale = 1e-6 ** (order - 1) * (N_AVOGADRO ** (order - 1) if molecules else 1.0)
            e[0, 0] += math.log10(scale)
            r.cheb_shape, r.cheb_eta = (nt, npr), e
            r.cheb_range = (tr[0], tr[1], pr[0] * P_ATM, pr[1] * P_ATM)
        else:
            r.arr = _arr(A, b, E, order, ea_to_K, molecules)
        if "EFF" in kw and third is None:
            raise ChemkinError("line %d: efficiencies without a third body" % n)
        out.append(r)
    return out


_SUPPORTED_AUX = {"LOW", "HIGH", "TROE", "SRI", "REV", "PLOG", "CHEB", "TCHEB", "PCHEB", "DUPLICATE", "DUP"}


def _aux(aux: List[Tuple[int, str]], sidx: Dict[str, int], n0: int) -> dict:
    """Auxiliary keywords of one reaction: KEY / numbers / groups and name/value/ efficiencies."""
    kw: dict = {}
    text = " ".join(line for _, line in aux)
    for m in re.finditer(r"([A-Za-z0-9_()*,.#\-\[\]']+)\s*(?:/([^/]*)/)?", text):
        key, val = m.group(1), m.group(2)
        ku = key.upper()
        if val is None:
            if ku in ("DUPLICATE", "DUP"):
                continue
            raise ChemkinError("reaction at line %d: unsupported keyword %s" % (n0, key))
        if ku not in _SUPPORTED_AUX and key not in sidx:
            raise ChemkinError("reaction at line %d: unsupported keyword %s" % (n0, key))
        try:
            nums = [_float(x) for x in val.split()] if val.strip() else []
        except ValueError:
            raise ChemkinError("reaction at line %d: bad number in %s /%s/" % (n0, key, val))
        if key in sidx and ku not in _SUPPORTED_AUX:
            if len(nums) != 1:
                raise ChemkinError("reaction at line %d: efficiency of %s needs one value" % (n0, key))
            kw.setdefault("EFF", []).append((sidx[key], nums[0]))
        elif ku in ("LOW", "HIGH", "REV"):
            if len(nums) != 3:
                raise ChemkinError("reaction at line %d: %s needs 3 values" % (n0, ku))
            kw[ku] = tuple(nums)
        elif ku in ("TROE", "SRI"):
            kw[ku] = tuple(nums)
        elif ku == "PLOG":
            if len(nums) != 4:
                raise ChemkinError("reaction at line %d: PLOG needs 4 values" % n0)
            kw.setdefault("PLOG", []).append(tuple(nums))
        elif ku in ("TCHEB", "PCHEB"):
            kw[ku] = tuple(nums[:2])
        elif ku == "CHEB":
            prev = kw.get("CHEB_RAW", [])
            kw["CHEB_RAW"] = prev + nums
        elif key in sidx:
            kw.setdefault("EFF", []).append((sidx[key], nums[0]))
        else:
            raise ChemkinError("reaction at line %d: unsupported keyword %s" % (n0, key))
    if "CHEB_RAW" in kw:
        raw = kw.pop("CHEB_RAW")
        nt, npr = int(raw[0]), int(raw[1])
        if len(raw) != 2 + nt * npr:
            raise ChemkinError("reaction at line %d: CHEB has %d coefficients, expected %d" % (n0, len(raw) - 2, nt * npr))
        kw["CHEB"] = (nt, npr, raw[2:])
    return kw


def parse_file(path: str, thermo_path: Optional[str] = None) -> Model:
    with open(path) as f:
        text = f.read()
    thermo = None
    if thermo_path:
        with open(thermo_path) as f:
            thermo = f.read()
    return parse(text, thermo, name=path)


# ----------------------------------------------------------------------------------------------
# writing

def _fmt(x: float) -> str:
    return repr(float(x))


def write(model: Model, species_names: Optional[Sequence[str]] = None,
          element_names: Optional[Sequence[str]] = None, element_weights: Optional[Sequence[float]] = None) -> str:
    """Chemkin text of ``model`` (energies in KELVINS, A in cm^3-mol-s), readable by :func:`parse`.

    Elements are declared with explicit atomic weights (g/mol; default: the synthetic generator's
    element masses), so molecular weights come back to rounding. NASA coefficients are written in
    the format's 15-character fields (9 significant digits), as in any Chemkin thermo file."""
    ne = model.n_elements
    els = list(element_names) if element_names else ["E%d" % i for i in range(ne)]
    wts = list(element_weights) if element_weights else [m * 1e3 for m in synth._ELEMENT_MASS[:ne]]
    if len(els) != ne or len(wts) != ne or any(len(e) > 2 for e in els):
        raise ChemkinError("need one element name of at most 2 characters and one weight per element")
    names = list(species_names) if species_names else ["S%d" % i for i in range(model.n_species)]
    lines = ["ELEMENTS"] + ["%s/%s/" % (e, _fmt(w)) for e, w in zip(els, wts)] + ["END", "SPECIES"]
    lines += names
    lines += ["END", "THERMO"]
    for k, s in enumerate(model.species):
        comp = [(e, int(c)) for e, c in zip(els, s.elem) if int(c)]
        if len(comp) > 5:
            raise ChemkinError("the fixed-column thermo format takes at most 5 elements per species")
        l1 = "%-18s%6s" % (names[k], "")
        for e, c in comp[:4]:
            l1 += "%-2s%3d" % (e, c)
        l1 = l1.ljust(44) + "G" + "%10.3f%10.3f%8.2f" % (s.T_low, s.T_high, s.T_mid)
        if len(comp) == 5:
            l1 = l1.ljust(73) + "%-2s%3d" % comp[4]
        lines.append(l1.ljust(79) + "1")
        c = list(s.a_high) + list(s.a_low)
        rows = [c[0:5], c[5:10], c[10:14]]
        for i, row in enumerate(rows):
            lines.append("".join("%15.8E" % v for v in row).ljust(79) + str(i + 2))
    lines.append("END")
    lines.append("REACTIONS KELVINS MOLES")
    for r in model.reactions:
        lines += _write_reaction(r, names)
    lines.append("END")
    return "\n".join(lines) + "\n"


def _write_reaction(r: Reaction, names: Sequence[str]) -> List[str]:
    def side(terms):
        return " + ".join(("%d%s" % (nu, names[s]) if nu != 1 else names[s]) for s, nu in terms)

    order = sum(nu for _, nu in r.reac)
    tb = "M" if r.tb_mode == TB_MIXTURE else (names[r.tb_species] if r.tb_mode == TB_SPECIES else None)
    arrow = "=>" if r.rev_mode == REV_IRREVERSIBLE else "<=>"

    def cgs(arr, o):
        A, b, Ta = arr
        return "%s %s %s" % (_fmt(A / 1e-6 ** (o - 1)), _fmt(b), _fmt(Ta))

    extra = []
    if r.kind in (KIND_FALLOFF, KIND_CHEM):
        eq = "%s (+%s) %s %s (+%s)" % (side(r.reac), tb, arrow, side(r.prod), tb)
        if r.kind == KIND_FALLOFF:
            head = cgs(r.kinf, order)
            extra.append("LOW / %s /" % cgs(r.k0, order + 1))
        else:
            head = cgs(r.k0, order + 1)
            extra.append("HIGH / %s /" % cgs(r.kinf, order))
        if r.ftype == F_TROE:
            n = 4 if r.troe_has_T2 else 3
            extra.append("TROE / %s /" % " ".join(_fmt(x) for x in r.fparams[:n]))
        elif r.ftype == F_SRI:
            extra.append("SRI / %s /" % " ".join(_fmt(x) for x in r.fparams[:5]))
    elif r.kind == KIND_THIRD_BODY:
        eq = "%s + %s %s %s + %s" % (side(r.reac), tb, arrow, side(r.prod), tb)
        head = cgs(r.arr, order + 1)
    elif r.kind == KIND_PLOG:
        eq = "%s %s %s" % (side(r.reac), arrow, side(r.prod))
        head = cgs(r.plog[0][1:], order)
        for p, A, b, Ta in r.plog:
            extra.append("PLOG / %s %s /" % (_fmt(p / P_ATM), cgs((A, b, Ta), order)))
    elif r.kind == KIND_CHEB:
        eq = "%s %s %s" % (side(r.reac), arrow, side(r.prod))
        head = "1.0 0.0 0.0"
        nt, npr = r.cheb_shape
        e = np.array(r.cheb_eta, dtype=np.float64).reshape(nt, npr).copy()
        e[0, 0] -= math.log10(1e-6 ** (order - 1))
        extra.append("TCHEB / %s %s /" % (_fmt(r.cheb_range[0]), _fmt(r.cheb_range[1])))
        extra.append("PCHEB / %s %s /" % (_fmt(r.cheb_range[2] / P_ATM), _fmt(r.cheb_range[3] / P_ATM)))
        extra.append("CHEB / %d %d %s /" % (nt, npr, " ".join(_fmt(x) for x in e.ravel())))
    else:
        eq = "%s %s %s" % (side(r.reac), arrow, side(r.prod))
        head = cgs(r.arr, order)
    if r.tb_mode == TB_MIXTURE and r.eff:
        extra.append(" ".join("%s/%s/" % (names[s], _fmt(a)) for s, a in r.eff))
    if r.rev_mode == REV_EXPLICIT:
        ro = sum(nu for _, nu in r.prod) + (1 if r.kind == KIND_THIRD_BODY else 0)
        extra.append("REV / %s /" % cgs(r.rev_arr, ro))
    return ["%s   %s" % (eq, head)] + extra
