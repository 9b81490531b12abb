"""Small hand-built kinetic models for tests (inputs only; no method arithmetic)."""
import numpy as np

from paper_1605_03262_b300 import synth
from paper_1605_03262_b300.synth import Model, Reaction, Species


def species_from_vectors(vecs, seed=0):
    """Species with distinct element vectors and random smooth NASA7 fits."""
    rng = np.random.default_rng(seed)
    out = []
    for v in vecs:
        W = float(sum(c * m for c, m in zip(v, synth._ELEMENT_MASS)))
        a_lo, a_hi = synth._fit_nasa7(rng, 300.0, 1000.0, 3000.0)
        out.append(Species(W, 300.0, 1000.0, 3000.0, a_lo, a_hi, np.array(v, dtype=np.int32)))
    return out


def one_reaction_model(r: Reaction, vecs, seed=0) -> Model:
    return Model(n_elements=len(vecs[0]), species=species_from_vectors(vecs, seed), reactions=[r])


def typed_model(label, seed, n_species=8, n_reactions=6, **kw):
    mix = {label: 1.0}
    return synth.generate_model(n_species, n_reactions, 3, mix, seed=seed, **kw)


# every (label, options) combination the oracle and the kernels must cover
TYPE_CASES = [
    ("elementary", dict(rev_modes=(0, 1, 2))),
    ("third_body", dict(species_tb_fraction=0.0, rev_modes=(1, 2))),
    ("third_body", dict(species_tb_fraction=1.0)),
    ("third_body", dict(species_tb_fraction=0.0, eff_fraction=0.0)),
    ("lindemann", dict(species_tb_fraction=0.0, chem_fraction=0.0)),
    ("troe", dict(species_tb_fraction=0.0, chem_fraction=0.0, rev_modes=(0, 1, 2))),
    ("sri", dict(species_tb_fraction=0.0, chem_fraction=0.0)),
    ("lindemann", dict(species_tb_fraction=0.0, chem_fraction=1.0)),
    ("troe", dict(species_tb_fraction=0.3, chem_fraction=1.0)),
    ("sri", dict(species_tb_fraction=0.0, chem_fraction=1.0)),
    ("troe", dict(species_tb_fraction=1.0, chem_fraction=0.0)),
    ("plog", dict()),
    ("cheb", dict()),
]


def mixed_model(seed=11, n_species=12, n_reactions=40):
    mix = {"elementary": 0.3, "third_body": 0.15, "troe": 0.15, "lindemann": 0.1, "sri": 0.1,
           "plog": 0.1, "cheb": 0.1}
    return synth.generate_model(n_species, n_reactions, 4, mix, seed=seed, rev_modes=(0, 1, 2),
                                chem_fraction=0.3, species_tb_fraction=0.2)
