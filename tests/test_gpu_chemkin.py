"""A mechanism read from Chemkin text goes through the library like any other: parity of the GPU
Jacobian and source terms with the oracle on the invented feature fixture."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1605_03262_b300 import chemkin, synth
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "chemkin_features.inp")


def test_chemkin_fixture_parity():
    import paper_1605_03262_b300 as pj
    with open(GOLDEN) as f:
        model = chemkin.parse(f.read())
    blob = synth.to_bytes(model)
    T, P, Y = synth.generate_states(model.n_species, 200, seed=11)
    g = pj.Model(blob)
    Td, Pd, Yd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, Y))
    J, f = g.eval_jacobian(Td, Pd, Yd, dydt=True)
    Jo, fo, Js, fs = oracle.load_model(blob).jacobian(T, P, Y, with_scale=True)
    assert_parity(J.cpu().numpy(), Jo, Js, "chemkin fixture")
    assert_parity(f.cpu().numpy(), fo, fs, "chemkin fixture dydt")
