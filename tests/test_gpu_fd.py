"""GPU forward-difference Jacobian (the paper's finite-difference comparison, Section 5.2) against
the oracle's, entry by entry.

Both sides use the same increments (exact functions of the inputs), so the columns differ only by
the rounding of the source terms, divided by the increment. The bar is the parity bar with the
oracle's per-entry scale (S(y + h d) + S(y)) / h and 256 eps instead of 64 eps: the term scale S
counts each term's magnitude but not the conditioning of the rate exponentials inside it (the
argument ln A + beta ln T - Ta/T reaches ~100 in magnitude, so two correct evaluations of a rate
differ by up to ~100 ulp). The source-term parity tests absorb this in their 1e-10 relative term;
a forward difference divides it by h, so here it has to be in the scale term (measured: up to
~92 eps S on the 53-species model)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_03262_b300 import synth
from tests import mechs
from tests.parity import EPS, compare

pytestmark = pytest.mark.gpu
KAPPA_FD = 256.0


def _dev(*arrays):
    return [torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in arrays]


def _check(J, Jo, Js, what):
    rep = compare(J, Jo, Js, kappa_mult=KAPPA_FD)
    assert rep["n_nonfinite"] == 0 and rep["n_bad"] == 0, (what, rep)


@pytest.mark.parametrize("cfg,n", [(0, 96), (1, 12), (2, 3)])
def test_fd_parity_with_oracle(cfg, n):
    import paper_1605_03262_b300 as pj
    model = synth.config_model(cfg)
    blob = synth.to_bytes(model)
    T, P, Y = synth.config_states(cfg, n, seed_offset=2024)
    J = pj.Model(blob).eval_jacobian_fd(*_dev(T, P, Y)).cpu().numpy()
    Jo, Js = oracle.load_model(blob).jacobian_fd(T, P, Y, with_scale=True)
    _check(J, Jo, Js, cfg)
    assert np.all(J[:, :, -1] == 0.0)


@pytest.mark.parametrize("case", range(len(mechs.TYPE_CASES)))
def test_fd_parity_per_reaction_type(case):
    import paper_1605_03262_b300 as pj
    lab, kw = mechs.TYPE_CASES[case]
    model = mechs.typed_model(lab, seed=500 + case, **kw)
    blob = synth.to_bytes(model)
    T, P, Y = synth.generate_states(model.n_species, 9, seed=900 + case)
    J = pj.Model(blob).eval_jacobian_fd(*_dev(T, P, Y)).cpu().numpy()
    Jo, Js = oracle.load_model(blob).jacobian_fd(T, P, Y, with_scale=True)
    _check(J, Jo, Js, lab)


def test_fd_chunked_workspace_equals_one_pass():
    """A workspace for 3 states processes 10 states in four passes with the same bits."""
    import paper_1605_03262_b300 as pj
    model = synth.config_model(0)
    g = pj.Model(synth.to_bytes(model))
    T, P, Y = _dev(*synth.config_states(0, 10, seed_offset=31))
    one = g.eval_jacobian_fd(T, P, Y)
    ws = torch.empty(g.fd_workspace_bytes(3), dtype=torch.uint8, device="cuda")
    chunked = g.eval_jacobian_fd(T, P, Y, workspace=ws)
    assert torch.equal(one, chunked)


def test_fd_close_to_analytical_jacobian():
    """The forward difference lies within its rounding bound (KAPPA_FD eps times the oracle's scale)
    plus a 1e-5 relative truncation allowance of the analytical Jacobian."""
    import paper_1605_03262_b300 as pj
    model = synth.config_model(1)
    blob = synth.to_bytes(model)
    T, P, Y = synth.config_states(1, 8, seed_offset=404)
    g = pj.Model(blob)
    Td, Pd, Yd = _dev(T, P, Y)
    Jfd = g.eval_jacobian_fd(Td, Pd, Yd).cpu().numpy()
    Jan = g.eval_jacobian(Td, Pd, Yd).cpu().numpy()
    _, Js = oracle.load_model(blob).jacobian_fd(T, P, Y, with_scale=True)
    assert np.all(np.abs(Jfd - Jan) <= KAPPA_FD * EPS * Js + 1e-5 * np.abs(Jan) + 1e-300)


def test_fd_argument_errors():
    import paper_1605_03262_b300 as pj
    model = synth.config_model(0)
    g = pj.Model(synth.to_bytes(model))
    T, P, Y = _dev(*synth.config_states(0, 4))
    tiny = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(pj.LibraryError):
        g.eval_jacobian_fd(T, P, Y, workspace=tiny)
    assert g.eval_jacobian_fd(T[:0], P[:0], Y[:0]).shape == (0, model.n_species + 1, model.n_species + 1)
