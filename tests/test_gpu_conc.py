"""Molar-concentration basis at constant pressure on the CUDA path against the oracle: the sparse
Jacobian of (dT/dt, dV/dt, dn_k/dt) with respect to (T, V, n_1..n_{N-1}), value by value at the
pattern's entries, the oracle's entries outside the pattern zero to rounding, and the source terms;
on the four benchmark models, every reaction type, seeded random models and launch shapes, states
with absent species, and the benchmark's full-size batch on sampled states."""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_03262_b300 import synth
from tests import mechs
from tests.parity import EPS, KAPPA_MULT, assert_parity, compare, rate_exponent_condition

pytestmark = pytest.mark.gpu


def _dev(*arrays):
    return [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in arrays]


def _check(model, T, P, V, nmol, g=None, what=""):
    import paper_1605_03262_b300 as pj
    blob = synth.to_bytes(model)
    g = g if g is not None else pj.Model(blob)
    N = model.n_species
    rp, ci = g.conc_pattern()
    assert rp[0] == 0 and rp[-1] == len(ci) and len(rp) == N + 2
    vals, f = g.eval_jacobian_conc(*_dev(T, P, V, nmol), dydt=True)
    vals, f = vals.cpu().numpy(), f.cpu().numpy()
    Jo, fo, Js, fs = oracle.load_model(blob).jacobian_conc(T, P, V, nmol, with_scale=True)
    rows = np.repeat(np.arange(N + 1), np.diff(rp))
    kappa = KAPPA_MULT + rate_exponent_condition(model, T)
    rep = compare(vals, Jo[:, rows, ci], Js[:, rows, ci], kappa_mult=kappa)
    assert rep["n_nonfinite"] == 0 and rep["n_bad"] == 0, (what, "jacobian", rep)
    rep = compare(f, fo, fs, kappa_mult=kappa)
    assert rep["n_nonfinite"] == 0 and rep["n_bad"] == 0, (what, "dydt", rep)
    # outside the pattern the oracle's derivative is zero up to its own rounding
    mask = np.ones((N + 1, N + 1), bool)
    mask[rows, ci] = False
    rowmax = np.abs(Jo).max(axis=2, keepdims=True)
    off = np.abs(Jo) <= 1e-13 * rowmax + 64 * EPS * Js
    assert np.all(off[:, mask]), (what, "entry outside the pattern")
    return vals, f


@pytest.mark.parametrize("cfg,n", [(0, 64), (1, 24), (2, 6), (3, 2)])
def test_benchmark_models(cfg, n):
    model = synth.config_model(cfg)
    T, P, V, nmol = synth.config_conc_states(cfg, n)
    _check(model, T, P, V, nmol, what="cfg%d" % cfg)


@pytest.mark.parametrize("case", range(len(mechs.TYPE_CASES)))
def test_every_reaction_type(case):
    label, kw = mechs.TYPE_CASES[case]
    model = mechs.typed_model(label, seed=900 + case, **kw)
    T, P, V, nmol = synth.generate_conc_states(model.n_species, 40, seed=910 + case)
    _check(model, T, P, V, nmol, what=label)


@pytest.mark.parametrize("seed", range(8))
def test_random_models_and_launch_shapes(seed):
    import paper_1605_03262_b300 as pj
    rng = np.random.default_rng(5000 + seed)
    N = int(rng.integers(6, 60))
    labels = ("elementary", "third_body", "troe", "lindemann", "sri", "plog", "cheb")
    w = rng.dirichlet(np.full(len(labels), 0.6))
    model = synth.generate_model(N, int(rng.integers(3, 4 * N)), int(rng.integers(4, 6)),
                                 {k: float(x) for k, x in zip(labels, w)}, seed=5000 + seed,
                                 species_tb_fraction=float(rng.uniform(0, 0.4)), chem_fraction=0.2)
    g = pj.Model(synth.to_bytes(model))
    shape = [(1, int(rng.integers(1, 9))), (2, int(rng.integers(1, 5))), (4, 1)][int(rng.integers(0, 3))]
    try:
        g.set_launch(*shape)
    except pj.LibraryError:
        pass
    T, P, V, nmol = synth.generate_conc_states(N, int(rng.integers(1, 90)), seed=5100 + seed)
    _check(model, T, P, V, nmol, g=g, what="seed %d" % seed)


def test_absent_species_and_scarce_last_species():
    model = synth.config_model(0)
    N = model.n_species
    T, P, V, nmol = synth.generate_conc_states(N, 12, seed=77)
    nmol = nmol.copy()
    nmol[0, :] = 0.0                                        # only the last species present
    nmol[1, 3] = 0.0
    nmol[2, :: 2] = 0.0
    ntot = P * V / (synth.R_GAS * T)
    nmol[3] = nmol[3] / nmol[3].sum() * ntot[3] * (1 - 1e-6)   # the last species scarce
    _check(model, T, P, V, nmol, what="edge")


def test_full_size_batch_sampled():
    """The 53-species model over 65,536 states in the default launch: sampled states against the
    oracle, and every state's values against a second launch of the same states in another order
    (the states are independent, so each state's values must not depend on its position)."""
    import paper_1605_03262_b300 as pj
    model = synth.config_model(1)
    blob = synth.to_bytes(model)
    g = pj.Model(blob)
    T, P, V, nmol = synth.config_conc_states(1)
    Td, Pd, Vd, nd = _dev(T, P, V, nmol)
    vals = g.eval_jacobian_conc(Td, Pd, Vd, nd)
    perm = torch.randperm(len(T), generator=torch.Generator().manual_seed(3)).cuda()
    vals2 = g.eval_jacobian_conc(Td[perm], Pd[perm], Vd[perm], nd[perm])
    torch.cuda.synchronize()
    assert torch.equal(vals[perm], vals2)
    del vals2
    idx = np.unique(np.concatenate([[0, len(T) - 1], np.random.default_rng(8).integers(0, len(T), 24)]))
    rp, ci = g.conc_pattern()
    rows = np.repeat(np.arange(model.n_species + 1), np.diff(rp))
    Jo, _, Js, _ = oracle.load_model(blob).jacobian_conc(T[idx], P[idx], V[idx], nmol[idx], with_scale=True)
    sub = vals[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    rep = compare(sub, Jo[:, rows, ci], Js[:, rows, ci], kappa_mult=KAPPA_MULT + rate_exponent_condition(model, T[idx]))
    assert rep["n_nonfinite"] == 0 and rep["n_bad"] == 0, rep


@pytest.mark.parametrize("cfg", [0, 2])
def test_specialised_kernel_same_bits(cfg):
    """The kernel compiled for the model (NVRTC) returns the data-driven kernel's bits."""
    import paper_1605_03262_b300 as pj
    model = synth.config_model(cfg)
    blob = synth.to_bytes(model)
    T, P, V, nmol = _dev(*synth.config_conc_states(cfg, 300))
    base, fb = pj.Model(blob).eval_jacobian_conc(T, P, V, nmol, dydt=True)
    g = pj.Model(blob)
    assert g.specialize()["jacobian"]
    vals, f = g.eval_jacobian_conc(T, P, V, nmol, dydt=True)
    torch.cuda.synchronize()
    assert torch.equal(vals, base) and torch.equal(f, fb)


def test_values_do_not_depend_on_the_launch_shape():
    """Every sum runs in a fixed lane order, so the bits are the same at every group width."""
    import paper_1605_03262_b300 as pj
    model = synth.config_model(1)
    blob = synth.to_bytes(model)
    T, P, V, nmol = _dev(*synth.config_conc_states(1, 200))
    ref = None
    for shape in ((1, 4, 1), (2, 7, 1), (4, 3, 1), (8, 1, 1)):
        g = pj.Model(blob)
        g.set_launch(*shape)
        vals, f = g.eval_jacobian_conc(T, P, V, nmol, dydt=True)
        torch.cuda.synchronize()
        if ref is None:
            ref = (vals, f)
        else:
            assert torch.equal(vals, ref[0]) and torch.equal(f, ref[1]), shape


def test_argument_errors():
    import paper_1605_03262_b300 as pj
    model = synth.config_model(0)
    g = pj.Model(synth.to_bytes(model))
    T, P, V, nmol = _dev(*synth.config_conc_states(0, 4))
    with pytest.raises(ValueError):
        g.eval_jacobian_conc(T, P, V[:3], nmol)
    rp, ci = g.conc_pattern()
    out = torch.empty((4, len(ci) - 1), dtype=torch.float64, device="cuda")
    with pytest.raises(pj.LibraryError):
        g.eval_jacobian_conc(T, P, V, nmol, out=out)
