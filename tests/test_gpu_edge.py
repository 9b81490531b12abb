"""Edge cases of the CUDA path against the oracle: states at the boundaries the method has (a
species absent, all the mass in one species, T on a NASA7 range boundary, p on and outside the
PLOG grid, a single-species third body with zero concentration), and the benchmark's own launch
configuration (autotuned shape, specialised kernel) at full size, on sampled states."""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_03262_b300 import autotune, synth
from paper_1605_03262_b300.synth import P_ATM
from tests import mechs
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu


def _dev(*arrays):
    return [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in arrays]


def _edge_states(model, n, seed):
    """Seeded states with the method's degenerate cases planted in them."""
    N = model.n_species
    T, P, Y = synth.generate_states(N, n, seed=seed)
    rng = np.random.default_rng(seed)
    Y = Y.copy()
    # species absent (including the last species, whose column is the reference direction)
    for s in range(0, n, 3):
        for k in rng.choice(N, size=max(1, N // 4), replace=False):
            Y[s, k] = 0.0
        Y[s] /= Y[s].sum()
    Y[1, :] = 0.0
    Y[1, N - 1] = 1.0                                   # all the mass in the last species
    Y[2, :] = 0.0
    Y[2, 0] = 1.0                                       # ... in the first one
    Y[4, N - 1] = 0.0
    Y[4] /= Y[4].sum()
    T[5:9] = [1000.0, np.nextafter(1000.0, 0.0), 300.0, 2999.0]   # NASA7 boundary and range ends
    grid = sorted({g[0] for r in model.reactions for g in r.plog})
    if grid:
        P[9] = grid[0]                                  # on the PLOG grid (tie rule)
        P[10] = grid[-1]
        P[11] = 0.5 * grid[0]                           # below and above: the end rates
        P[12] = 2.0 * grid[-1]
    return T, P, Y


@pytest.mark.parametrize("cfg", [0, 2])
def test_degenerate_states_parity(cfg):
    import paper_1605_03262_b300 as pj
    model = synth.config_model(cfg)
    T, P, Y = _edge_states(model, 40, seed=71 + cfg)
    blob = synth.to_bytes(model)
    g = pj.Model(blob)
    J, f = g.eval_jacobian(*_dev(T, P, Y), dydt=True)
    Jo, fo, Js, fs = oracle.load_model(blob).jacobian(T, P, Y, with_scale=True)
    assert_parity(J.cpu().numpy(), Jo, Js, "cfg%d edge" % cfg)
    assert_parity(f.cpu().numpy(), fo, fs, "cfg%d edge dydt" % cfg)


@pytest.mark.parametrize("case", [i for i, (lab, kw) in enumerate(mechs.TYPE_CASES)
                                  if kw.get("species_tb_fraction", 0.0) > 0 or lab in ("plog", "cheb")])
def test_degenerate_states_per_reaction_type(case):
    """Species-m third bodies and falloff with [X_m] = 0 (P_r = 0, the clamped log10 P_r), PLOG on
    and outside its grid, Chebyshev near its temperature limits."""
    import paper_1605_03262_b300 as pj
    label, kw = mechs.TYPE_CASES[case]
    model = mechs.typed_model(label, seed=640 + case, **kw)
    T, P, Y = _edge_states(model, 30, seed=650 + case)
    for r in model.reactions:                            # every species-m third body absent in state 0
        if r.tb_species >= 0:
            Y[0, r.tb_species] = 0.0
    Y[0] /= Y[0].sum()
    blob = synth.to_bytes(model)
    J = pj.Model(blob).eval_jacobian(*_dev(T, P, Y))
    Jo, _, Js, _ = oracle.load_model(blob).jacobian(T, P, Y, with_scale=True)
    assert_parity(J.cpu().numpy(), Jo, Js, label + " edge")


def test_benchmark_configuration_full_size_sampled_parity():
    """The benchmark's configuration on the 53-species model: all 65,536 states, the autotuned
    launch shape and the kernel specialised for the model; sampled states against the oracle and
    every state against the data-driven default launch, bitwise."""
    import paper_1605_03262_b300 as pj
    model = synth.config_model(1)
    blob = synth.to_bytes(model)
    T, P, Y = synth.config_states(1)
    Td, Pd, Yd = _dev(T, P, Y)
    base = pj.Model(blob).eval_jacobian(Td, Pd, Yd)
    g = pj.Model(blob)
    autotune.autotune(g, blob, use_cache=False)
    assert g.specialize()["jacobian"]
    J = g.eval_jacobian(Td, Pd, Yd)
    torch.cuda.synchronize()
    assert torch.equal(J, base)
    del base
    idx = np.unique(np.concatenate([[0, len(T) - 1], np.random.default_rng(5).integers(0, len(T), 40)]))
    Jo, _, Js, _ = oracle.load_model(blob).jacobian(T[idx], P[idx], Y[idx], with_scale=True)
    assert_parity(J[torch.as_tensor(idx, device="cuda")].cpu().numpy(), Jo, Js, "benchmark configuration")
