"""Run-time specialised kernels (NVRTC; the paper's per-mechanism code generation): the same bits as
the data-driven kernels for every output, both formulations and several launch shapes, and used
only for the launch shape they were compiled for."""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_03262_b300 import synth
from paper_1605_03262_b300.synth import R_GAS
from tests import mechs
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu


def _dev(*arrays):
    return [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in arrays]


def _all_outputs(g, T, P, rho, Y):
    J, f = g.eval_jacobian(T, P, Y, dydt=True)
    Jv, fv = g.eval_jacobian_cv(T, rho, Y, dydt=True)
    out = [J, f, g.eval_dydt(T, P, Y), Jv, fv, g.eval_dydt_cv(T, rho, Y)]
    torch.cuda.synchronize()
    return [x.cpu() for x in out]


def _rho(model, T, P, Y):
    W = np.array([s.W for s in model.species])
    return P / (R_GAS * T * (Y / W).sum(axis=1))


def _case(model, T, P, Y, shapes):
    import paper_1605_03262_b300 as pj
    blob = synth.to_bytes(model)
    base, spec = pj.Model(blob), pj.Model(blob)
    Td, Pd, rd, Yd = _dev(T, P, _rho(model, T, P, Y), Y)
    for shape in shapes:
        try:
            base.set_launch(*shape)
            spec.set_launch(*shape)
        except Exception:
            continue
        info = spec.specialize()
        assert info["jacobian"] and info["dydt"] and info["cubin_bytes"] > 0, info
        ref = _all_outputs(base, Td, Pd, rd, Yd)
        got = _all_outputs(spec, Td, Pd, rd, Yd)
        for a, b in zip(ref, got):
            assert torch.equal(a, b), (model.n_species, shape)
    return spec, (Td, Pd, rd, Yd), got


@pytest.mark.parametrize("cfg,n", [(0, 300), (1, 200), (2, 40), (3, 6)])
def test_specialised_kernels_match_data_driven_bitwise(cfg, n):
    model = synth.config_model(cfg)
    T, P, Y = synth.config_states(cfg, n, seed_offset=55)
    import paper_1605_03262_b300 as pj
    tuned = pj.Model(synth.to_bytes(model)).get_launch()
    shapes = [tuned[:2], (1, 2), (2, 3)]
    _, _, got = _case(model, T, P, Y, shapes)
    # and the parity bar against the oracle, on the last shape's outputs
    Jo, fo, Js, fs = oracle.load_model(synth.to_bytes(model)).jacobian(T, P, Y, with_scale=True)
    assert_parity(got[0].numpy(), Jo, Js, "specialised cfg%d" % cfg)


@pytest.mark.parametrize("case", range(len(mechs.TYPE_CASES)))
def test_specialised_kernels_every_reaction_type(case):
    label, kw = mechs.TYPE_CASES[case]
    model = mechs.typed_model(label, seed=900 + case, **kw)
    T, P, Y = synth.generate_states(model.n_species, 33, seed=950 + case)
    _case(model, T, P, Y, [(1, 4)])


def test_specialisation_follows_the_launch_shape():
    import paper_1605_03262_b300 as pj
    model = synth.config_model(1)
    T, P, Y = synth.config_states(1, 64, seed_offset=3)
    g = pj.Model(synth.to_bytes(model))
    g.set_launch(2, 5)
    info = g.specialize()
    assert info["jacobian"] and info["dydt"] and info["compile_seconds"] > 0
    Td, Pd, Yd = _dev(T, P, Y)
    a = g.eval_jacobian(Td, Pd, Yd).cpu()
    g.set_launch(1, 3)                       # another shape: the data-driven kernels run
    assert not g.spec_info()["jacobian"] and g.spec_info()["dydt"]
    b = g.eval_jacobian(Td, Pd, Yd).cpu()
    assert torch.equal(a, b)
    g.set_launch(2, 5)                       # back to the compiled shape
    assert g.spec_info()["jacobian"]
    g.specialize(False)
    assert g.spec_info() == {"jacobian": False, "dydt": False, "compile_seconds": 0.0, "cubin_bytes": 0}
    assert torch.equal(g.eval_jacobian(Td, Pd, Yd).cpu(), a)
