"""Constant-volume form (Section 3.3) of the CUDA path against the oracle, entry by entry.

The oracle's constant-volume Jacobian is the complex-step derivative of its constant-volume source
terms (exact to rounding); the kernels evaluate the analytical one (the constant-pressure
reuse order with the constant-volume terms). The bar is the constant-pressure one,
|x - x_oracle| <= 1e-10 |x_oracle| + kappa eps S, with kappa = 64 plus the conditioning of the
model's rate exponentials (tests.parity.rate_exponent_condition, 240-410 on the four models):
the oracle's scale S here is the size of each reaction's derivative, not of every term inside
it, so the rates' own rounding (up to that many ulps, which the relative term absorbs elsewhere)
has to be in the scale term for cancelled entries."""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_03262_b300 import synth
from paper_1605_03262_b300.synth import R_GAS
from tests import mechs
from tests.parity import KAPPA_MULT, REL, compare, rate_exponent_condition

pytestmark = pytest.mark.gpu


def _rho(model, T, P, Y):
    W = np.array([s.W for s in model.species])
    return P / (R_GAS * T * (Y / W).sum(axis=1))


def _dev(*arrays):
    return [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in arrays]


def _check(model, T, P, Y, what):
    import paper_1605_03262_b300 as pj
    blob = synth.to_bytes(model)
    rho = _rho(model, T, P, Y)
    g = pj.Model(blob)
    Td, rd, Yd = _dev(T, rho, Y)
    J, f = g.eval_jacobian_cv(Td, rd, Yd, dydt=True)
    fd = g.eval_dydt_cv(Td, rd, Yd)
    torch.cuda.synchronize()
    om = oracle.load_model(blob)
    Jo, Js = om.jacobian_cv(T, rho, Y, with_scale=True)
    fo, fs = om.dydt_cv(T, rho, Y, with_scale=True)
    J, f, fd = J.cpu().numpy(), f.cpu().numpy(), fd.cpu().numpy()
    kappa = KAPPA_MULT + rate_exponent_condition(model, T)
    for x, xo, xs, name in ((J, Jo, Js, "jacobian"), (f, fo, fs, "dydt (jacobian kernel)"), (fd, fo, fs, "dydt")):
        rep = compare(x, xo, xs, kappa_mult=kappa)
        assert rep["n_nonfinite"] == 0 and rep["n_bad"] == 0, (what, name, rep)
        assert rep["max_rel_well_conditioned"] <= REL, (what, name, rep)
    assert np.all(J[:, :, -1] == 0.0)
    return g, (Td, rd, Yd), J


@pytest.mark.parametrize("case", range(len(mechs.TYPE_CASES)))
def test_cv_parity_per_reaction_type(case):
    label, kw = mechs.TYPE_CASES[case]
    model = mechs.typed_model(label, seed=700 + case, **kw)
    T, P, Y = synth.generate_states(model.n_species, 67, seed=800 + case)
    _check(model, T, P, Y, label)


def test_cv_parity_mixed_model():
    model = mechs.mixed_model(seed=61, n_species=17, n_reactions=90)
    T, P, Y = synth.generate_states(model.n_species, 200, seed=62)
    _check(model, T, P, Y, "mixed")


@pytest.mark.parametrize("cfg,n", [(0, 1024), (1, 120), (2, 30), (3, 6)])
def test_cv_parity_configs(cfg, n):
    model = synth.config_model(cfg)
    T, P, Y = synth.config_states(cfg, n, seed_offset=77)
    _check(model, T, P, Y, "cfg%d" % cfg)


def test_cv_launch_shape_does_not_change_results():
    model = synth.config_model(1)
    T, P, Y = synth.config_states(1, 150, seed_offset=5)
    g, (Td, rd, Yd), J = _check(model, T, P, Y, "cfg1 shapes")
    ref = torch.as_tensor(J)
    for wps, groups in [(1, 2), (4, 1), (2, 5)]:
        g.set_launch(wps, groups)
        assert torch.equal(g.eval_jacobian_cv(Td, rd, Yd).cpu(), ref), (wps, groups)


def test_cv_species_rows_of_source_terms_match_constant_pressure():
    """At the density of the same states, dY_k/dt of both forms agrees to rounding (the kernels
    recompute p from rho in the constant-volume form)."""
    import paper_1605_03262_b300 as pj
    model = synth.config_model(1)
    T, P, Y = synth.config_states(1, 500, seed_offset=9)
    g = pj.Model(synth.to_bytes(model))
    Td, Pd, rd, Yd = _dev(T, P, _rho(model, T, P, Y), Y)
    fcp, fcv = g.eval_dydt(Td, Pd, Yd).cpu().numpy(), g.eval_dydt_cv(Td, rd, Yd).cpu().numpy()
    scale = np.abs(fcp[:, 1:]).max(axis=1, keepdims=True)
    assert np.all(np.abs(fcv[:, 1:] - fcp[:, 1:]) <= 1e-12 * scale)


def test_cv_argument_errors():
    import paper_1605_03262_b300 as pj
    model = synth.config_model(0)
    g = pj.Model(synth.to_bytes(model))
    N = model.n_species
    T, P, Y = synth.config_states(0, 4)
    Td, rd, Yd = _dev(T, _rho(model, T, P, Y), Y)
    J = torch.empty((4, N + 1, N + 1), dtype=torch.float64, device="cuda")
    lib = pj.library()
    s = torch.cuda.current_stream().cuda_stream
    rh = np.ascontiguousarray(_rho(model, T, P, Y))
    assert lib.pj_eval_jacobian_cv(g.handle, 4, Td.data_ptr(), rh.ctypes.data, Yd.data_ptr(), N, J.data_ptr(),
                                   (N + 1) ** 2, None, 0, s) == -1
    assert b"rho" in lib.pj_last_error()
    assert lib.pj_eval_dydt_cv(g.handle, 4, Td.data_ptr(), rd.data_ptr(), Yd.data_ptr(), N, J.data_ptr(), N, s) == -1
    assert lib.pj_eval_jacobian_cv(g.handle, 0, None, None, None, N, None, (N + 1) ** 2, None, 0, s) == 0
