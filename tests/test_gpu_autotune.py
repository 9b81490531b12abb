"""The launch-shape autotuner: its second pass re-times the first pass's fastest shapes one cold
launch at a time and sets the fastest of those on the model; results do not depend on the shape
it picks."""
import numpy as np
import pytest
import torch

from paper_1605_03262_b300 import autotune, synth

pytestmark = pytest.mark.gpu


def _shape(key):
    return tuple(int(x) for x in key.split(","))


def test_refine_pass_picks_the_cold_minimum_of_the_fastest_shapes():
    import paper_1605_03262_b300 as pj
    model = synth.config_model(0)
    blob = synth.to_bytes(model)
    T, P, Y = synth.config_states(0)
    probe = tuple(torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, Y))
    g = pj.Model(blob)
    rep = autotune.autotune(g, blob, use_cache=False, probe=probe, refine=3, refine_reps=3)
    first = list(rep["timings"])[:3]
    assert set(rep["refined"]) == set(first)
    best = min(rep["refined"], key=rep["refined"].get)
    assert _shape(best) == tuple(rep["shape"]) == tuple(g.get_launch())
    assert rep["ms"] == rep["refined"][best]
    J = g.eval_jacobian(*probe)

    # without the second pass the first pass's fastest shape stays
    rep0 = autotune.autotune(g, blob, use_cache=False, probe=probe, refine=0)
    assert rep0["refined"] == {}
    assert tuple(rep0["shape"]) == _shape(next(iter(rep0["timings"]))) == tuple(g.get_launch())
    J0 = g.eval_jacobian(*probe)
    torch.cuda.synchronize()
    assert torch.equal(J, J0)
    assert np.isfinite(J.cpu().numpy()).all()
