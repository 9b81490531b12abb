"""The batched form: one persistent launch over models of uneven size gives the plain per-model
results (bitwise), also when captured into a CUDA graph and replayed with new inputs."""
import numpy as np
import pytest

from paper_1605_03262_b300 import synth
from tests import mechs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(*arrs):
    return [torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in arrs]


def _items(seed=0):
    models = [synth.config_model(0), synth.config_model(1), mechs.mixed_model(seed=41, n_species=17, n_reactions=90),
              synth.config_model(3), synth.config_model(2)]
    sizes = [1024, 1500, 333, 40, 257]
    out = []
    import paper_1605_03262_b300 as pj
    for k, (m, n) in enumerate(zip(models, sizes)):
        T, P, Y = synth.generate_states(m.n_species, n, seed=seed + 7 * k)
        g = pj.Model(synth.to_bytes(m))
        out.append((g, *_dev(T, P, Y)))
    return out


def test_batched_jacobians_equal_plain_launches():
    import paper_1605_03262_b300 as pj
    items = _items()
    outs, fouts, plan_items = [], [], []
    for g, T, P, Y in items:
        N = g.n_species
        J = torch.full((T.shape[0], N + 1, N + 1), float("nan"), dtype=torch.float64, device="cuda")
        f = torch.full((T.shape[0], N + 1), float("nan"), dtype=torch.float64, device="cuda")
        outs.append(J)
        fouts.append(f)
        plan_items.append((g, T, P, Y, J, f))
    plan = pj.BatchPlan(plan_items)
    assert plan.n_tiles > len(items)
    plan.run()
    for (g, T, P, Y), J, f in zip(items, outs, fouts):
        ref, fref = g.eval_jacobian(T, P, Y, dydt=True)
        torch.cuda.synchronize()
        assert torch.equal(J, ref)
        assert torch.equal(f, fref)


def test_batched_dydt_equals_plain():
    import paper_1605_03262_b300 as pj
    items = _items(seed=3)
    outs = [torch.empty((T.shape[0], g.n_species + 1), dtype=torch.float64, device="cuda") for g, T, P, Y in items]
    plan = pj.BatchPlan([(g, T, P, Y, o) for (g, T, P, Y), o in zip(items, outs)], which="dydt", tile_states=50)
    plan.run()
    for (g, T, P, Y), o in zip(items, outs):
        assert torch.equal(o, g.eval_dydt(T, P, Y))


def test_graph_capture_and_replay_with_new_inputs():
    import paper_1605_03262_b300 as pj
    items = _items(seed=5)
    outs = [torch.empty((T.shape[0], g.n_species + 1, g.n_species + 1), dtype=torch.float64, device="cuda")
            for g, T, P, Y in items]
    plan = pj.BatchPlan([(g, T, P, Y, o) for (g, T, P, Y), o in zip(items, outs)], threads_per_cta=256)
    graph = plan.capture()
    for rep in range(2):
        for k, (g, T, P, Y) in enumerate(items):       # new states, same buffers
            T2, P2, Y2 = synth.generate_states(g.n_species, T.shape[0], seed=100 + 10 * rep + k)
            T.copy_(torch.as_tensor(T2))
            P.copy_(torch.as_tensor(P2))
            Y.copy_(torch.as_tensor(Y2))
        graph.replay()
        torch.cuda.synchronize()
        for (g, T, P, Y), o in zip(items, outs):
            assert torch.equal(o, g.eval_jacobian(T, P, Y))


def test_batch_argument_errors():
    import paper_1605_03262_b300 as pj
    g, T, P, Y = _items()[0]
    bad = torch.empty((T.shape[0], 3), dtype=torch.float64, device="cuda")
    with pytest.raises(pj.LibraryError):
        pj.BatchPlan([(g, T, P, Y, bad)])
    with pytest.raises(pj.LibraryError):
        pj.BatchPlan([(g, T, P, Y, torch.empty((T.shape[0], g.n_species + 1, g.n_species + 1),
                                                dtype=torch.float64, device="cuda"))], threads_per_cta=100)
