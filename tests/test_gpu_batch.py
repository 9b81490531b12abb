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


def _jac_items(items):
    outs = []
    for g, T, P, Y in items:
        N = g.n_species
        outs.append((torch.full((T.shape[0], N + 1, N + 1), float("nan"), dtype=torch.float64, device="cuda"),
                     torch.full((T.shape[0], N + 1), float("nan"), dtype=torch.float64, device="cuda")))
    return outs


@pytest.mark.parametrize("which", ["jacobian", "dydt"])
def test_specialised_batch_kernel_equals_plain_launches(which):
    """The plan's kernel compiled for its models (NVRTC; one part per (model, group width)) gives
    the plain per-model results bit for bit, with per-item shapes, also from a graph."""
    import paper_1605_03262_b300 as pj
    items = _items(seed=11)
    g0 = items[0][0]                                    # the first model again, at another width
    items.append((g0, *_dev(*synth.generate_states(g0.n_species, 200, seed=99))))
    outs = _jac_items(items)
    if which == "jacobian":
        plan_items = [(g, T, P, Y, J, f) for (g, T, P, Y), (J, f) in zip(items, outs)]
    else:
        plan_items = [(g, T, P, Y, f) for (g, T, P, Y), (J, f) in zip(items, outs)]
    # the first and last items share a model at different widths: two branches for it
    shapes = [(1, 8, 24), (2, 0, 0), (0, 3, 0), (0, 0, 5), (4, 2, 7), (2, 0, 9)]
    plan = pj.BatchPlan(plan_items, which=which, item_shapes=shapes)
    info = plan.specialize()
    assert info["active"] and info["slots"] == len(items) and info["cubin_bytes"] > 0
    graph = plan.capture()
    graph.replay()
    torch.cuda.synchronize()
    for (g, T, P, Y), (J, f) in zip(items, outs):
        if which == "jacobian":
            ref, fref = g.eval_jacobian(T, P, Y, dydt=True)
            assert torch.equal(J, ref)
            assert torch.equal(f, fref)
        else:
            assert torch.equal(f, g.eval_dydt(T, P, Y))
    assert not plan.specialize(False)["active"]


def test_specialised_plan_with_chosen_widths_and_an_empty_item():
    """Widths left to the plan (the 360-species model's among them, which the specialised kernel
    may widen to the model's own), an item without states between others, a tile table cut into
    shorter tiles for the costly models: the specialised plan still gives the plain launches'
    bits, and a plan that runs only the data-driven kernel gives the same."""
    import paper_1605_03262_b300 as pj
    items = _items(seed=17)
    for g, _, _, _ in items:
        g.specialize()                                  # the models' own widths, as a server has them
    g1, T1, P1, Y1 = items[1]
    items.insert(2, (g1, T1[:0], P1[:0], Y1[:0]))       # no states
    outs = _jac_items(items)
    plan_items = [(g, T, P, Y, J) for (g, T, P, Y), (J, f) in zip(items, outs)]
    plan = pj.BatchPlan(plan_items, tile_states=64)
    refs = [g.eval_jacobian(T, P, Y) for g, T, P, Y in items]
    plan.run()
    torch.cuda.synchronize()
    for (J, _), ref in zip(outs, refs):
        assert torch.equal(J, ref)
        J.fill_(float("nan"))
    assert plan.specialize()["active"]
    plan.run()
    torch.cuda.synchronize()
    for (J, _), ref in zip(outs, refs):
        assert torch.equal(J, ref)


def test_batch_autotuner_picks_a_timed_candidate_and_keeps_results():
    import paper_1605_03262_b300 as pj
    from paper_1605_03262_b300 import autotune
    items = _items(seed=13)[:3]
    outs = _jac_items(items)
    plan_items = [(g, T, P, Y, J) for (g, T, P, Y), (J, f) in zip(items, outs)]
    plan, rep = autotune.autotune_batch(plan_items, use_cache=False)
    assert rep["choice"] in rep["timings"] and rep["specialised_ms"] is not None
    assert rep["specialised"]["active"] == (rep["specialised_ms"] < rep["timings"][rep["choice"]])
    assert len(rep["timings"]) == len(autotune.batch_candidates(plan_items))
    for J, _ in outs:
        J.fill_(float("nan"))
    plan.run()
    torch.cuda.synchronize()
    for (g, T, P, Y), (J, f) in zip(items, outs):
        assert torch.equal(J, g.eval_jacobian(T, P, Y))
