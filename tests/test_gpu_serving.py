"""The serving form: continuous batching over several resident models. A request's result is the
same alone and in the mix; work waits for device memory instead of failing; requests overlap."""
import time

import numpy as np
import pytest

from paper_1605_03262_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _models():
    import paper_1605_03262_b300 as pj
    return {synth.CONFIGS[c]["name"]: pj.Model(synth.to_bytes(synth.config_model(c))) for c in (0, 1, 3)}


def _trace(models, n_req, seed):
    rng = np.random.default_rng(seed)
    names = sorted(models)
    out = []
    for k in range(n_req):
        name = names[int(rng.integers(0, len(names)))]
        n = int(np.exp(rng.uniform(0.0, np.log(300.0))))
        T, P, Y = synth.generate_states(models[name].n_species, n, seed=seed * 1000 + k)
        out.append((name, T, P, Y))
    return out


def test_results_alone_equal_results_in_the_mix():
    from paper_1605_03262_b300.serving import Server
    models = _models()
    trace = _trace(models, 40, seed=1)
    probe = trace[17]
    with Server(models, max_inflight=1) as srv:
        alone = srv.submit(*probe).result(timeout=60).cpu()
    with Server(models, max_inflight=4) as srv:
        futs = [srv.submit(*r) for r in trace]
        results = [f.result(timeout=120) for f in futs]
        stats = dict(srv.stats)
    assert torch.equal(results[17].cpu(), alone)
    assert stats["requests"] == len(trace)
    # plain per-request evaluation agrees too
    for (name, T, P, Y), res in zip(trace[:6], results[:6]):
        ref = models[name].eval_jacobian(T, P, Y)
        assert torch.equal(res, ref)


def test_admission_waits_for_memory_instead_of_failing():
    from paper_1605_03262_b300.serving import Server
    models = _models()
    name = synth.CONFIGS[3]["name"]
    N = models[name].n_species
    per_state = 8 * ((N + 1) ** 2 + 2 * (N + 1) + 2)
    trace = []
    for k in range(6):
        T, P, Y = synth.generate_states(N, 50, seed=50 + k)
        trace.append((name, T, P, Y))
    budget = int(per_state * 60)        # room for one 50-state request at a time
    with Server(models, hbm_budget=budget, max_inflight=4) as srv:
        futs = [srv.submit(*r) for r in trace]
        res = [f.result(timeout=120) for f in futs]
        stats = dict(srv.stats)
    assert len(res) == 6 and all(r.shape == (50, N + 1, N + 1) for r in res)
    assert stats["max_inflight_seen"] == 1
    assert stats["waits_for_memory"] > 0
    with Server(models, hbm_budget=budget) as srv:
        with pytest.raises(ValueError):
            srv.submit(name, *synth.generate_states(N, 100, seed=3))


def test_requests_overlap_and_latencies_are_recorded():
    from paper_1605_03262_b300.serving import Server, latency_summary
    models = _models()
    trace = _trace(models, 60, seed=7)
    with Server(models, max_inflight=6, max_batch_states=512) as srv:
        futs = []
        for r in trace:
            futs.append(srv.submit(*r))
            time.sleep(0.0005)
        for f in futs:
            f.result(timeout=120)
        stats = dict(srv.stats)
    summ = latency_summary([f.request for f in futs])
    assert summ["n"] == len(trace) and summ["p99_ms"] >= summ["p50_ms"] > 0
    assert stats["max_inflight_seen"] > 1
