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
    # the mix with request chunking on (chunks of about 20 us of GPU time: every request of more
    # than a few states of the larger models is cut)
    with Server(models, max_inflight=4, chunk_ms=0.02) as srv:
        futs = [srv.submit(*r) for r in trace]
        results = [f.result(timeout=120) for f in futs]
        stats = dict(srv.stats)
    assert torch.equal(results[17].cpu(), alone)
    assert stats["requests"] == len(trace) and stats["chunked_requests"] > 0
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


def test_merged_and_mixed_iterations_give_the_same_results():
    """Per-model merged launches (the default) and mixed-model batched launches (mixed=True) return
    the same bits for every request."""
    from paper_1605_03262_b300.serving import Server
    models = _models()
    trace = _trace(models, 30, seed=11)
    out = {}
    for mixed in (False, True):
        with Server(models, max_inflight=3, mixed=mixed) as srv:
            futs = [srv.submit(*r) for r in trace]
            out[mixed] = [f.result(timeout=120).cpu() for f in futs]
            if mixed:
                assert srv.stats["merged_requests"] > 0
    for a, b in zip(out[False], out[True]):
        assert torch.equal(a, b)


def test_run_batch_with_workspaces_equals_plain_launches():
    """pj_batch_run_ws on two workspaces on two streams, and pj_batch_run_noalloc, equal the plain
    launches of every item."""
    import paper_1605_03262_b300 as pj
    models = _models()
    trace = _trace(models, 12, seed=21)
    items, refs = [], []
    for name, T, P, Y in trace:
        g = models[name]
        Td, Pd, Yd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, Y))
        N = g.n_species
        items.append((g, Td, Pd, Yd, torch.empty((len(T), N + 1, N + 1), dtype=torch.float64, device="cuda")))
        refs.append(g.eval_jacobian(Td, Pd, Yd))
    nb = pj.batch_workspace_bytes()
    ws = [torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    torch.cuda.synchronize()
    pj.run_batch(items[:6], workspace=ws[0], stream=streams[0])
    pj.run_batch(items[6:], workspace=ws[1], stream=streams[1])
    torch.cuda.synchronize()
    for it, ref in zip(items, refs):
        assert torch.equal(it[4], ref)
    for it in items:
        it[4].zero_()
    pj.run_batch(items)                               # the static array
    torch.cuda.synchronize()
    for it, ref in zip(items, refs):
        assert torch.equal(it[4], ref)
    with pytest.raises(pj.LibraryError):
        pj.run_batch(items, workspace=ws[0][:16])      # too small


@pytest.mark.parametrize("host", [False, True])
def test_chunked_request_equals_unchunked_result(host):
    """A large request cut into chunks (each launch writing its slice of the output, chunks on
    several streams, small requests admitted between them) returns the plain launch's bits, with
    the source terms beside the Jacobian, on the device or copied to host memory."""
    from paper_1605_03262_b300.serving import Server
    models = _models()
    big = synth.CONFIGS[1]["name"]
    N = models[big].n_species
    T, P, Y = synth.generate_states(N, 3000, seed=61)
    small = _trace(models, 8, seed=62)
    with Server(models, max_inflight=4, chunk_ms=0.05, host_results=host) as srv:
        f_big = srv.submit(big, T, P, Y, dydt=True)
        f_small = [srv.submit(*r) for r in small]
        J, F = f_big.result(timeout=120)
        rest = [f.result(timeout=120) for f in f_small]
        stats = dict(srv.stats)
    assert stats["chunked_requests"] >= 1 and stats["chunks"] > 2
    Jr, Fr = models[big].eval_jacobian(*(torch.as_tensor(a, device="cuda") for a in (T, P, Y)), dydt=True)
    J, F = torch.as_tensor(J).cuda(), torch.as_tensor(F).cuda()
    assert torch.equal(J, Jr) and torch.equal(F, Fr)
    for (name, Ts, Ps, Ys), res in zip(small, rest):
        ref = models[name].eval_jacobian(*(torch.as_tensor(a, device="cuda") for a in (Ts, Ps, Ys)))
        assert torch.equal(torch.as_tensor(res).cuda(), ref)
    # the big request did not hold the small ones back until its end: some finished before it
    assert min(f.request.t_done for f in f_small) <= f_big.request.t_done



def test_input_kinds_give_the_same_results():
    """Requests given as numpy arrays (float64 or float32), pageable or pinned host tensors, or
    CUDA tensors return the plain launch's bits, in launches that merge host inputs only, device
    inputs only, both kinds, or hold a single request (host or device)."""
    from paper_1605_03262_b300.serving import Server
    models = _models()
    name = synth.CONFIGS[1]["name"]
    N = models[name].n_species
    kinds = {"numpy": lambda a: a, "numpy32": lambda a: a.astype(np.float32),
             "pageable": lambda a: torch.from_numpy(a), "pinned": lambda a: torch.from_numpy(a).pin_memory(),
             "cuda": lambda a: torch.as_tensor(a, device="cuda")}
    phases = [["numpy", "pageable", "pinned", "numpy32"], ["cuda", "cuda", "cuda"],
              ["cuda", "numpy", "pinned", "cuda"], ["pinned"], ["cuda"]]
    seed = 300
    for phase in phases:
        reqs = []
        for kind in phase:
            seed += 1
            T, P, Y = synth.generate_states(N, 5 + seed % 37, seed=seed)
            if kind == "numpy32":
                T, P, Y = (a.astype(np.float32).astype(np.float64) for a in (T, P, Y))
            reqs.append(((T, P, Y), tuple(kinds[kind](np.ascontiguousarray(a)) for a in (T, P, Y))))
        srv = Server(models, max_inflight=1)
        futs = [srv.submit(name, *given) for _, given in reqs]   # queued before the loop starts
        srv.start()
        try:
            res = [f.result(timeout=120) for f in futs]
        finally:
            srv.stop()
        assert srv.stats["merged_requests"] == len(reqs) - 1   # one launch for the phase
        for ((T, P, Y), _), J in zip(reqs, res):
            ref = models[name].eval_jacobian(*(torch.as_tensor(a, device="cuda") for a in (T, P, Y)))
            assert torch.equal(J, ref)


def test_chunked_requests_proceed_while_a_new_one_waits_for_memory():
    """With room for two large requests, four of them cut into chunks that rotate through the
    queue: when a request that has not started waits for memory at the head of the queue, the
    started ones still get their next chunks (they free the memory it waits for), and all four
    complete with the plain launch's results."""
    from paper_1605_03262_b300.serving import Server
    models = _models()
    name = synth.CONFIGS[1]["name"]
    N = models[name].n_species
    n = 2000
    per_request = Server._bytes(models[name], n)
    reqs = [synth.generate_states(N, n, seed=400 + k) for k in range(4)]
    srv = Server(models, hbm_budget=int(2.5 * per_request), max_inflight=2, chunk_ms=0.02)
    srv.start()
    try:
        futs = [srv.submit(name, *r) for r in reqs]
        res = [f.result(timeout=60) for f in futs]
        stats = dict(srv.stats)
    finally:
        srv.stop(drain=False)
    assert stats["chunked_requests"] == 4 and stats["waits_for_memory"] > 0
    for (T, P, Y), J in zip(reqs, res):
        ref = models[name].eval_jacobian(*(torch.as_tensor(a, device="cuda") for a in (T, P, Y)))
        assert torch.equal(J, ref)
