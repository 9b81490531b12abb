"""Launch-shape autotuner for the evaluation kernels.

A launch shape is (warps per state, states per CTA, CTAs per SM). Results are bitwise identical
for every shape (fixed-order reductions and per-lane schedules), so the tuner only times: it
evaluates a probe batch with each feasible shape and keeps the fastest. Choices are cached per
(model bytes, device name, kernel) in a JSON file (``$PYJAC_B300_CACHE`` or
``~/.cache/pyjac_b300/autotune.json``).
"""
from __future__ import annotations

import hashlib
import math
import json
import os
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

__all__ = ["candidate_shapes", "autotune", "cache_path", "batch_candidates", "autotune_batch"]

_lock = threading.Lock()

Shape = Tuple[int, int, int]


def cache_path() -> str:
    return os.environ.get("PYJAC_B300_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pyjac_b300", "autotune.json"))


def _load_cache() -> Dict[str, list]:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: Dict[str, list]) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".tmp.%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def candidate_shapes(model, which: str = "jacobian") -> List[Shape]:
    """Every (warps per state, states per CTA, CTAs per SM) the library accepts for this model:
    one CTA per SM of up to 512 threads, or two of up to 256 threads (the register file holds
    512 threads at the kernels' 128 registers)."""
    out = []
    for ctas in (1, 2):
        for wps in (1, 2, 4, 8, 16):
            for groups in range(1, 17):
                if wps * 32 * groups > 512 // ctas or (wps > 1 and groups > 15):
                    continue
                try:
                    model.launch_smem_bytes(wps, groups, ctas, which=which)
                    model.set_launch(wps, groups, ctas, which=which)
                except Exception:
                    continue
                out.append((wps, groups, ctas))
    return out


def _key(model, blob_digest: str, which: str) -> str:
    import torch
    name = torch.cuda.get_device_name(model.device)
    return "%s|%s|%s" % (blob_digest, name, which)


def autotune(model, blob: bytes, which: str = "jacobian", probe: Optional[Sequence] = None,
             n_probe: int = 0, reps: int = 2, use_cache: bool = True, shapes: Optional[List[Shape]] = None,
             refine: int = 4, refine_reps: int = 7) -> Dict[str, object]:
    """Time the candidate shapes on a probe batch, set the fastest on ``model`` and return a report.

    probe: optional (T, P, Y) device tensors; else a synthetic batch of n_probe states (default:
    enough states to fill every SM several times over) is drawn.
    refine: the fastest ``refine`` shapes of the first pass (back-to-back launches, warm L2) are
    timed again one launch at a time, each after a write larger than L2, and the lowest median of
    ``refine_reps`` launches wins. A batch small enough to sit in L2 ranks the shapes differently
    warm and cold, and two launches of a few tens of microseconds are too few to rank them."""
    import torch
    from . import synth
    digest = hashlib.sha1(blob).hexdigest()
    key = _key(model, digest, which)
    if use_cache and shapes is None:
        with _lock:
            hit = _load_cache().get(key)
        if hit:
            try:
                model.set_launch(*hit, which=which)
                return {"shape": tuple(hit), "cached": True}
            except Exception:
                pass
    cands = shapes if shapes is not None else candidate_shapes(model, which)
    if not cands:
        raise RuntimeError("no feasible launch shape for this model")
    if probe is None:
        sms = torch.cuda.get_device_properties(model.device).multi_processor_count
        n = n_probe or max(4096, sms * 16 * 8)
        N = model.n_species
        budget = 2 << 30                                          # keep the probe output under 2 GB
        n = max(sms, min(n, budget // (8 * (N + 1) ** 2)))
        T, P, Y = synth.generate_states(N, n, seed=12345)
        probe = tuple(torch.as_tensor(a, dtype=torch.float64, device=model.device) for a in (T, P, Y))
    T, P, Y = probe
    n, N = Y.shape[0], model.n_species
    out = (torch.empty((n, N + 1, N + 1), dtype=torch.float64, device=model.device) if which == "jacobian"
           else torch.empty((n, N + 1), dtype=torch.float64, device=model.device))
    fn = model.eval_jacobian if which == "jacobian" else model.eval_dydt
    timings = {}
    for shape in cands:
        model.set_launch(*shape, which=which)
        fn(T, P, Y, out=out)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            fn(T, P, Y, out=out)
        e.record()
        torch.cuda.synchronize()
        timings[shape] = s.elapsed_time(e) / reps
    best = min(timings, key=timings.get)
    refined = {}
    if refine > 1 and len(timings) > 1:
        l2 = torch.cuda.get_device_properties(model.device).L2_cache_size
        flush = torch.empty(max(2 * l2, 1 << 20) // 8, dtype=torch.float64, device=model.device)
        for shape in sorted(timings, key=timings.get)[:refine]:
            model.set_launch(*shape, which=which)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(refine_reps)]
            for s, e in ev:
                flush.zero_()
                s.record()
                fn(T, P, Y, out=out)
                e.record()
            torch.cuda.synchronize()
            refined[shape] = float(np.median([s.elapsed_time(e) for s, e in ev]))
        del flush
        best = min(refined, key=refined.get)
    model.set_launch(*best, which=which)
    if use_cache:
        with _lock:
            cache = _load_cache()
            cache[key] = list(best)
            _store_cache(cache)
    return {"shape": best, "cached": False, "ms": refined.get(best, timings[best]), "n_probe": n,
            "timings": {"%d,%d,%d" % k: v for k, v in sorted(timings.items(), key=lambda kv: kv[1])[:8]},
            "refined": {"%d,%d,%d" % k: v for k, v in sorted(refined.items(), key=lambda kv: kv[1])}}


# ---------------------------------------------------------------------------------------------
# the batched form: one persistent launch over items of several models

def batch_candidates(items, which: str = "jacobian") -> List[dict]:
    """Candidate plans for a batched launch: CTA sizes (512, 448 or 384 threads) and tiles of 1, 2, 4,
    8 or 16 rounds of each item's states per CTA (states per CTA from the model's tuned launch shape;
    the group width is the model's, halved by the library where a state does not fit the CTA, so
    that the candidates of one CTA size share one specialised kernel)."""
    out = []
    for threads in (512, 448, 384):
        base = []
        for it in items:
            wps, groups, _ = it[0].get_launch(which)
            base.append(max(1, min(groups, threads // (32 * wps))))
        for rounds in (1, 2, 4, 8, 16):
            # width 0: the model's own, halved by the library while a state does not fit the CTA
            out.append({"threads_per_cta": threads, "rounds": rounds,
                        "item_shapes": [(0, g, rounds * g) for g in base]})
    return out


def _mix_key(items, which: str) -> str:
    import torch
    parts = []
    for it in items:
        m = it[0]
        n = int(it[3].shape[0])
        parts.append("%d:%d:%s:%d" % (m.n_species, m.n_reactions, ",".join(map(str, m.get_launch(which))),
                                      int(math.log2(max(n, 1)))))
    return "batch|%s|%s|%s" % (torch.cuda.get_device_name(items[0][0].device), which, ";".join(parts))


TOP = 2   # batched candidates specialised after the data-driven ranking


def autotune_batch(items, which: str = "jacobian", specialise: bool = True, reps: int = 3,
                   use_cache: bool = True, candidates: Optional[List[dict]] = None):
    """Choose the batched launch's CTA size and per-item tile sizes for this item mix by timing
    candidate plans on the data-driven batched kernel (each run after a write larger than L2;
    median of ``reps``), then, with ``specialise``, the ``TOP`` fastest candidates again with their
    kernels specialised for the mix's models (NVRTC), keeping the fastest plan of all. Returns
    (plan, report).
    The choice is cached by the mix's shape (models' sizes and launch shapes, log2 of each item's
    state count)."""
    import torch
    from . import BatchPlan, LibraryError
    key = _mix_key(items, which)
    cands = candidates if candidates is not None else batch_candidates(items, which)
    hit = None
    if use_cache and candidates is None:
        with _lock:
            hit = _load_cache().get(key)
        if hit:
            cands = [c for c in cands if c["threads_per_cta"] == hit[0] and c["rounds"] == hit[1]] or cands
    if not cands:
        raise RuntimeError("no feasible batched launch for these items")
    l2 = torch.cuda.get_device_properties(items[0][0].device).L2_cache_size
    flush = torch.empty(max(2 * l2, 1 << 20) // 8, dtype=torch.float64, device=items[0][0].device)

    def time_plan(plan):
        plan.run()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for s, e in ev:
            flush.zero_()
            s.record()
            plan.run()
            e.record()
        torch.cuda.synchronize()
        return float(np.median([s.elapsed_time(e) for s, e in ev]))

    def name_of(c):
        return "%d threads, %d rounds per tile" % (c["threads_per_cta"], c["rounds"])

    timings, kept = {}, []                  # kept: the TOP fastest (time, candidate, plan)
    for c in cands:
        plan = BatchPlan(items, which=which, threads_per_cta=c["threads_per_cta"], item_shapes=c["item_shapes"])
        timings[name_of(c)] = time_plan(plan)
        kept.append((timings[name_of(c)], len(kept), c, plan))
        kept.sort(key=lambda x: (x[0], x[1]))
        for _, _, _, p in kept[TOP:]:
            p.close()
        kept = kept[:TOP]
    best_ms, _, choice, best_plan = kept[0]
    best = name_of(choice)
    spec_ms, spec_error = None, None
    use_spec = bool(hit[2]) if hit and len(hit) > 2 else None
    if specialise and use_spec is not False:
        # the kept candidates again with their kernels specialised (the ranking can change)
        spec_times = []
        for _, _, c, plan in kept:
            try:
                plan.specialize()
            except LibraryError as exc:  # NVRTC missing, or a plan it cannot specialise: data-driven
                spec_error = str(exc)
                break
            spec_times.append((time_plan(plan), c, plan))
        if spec_times:
            s_ms, s_c, s_plan = min(spec_times, key=lambda x: x[0])
            if use_spec is None:
                use_spec = s_ms < best_ms
            if use_spec:
                choice, best, best_plan, spec_ms = s_c, name_of(s_c), s_plan, s_ms
            else:
                spec_ms = spec_times[0][0]          # the fastest data-driven candidate's, specialised
        else:
            use_spec = False
        if not use_spec:
            best_plan.specialize(False)
    for _, _, _, plan in kept:
        if plan is not best_plan:
            plan.close()
    del flush
    if use_cache:
        with _lock:
            cache = _load_cache()
            cache[key] = [choice["threads_per_cta"], choice["rounds"], bool(use_spec)]
            _store_cache(cache)
    return best_plan, {"choice": best, "ms": spec_ms if use_spec else timings[best], "timings": timings,
                       "specialised_ms": spec_ms, "specialise_error": spec_error, "item_shapes": choice["item_shapes"],
                       "specialised": best_plan.spec_info()}
