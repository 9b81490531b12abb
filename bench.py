#!/usr/bin/env python
"""Benchmark: batched FP64 analytical Jacobians per second on B300 (pyJac method, arXiv:1605.03262).

One step = one pass of the whole hot path over one batch: thermodynamics, rate coefficients and
rates of every reaction, the per-reaction Jacobian terms, the species gathers and the dense
(N+1)^2 Jacobian of every state, written to HBM (one kernel launch through the C ABI).

Workload of the headline line: synthetic 53-species, 325-reaction model (5 elements; 70 %
Arrhenius, 15 % third-body, 12 % Troe/Lindemann falloff, 3 % SRI; all reversible through the
equilibrium constant) and 65,536 states (T uniform 800-2500 K, P log-uniform 1-50 atm,
Y ~ Dirichlet(0.5)), FP64. The same line carries the other three model sizes under "per_config".

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU runs are launched with torch.distributed.run; each rank evaluates its own batch of the
same size (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1605_03262_b300 import autotune, synth  # noqa: E402

METRIC = "Jacobians/sec (FP64, 1 B300) per mechanism size vs roofline; p50/p99 serving latency"
UNIT = "Jacobians/s"
HEADLINE_CFG = 1
L2_FLUSH_BYTES = 256 << 20


# ---------------------------------------------------------------------------------------------
# algorithmic FP64 work per Jacobian (the roofline numerator)

def _distinct(side):
    d = {}
    for s, nu in side:
        d[s] = d.get(s, 0) + nu
    return d


def _side_ops(nus, kc: bool) -> int:
    """FP64 operations of one side of a reaction: powers [X]^nu and their derivatives (none for
    nu = 1), the product and its partial derivatives (without the factors d[X]^nu/d[X] = 1 when every
    coefficient is 1), and the sums nu*B, nu*dB/dT (K_c only), nu*H."""
    ops = sum({1: 0, 2: 2, 3: 3}.get(v, 4) for v in nus)
    if all(v == 1 for v in nus):
        ops += {1: 0, 2: 1, 3: 4}.get(len(nus), 7)
    else:
        ops += {1: 0, 2: 3, 3: 7}.get(len(nus), 11)
    return ops + len(nus) * (3 if kc else 1)


def work_model(model) -> dict:
    """FP64 operations the formulation needs per Jacobian, by kind.

    arith: FP64 add/mul/FMA operations (each one FP64 pipe issue); exp, log, div: calls of the
    transcendental functions and divisions. The counts follow the evaluation order of the kernels
    (reaction terms once per reaction; a short path for elementary reactions, whose c = 1 and
    psi = 0; gathers through the static lists at one FMA per term per sum; one FMA per sparse
    contribution, the W_k/W_j scale folded into its coefficient; one FMA per dense entry) without
    padding, replicated reductions or comparisons. It is a property of the model, not of a
    measurement, and stays at or below the FP64 thread instructions ncu counts."""
    N, R = model.n_species, model.n_reactions
    # per state: 1/T, ln T, ln P, 1/sum(Y/W), P/(RT), rho, 1/cp, 1/rho, J00 and dydt_0
    arith, n_exp, n_log, n_div = 12.0, 0.0, 2.0, 5.0
    # per species: thermo (c_p, H, B, dB/dT, dc_p/dT), 3 mixture sums, [X], gather finish (5),
    # HS scale, energy sums (5)
    arith += N * (32 + 3 + 2 + 5 + 1 + 5)
    pairs = contributions = colent = 0
    nnz = set()
    for r in model.reactions:
        reac, prod = _distinct(r.reac), _distinct(r.prod)
        kc = r.rev_mode == synth.REV_KC
        elem = r.kind == synth.KIND_ELEMENTARY
        net = {}
        for sp, nu in reac.items():
            net[sp] = net.get(sp, 0) - nu
        for sp, nu in prod.items():
            net[sp] = net.get(sp, 0) + nu
        net = [sp for sp, v in net.items() if v != 0]
        slots = set(reac) | set(prod)
        neff = 0
        if r.kind in (synth.KIND_THIRD_BODY, synth.KIND_FALLOFF, synth.KIND_CHEM):
            if r.tb_mode == synth.TB_SPECIES:
                slots.add(r.tb_species)
            else:
                slots |= {sp for sp, a in r.eff if a != 1.0}
                neff = len(r.eff) + 1                       # efficiency terms and M = C_tot + sum
        a = _side_ops(list(reac.values()), kc) + _side_ops(list(prod.values()), kc)
        if kc:
            a += 5                                          # ln K_c, k_r argument, d ln k_r / dT
            n_exp += 1
        elif r.rev_mode == synth.REV_EXPLICIT:
            a += 4
            n_exp += 1
        a += 3 + 4 + 2 + 1                                  # R_f, R_r, R; dR/dT; sigma; dH
        nside = sum((sp in reac) + (sp in prod) for sp in slots)
        if elem:
            a += 2 + nside                                  # theta, a; b' slots
        else:
            a += 1 + 3 + 4 + 3 + nside + len(slots)         # q, theta, a, c k_f / c k_r / psi R; b' slots
        if r.kind in (synth.KIND_ELEMENTARY, synth.KIND_THIRD_BODY):
            a += 4                                          # ln k_f, d ln k_f / dT
            n_exp += 1
            if r.kind == synth.KIND_THIRD_BODY:
                a += neff + 1                               # [M], dc/dT
        elif r.kind in (synth.KIND_FALLOFF, synth.KIND_CHEM):
            a += 8 + neff + 2 + 1 + 4                       # k_0, k_inf (+ derivatives), [M], Pr, 1 + Pr, dc/dT
            n_exp += 2                                      # k_0 / k_inf, k_f
            n_div += 1
            if r.ftype == synth.F_TROE:
                a += 32 + (6 if r.troe_has_T2 else 0)
                n_exp += 3 + (1 if r.troe_has_T2 else 0)
                n_log += 2
                n_div += 3
            elif r.ftype == synth.F_SRI:
                a += 21
                n_exp += 3
                n_log += 2
                n_div += 2
            if r.kind == synth.KIND_CHEM:
                a += 5
                n_div += 1
            else:
                a += 6
        elif r.kind == synth.KIND_PLOG:
            a += 16
            n_exp += 1
            n_div += 1
        else:
            nt, npc = r.cheb_shape
            a += 3 * nt * npc + 7 * nt + 11
            n_exp += 1
        arith += a
        pairs += len(net)
        colent += len(slots)
        for k in net:
            for l in slots:
                nnz.add((k, l))
                contributions += 1
    # gathers: omega, theta and A sums (3 per reaction-species pair), column sums (1 per reaction
    # slot), sparse block and C_k (1 per contribution)
    arith += 3 * pairs + colent + contributions
    arith += N * (N - 1) + 5 * (N - 1)                      # dense species block, energy row
    return {"arith": arith, "exp": n_exp, "log": n_log, "div": n_div, "nnz": len(nnz),
            "contributions": contributions}


# FP64 operations of one call of the table-driven exp and log (Tang's methods, as implemented):
# range reduction, polynomial and reconstruction. Division is weighted by its measured throughput.
EXP_OPS, LOG_OPS = 9.0, 12.0


def dfma_equivalents(work: dict, ratios: dict) -> float:
    """FP64-pipe time per Jacobian in units of one FMA issue: arithmetic ops, exp and log at the
    operation counts of the table-driven algorithms, division at its measured cost relative to FMA."""
    return work["arith"] + work["exp"] * EXP_OPS + work["log"] * LOG_OPS + work["div"] * ratios["div"]


# ---------------------------------------------------------------------------------------------
# measurement helpers

def calibrate():
    """Measured FP64 FMA peak, exp/log/div cost in FMA issues, store-only bandwidth."""
    from paper_1605_03262_b300 import build as pjbuild
    lib = ctypes.CDLL(pjbuild.build_calib())
    lib.pjc_fp64_fma_tflops.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.pjc_fp64_func_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.pjc_store_gbs.argtypes = [ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)]
    tf = ctypes.c_double()
    best_tf = 0.0
    for _ in range(3):
        if lib.pjc_fp64_fma_tflops(4096, ctypes.byref(tf)) == 0:
            best_tf = max(best_tf, tf.value)
    fma_rate = best_tf * 1e12 / 2.0
    ratios = {}
    for op, name in ((0, "exp"), (1, "log"), (2, "div")):
        r = ctypes.c_double()
        best = 0.0
        for _ in range(2):
            if lib.pjc_fp64_func_rate(op, 256, ctypes.byref(r)) == 0:
                best = max(best, r.value)
        ratios[name] = fma_rate / best if best > 0 else float("nan")
    g = ctypes.c_double()
    gbs = 0.0
    for _ in range(2):
        if lib.pjc_store_gbs(4 << 30, ctypes.byref(g)) == 0:
            gbs = max(gbs, g.value)
    return {"fp64_tflops": best_tf, "ratios": ratios, "store_gbs": gbs}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except ValueError:
                pass
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        out.update(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")


def kernel_source_hash() -> str:
    """SHA-1 of the CUDA sources of the library (a stored DRAM measurement is valid only for them)."""
    import hashlib
    d = os.path.join(ROOT, "paper_1605_03262_b300", "csrc")
    h = hashlib.sha1()
    for fn in sorted(os.listdir(d)):
        if fn.endswith((".cu", ".cuh", ".h")) and fn != "pj_calib.cu":
            with open(os.path.join(d, fn), "rb") as f:
                h.update(fn.encode() + b"\0" + f.read())
    return h.hexdigest()


def stored_traffic(cfg: int, n_states: int):
    """DRAM bytes (read + write) per launch of the Jacobian kernel from the committed ncu capture,
    scaled to n_states (traffic grows in proportion to the states), or None when the capture was
    taken on other kernel sources or another workload."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    ent = rec.get("captures", {}).get(synth.CONFIGS[cfg]["name"])
    if not ent or rec.get("kernel_source_sha1") != kernel_source_hash():
        return None
    return (ent["dram_bytes_read"] + ent["dram_bytes_write"]) / ent["n_states"] * n_states


def _reduce_device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def _max_over_ranks(ws, x: float) -> float:
    """Largest value over the ranks (the step time that counts for the whole job)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(ws, x: float) -> float:
    """Sum over the ranks (states processed by the whole job)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_states(cfg: int, rank: int, n_states=None):
    """The batch a rank evaluates: the configuration's state count, its own seeded draw (weak
    scaling: every rank owns a full-size batch, no data is exchanged)."""
    return synth.config_states(cfg, n_states, seed_offset=1000 + rank)


def workload_name(cfg: int) -> str:
    c = synth.CONFIGS[cfg]
    return "%s: %d states, synthetic %d-species %d-reaction model" % (c["name"], c["n_states"], c["n_species"],
                                                                     c["n_reactions"])


# ---------------------------------------------------------------------------------------------
# the CUDA arm

def specialise(g) -> dict:
    """Compile the model's specialised kernels (NVRTC); if that fails, the data-driven kernels (the
    same GPU arithmetic, the same bits) stay in use and the reason is reported."""
    try:
        return dict(g.specialize(), ok=True)
    except Exception as e:                 # NVRTC missing or failing: keep the data-driven kernels
        return {"ok": False, "error": str(e), "compile_seconds": 0.0, "cubin_bytes": 0}


def host_slack():
    """About 0.1 ms of a spinning GPU kernel before a timed launch: the host then enqueues the
    launch while the GPU is still busy, so the start event does not fire on an idle GPU that waits
    for the host (on kernels of tens of microseconds, the binding's argument checks and the C ABI's
    pointer checks otherwise land inside the timed interval, more so while the host is loaded)."""
    import torch
    torch.cuda._sleep(200000)


def time_device(g, Td, Pd, Yd, J, steps, warmup, flush):
    """Per-step CUDA-event time of the Jacobian launch, L2 flushed before every step."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.zero_()
        g.eval_jacobian(Td, Pd, Yd, out=J, stream=stream)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):                  # enqueued ahead of the GPU: no host gap before a start
        flush.zero_()
        starts[k].record(stream)
        g.eval_jacobian(Td, Pd, Yd, out=J, stream=stream)
        ends[k].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def run_config(cfg, steps, warmup, rank, cal, n_states=None, launch=None):
    import torch
    import paper_1605_03262_b300 as pj
    model = synth.config_model(cfg)
    T, P, Y = shard_states(cfg, rank, n_states)
    n, N = Y.shape
    blob = synth.to_bytes(model)
    g = pj.Model(blob)
    Td, Pd, Yd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, Y))
    # tune on the workload itself when its output fits a 2 GB probe (a small batch wants another
    # shape than a large one), else on the tuner's synthetic batch
    own = n * (N + 1) ** 2 * 8 <= (2 << 30)
    if launch:                                       # a fixed shape (--launch): no tuner launches
        g.set_launch(*launch)
        tune = {"n_probe": 0}
    else:
        tune = autotune.autotune(g, blob, use_cache=False, probe=(Td, Pd, Yd) if own else None)
    J = torch.empty((n, N + 1, N + 1), dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.float64, device="cuda")
    # the data-driven kernel, then the kernel specialised for this model and shape (NVRTC), which
    # the result reports: same bits, sizes and offsets compiled in
    ms_dd = time_device(g, Td, Pd, Yd, J, max(3, steps // 2), warmup, flush)
    spec = specialise(g)
    ms = time_device(g, Td, Pd, Yd, J, steps, warmup, flush)
    work = work_model(model)
    dfe = dfma_equivalents(work, cal["ratios"])
    ms_mean = float(np.mean(ms))
    achieved = 2.0 * dfe * n / (ms_mean * 1e-3) / 1e12
    fixed = bool(launch)
    launch = g.get_launch()
    res = {
        "n_states": n, "n_species": N, "n_reactions": model.n_reactions, "ms_per_step": ms_mean,
        "ms_min": float(np.min(ms)), "ms_median": float(np.median(ms)), "jacobians_per_s": n / (ms_mean * 1e-3),
        "fp64_dfma_equiv_per_jacobian": dfe, "work": work,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": cal["fp64_tflops"], "unit": "TFLOP/s",
                     "frac": achieved / cal["fp64_tflops"] if cal["fp64_tflops"] else None},
        "hbm_write_gbs": n * (N + 1) ** 2 * 8 / (ms_mean * 1e-3) / 1e9,
        "launch": {"warps_per_state": launch[0], "states_per_cta": launch[1], "ctas_per_sm": launch[2],
                   "chosen_by": ("fixed (--launch)" if fixed else
                                 "autotuner (%d probe states)" % tune.get("n_probe", 0))},
        "kernel": ("specialised for the model at run time (NVRTC, pj_mech_specialize)" if spec["ok"] else
                   "data-driven (specialisation failed: %s)" % spec["error"]),
        "specialisation": {"compile_s": spec["compile_seconds"], "cubin_bytes": spec["cubin_bytes"],
                           "data_driven_ms_median": float(np.median(ms_dd)),
                           "specialised_over_data_driven": float(np.median(ms)) / float(np.median(ms_dd))},
    }
    # sampled rows of the last timed launch's output, for the parity report of the CPU-baseline leg
    idx = np.unique(np.linspace(0, n - 1, min(n, PARITY_SAMPLE[cfg])).astype(np.int64))
    res["_parity_sample"] = (idx, J[torch.as_tensor(idx, device="cuda")].cpu().numpy())
    del J, flush
    return res, (g, model, T, P, Y, Td, Pd, Yd)


# states per model whose Jacobians from the timed launch are compared with the oracle (evenly
# spaced over the batch): about a second of oracle time each on 16 host cores
PARITY_SAMPLE = {0: 1024, 1: 1024, 2: 512, 3: 256}

FD_WORKSPACE_BYTES = 4 << 30


def fd_form(per_config: dict, steps: int, warmup: int):
    """The paper's finite-difference comparison on this GPU (Section 5.2): first-order forward-
    difference Jacobians from the library's source-term kernel, timed like the analytical ones on
    the same states; reports FD time / analytical time per model (the paper's Table of GPU
    ratios)."""
    import torch
    import paper_1605_03262_b300 as pj
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.float64, device="cuda")
    for cfg in (0, 1, 2, 3):
        name = synth.CONFIGS[cfg]["name"]
        if name not in per_config:
            continue
        model = synth.config_model(cfg)
        n = per_config[name]["n_states"]
        T, P, Y = synth.config_states(cfg, n)
        g = pj.Model(synth.to_bytes(model))
        Td, Pd, Yd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, Y))
        N = model.n_species
        J = torch.empty((n, N + 1, N + 1), dtype=torch.float64, device="cuda")
        ws = torch.empty(min(g.fd_workspace_bytes(n), FD_WORKSPACE_BYTES), dtype=torch.uint8, device="cuda")
        for _ in range(warmup):
            flush.zero_()
            g.eval_jacobian_fd(Td, Pd, Yd, out=J, workspace=ws)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            host_slack()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            g.eval_jacobian_fd(Td, Pd, Yd, out=J, workspace=ws)
            e.record()
            torch.cuda.synchronize()
            ms.append(s.elapsed_time(e))
        fd_ms = float(np.median(ms))
        an_ms = per_config[name]["ms_median"]
        out[name] = {"n_states": n, "fd_ms": fd_ms, "fd_jacobians_per_s": n / (fd_ms * 1e-3),
                     "analytic_ms": an_ms, "fd_over_analytic": fd_ms / an_ms,
                     "workspace_bytes": ws.numel()}
        del J, ws
        torch.cuda.empty_cache()
    del flush
    return out


def dydt_form(per_config: dict, steps: int, warmup: int):
    """The source terms alone (Eqs. e:ode and e:dTdt, the call an ODE solver makes most often) on
    the same states: launch shape tuned for this kernel, the kernel specialised for the model,
    timed like the Jacobian (L2 flushed before each step). Per state it reads T, P and Y and
    writes the N + 1 rates."""
    import torch
    import paper_1605_03262_b300 as pj
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.float64, device="cuda")
    for cfg in (0, 1, 2, 3):
        name = synth.CONFIGS[cfg]["name"]
        if name not in per_config:
            continue
        model = synth.config_model(cfg)
        n = per_config[name]["n_states"]
        T, P, Y = synth.config_states(cfg, n)
        blob = synth.to_bytes(model)
        g = pj.Model(blob)
        Td, Pd, Yd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, Y))
        N = model.n_species
        autotune.autotune(g, blob, which="dydt", use_cache=False, probe=(Td, Pd, Yd))
        spec = specialise(g)
        F = torch.empty((n, N + 1), dtype=torch.float64, device="cuda")
        for _ in range(warmup):
            flush.zero_()
            g.eval_dydt(Td, Pd, Yd, out=F)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            host_slack()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            g.eval_dydt(Td, Pd, Yd, out=F)
            e.record()
            torch.cuda.synchronize()
            ms.append(s.elapsed_time(e))
        d_ms = float(np.median(ms))
        lc = g.get_launch("dydt")
        out[name] = {"n_states": n, "ms": d_ms, "evaluations_per_s": n / (d_ms * 1e-3),
                     "bytes_per_state": 8 * (N + 2) + 8 * (N + 1),
                     "launch": {"warps_per_state": lc[0], "states_per_cta": lc[1], "ctas_per_sm": lc[2]},
                     "kernel": "specialised (NVRTC)" if spec["ok"] else "data-driven",
                     "jacobian_ms": per_config[name]["ms_median"],
                     "dydt_over_jacobian": d_ms / per_config[name]["ms_median"]}
        del F, g
        torch.cuda.empty_cache()
    return out


def cv_form(per_config: dict, steps: int, warmup: int):
    """The constant-volume form (Section 3.3) on the same states at their densities, in the same
    launch shape and kernel kind (specialised) as the constant-pressure Jacobian, timed like it (L2
    flushed before each step)."""
    import torch
    import paper_1605_03262_b300 as pj
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.float64, device="cuda")
    for cfg in (0, 1, 2, 3):
        name = synth.CONFIGS[cfg]["name"]
        if name not in per_config:
            continue
        model = synth.config_model(cfg)
        n = per_config[name]["n_states"]
        T, P, Y = synth.config_states(cfg, n)
        W = np.array([s.W for s in model.species])
        rho = P / (synth.R_GAS * T * (Y / W).sum(axis=1))
        g = pj.Model(synth.to_bytes(model))
        lc = per_config[name]["launch"]
        g.set_launch(lc["warps_per_state"], lc["states_per_cta"], lc["ctas_per_sm"])
        specialise(g)
        Td, rd, Yd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, rho, Y))
        N = model.n_species
        J = torch.empty((n, N + 1, N + 1), dtype=torch.float64, device="cuda")
        for _ in range(warmup):
            flush.zero_()
            g.eval_jacobian_cv(Td, rd, Yd, out=J)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            host_slack()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            g.eval_jacobian_cv(Td, rd, Yd, out=J)
            e.record()
            torch.cuda.synchronize()
            ms.append(s.elapsed_time(e))
        cv_ms = float(np.median(ms))
        cp_ms = per_config[name]["ms_median"]
        out[name] = {"n_states": n, "cv_ms": cv_ms, "cv_jacobians_per_s": n / (cv_ms * 1e-3),
                     "constant_pressure_ms": cp_ms, "cv_over_constant_pressure": cv_ms / cp_ms}
        del J
        torch.cuda.empty_cache()
    del flush
    return out


def conc_e2e(g, model, cfg: int, nnz: int, steps: int):
    """End to end through the Python API with host buffers, for the sparse concentration basis and
    the dense constant-pressure Jacobian on the same number of states (as many as keep the dense
    output within 2 GB): per step the pinned host inputs are copied to the device, the Jacobians
    evaluated, and the outputs copied back to pinned host memory, all inside the CUDA-event
    interval. The device-to-host copy (PCIe) bounds both, so the smaller sparse output shows here."""
    import torch
    N = model.n_species
    n = int(min(synth.CONFIGS[cfg]["n_states"], (2 << 30) // (8 * (N + 1) ** 2)))
    T, P, Y = synth.config_states(cfg, n)
    Tc, Pc, Vc, nc = synth.config_conc_states(cfg, n)
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
    hT, hP, hY, hTc, hPc, hVc, hnc = (pin(a) for a in (T, P, Y, Tc, Pc, Vc, nc))
    dT, dP, dY, dTc, dPc, dVc, dnc = (torch.empty_like(h, device="cuda") for h in (hT, hP, hY, hTc, hPc, hVc, hnc))
    dJ = torch.empty((n, N + 1, N + 1), dtype=torch.float64, device="cuda")
    hJ = torch.empty((n, N + 1, N + 1), dtype=torch.float64).pin_memory()
    dv = torch.empty((n, nnz), dtype=torch.float64, device="cuda")
    hv = torch.empty((n, nnz), dtype=torch.float64).pin_memory()

    def dense():
        for d, h in ((dT, hT), (dP, hP), (dY, hY)):
            d.copy_(h, non_blocking=True)
        g.eval_jacobian(dT, dP, dY, out=dJ)
        hJ.copy_(dJ, non_blocking=True)

    def sparse():
        for d, h in ((dTc, hTc), (dPc, hPc), (dVc, hVc), (dnc, hnc)):
            d.copy_(h, non_blocking=True)
        g.eval_jacobian_conc(dTc, dPc, dVc, dnc, out=dv)
        hv.copy_(dv, non_blocking=True)

    res = {"n_states": n}
    for key, fn, nbytes in (("dense_constant_pressure", dense, 8 * (N + 1) ** 2),
                            ("concentration_basis", sparse, 8 * nnz)):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(max(3, steps)):
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record()
            fn()
            e_.record()
            torch.cuda.synchronize()
            ms.append(s_.elapsed_time(e_))
        t = float(np.median(ms))
        res[key] = {"ms": t, "jacobians_per_s": n / (t * 1e-3), "d2h_bytes_per_state": nbytes}
    res["concentration_over_dense_throughput"] = (res["concentration_basis"]["jacobians_per_s"] /
                                                  res["dense_constant_pressure"]["jacobians_per_s"])
    del dJ, hJ, dv, hv
    torch.cuda.empty_cache()
    return res


def conc_form(per_config: dict, steps: int, warmup: int):
    """The molar-concentration basis at constant pressure (state T, V, n_1..n_{N-1}), written as a
    sparse Jacobian: the same numbers of states as the constant-pressure Jacobian, at its launch
    shape, with the kernel specialised for the model like it, L2 flushed before each step. Reports
    the pattern's size, the bytes written per state against the dense (N+1)^2, and the time against
    the constant-pressure Jacobian on the same batch size."""
    import torch
    import paper_1605_03262_b300 as pj
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.float64, device="cuda")
    for cfg in (0, 1, 2, 3):
        name = synth.CONFIGS[cfg]["name"]
        if name not in per_config:
            continue
        model = synth.config_model(cfg)
        N = model.n_species
        n = per_config[name]["n_states"]
        T, P, V, nmol = synth.config_conc_states(cfg, n)
        g = pj.Model(synth.to_bytes(model))
        lc = per_config[name]["launch"]
        g.set_launch(lc["warps_per_state"], lc["states_per_cta"], lc["ctas_per_sm"])
        specialise(g)
        rp, ci = g.conc_pattern()
        nnz = len(ci)
        Td, Pd, Vd, nd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, V, nmol))
        vals = torch.empty((n, nnz), dtype=torch.float64, device="cuda")
        for _ in range(warmup):
            flush.zero_()
            g.eval_jacobian_conc(Td, Pd, Vd, nd, out=vals)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            host_slack()
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_.record()
            g.eval_jacobian_conc(Td, Pd, Vd, nd, out=vals)
            e_.record()
            torch.cuda.synchronize()
            ms.append(s_.elapsed_time(e_))
        c_ms = float(np.median(ms))
        cp_ms = per_config[name]["ms_median"]
        e2e = conc_e2e(g, model, cfg, nnz, steps)
        out[name] = {"n_states": n, "nnz_per_state": nnz, "density": nnz / (N + 1) ** 2,
                     "species_block_density": (nnz - 2 * (N + 1) - 2 * (N - 1)) / (N - 1) ** 2,
                     "bytes_written_per_state": 8 * nnz, "dense_bytes_per_state": 8 * (N + 1) ** 2,
                     "ms": c_ms, "jacobians_per_s": n / (c_ms * 1e-3),
                     "hbm_write_gbs": n * nnz * 8 / (c_ms * 1e-3) / 1e9,
                     "constant_pressure_ms": cp_ms, "conc_over_constant_pressure": c_ms / cp_ms, "e2e": e2e}
        del vals
        torch.cuda.empty_cache()
    del flush
    return out


BATCH_MIX = ((0, 16384), (1, 65536), (2, 32768), (3, 2048))


def batched_form(steps: int, warmup: int):
    """The batched form against plain per-model launches on one mixed batch of the four model
    sizes: sequential plain launches (each model at its autotuned shape, its kernels specialised),
    one persistent batched launch with the default plan on the data-driven kernel, and the plan the
    batch autotuner picks with its kernel specialised for the four models; each plain and replayed
    from a CUDA graph. Same states and outputs in all of them. Then the same on 64 small requests."""
    import torch
    import paper_1605_03262_b300 as pj
    items, total = [], 0
    for cfg, n in BATCH_MIX:
        model = synth.config_model(cfg)
        blob = synth.to_bytes(model)
        g = pj.Model(blob)
        autotune.autotune(g, blob, use_cache=False)
        specialise(g)
        T, P, Y = synth.config_states(cfg, n, seed_offset=2000)
        Td, Pd, Yd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, Y))
        N = model.n_species
        J = torch.empty((n, N + 1, N + 1), dtype=torch.float64, device="cuda")
        items.append((g, Td, Pd, Yd, J))
        total += n
    flush = torch.empty(L2_FLUSH_BYTES // 8, dtype=torch.float64, device="cuda")

    def timed(fn):
        for _ in range(warmup):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            host_slack()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ms.append(s.elapsed_time(e))
        return float(np.median(ms))

    def forms(its, n_states):
        def plain():
            for g, Td, Pd, Yd, J in its:
                g.eval_jacobian(Td, Pd, Yd, out=J)

        plain_graph = torch.cuda.CUDAGraph()
        s_cap = torch.cuda.Stream()
        s_cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s_cap):
            plain()                        # warm-up outside the capture
            torch.cuda.synchronize()
            with torch.cuda.graph(plain_graph, stream=s_cap):
                for g, Td, Pd, Yd, J in its:
                    g.eval_jacobian(Td, Pd, Yd, out=J, stream=s_cap)
        torch.cuda.current_stream().wait_stream(s_cap)
        dflt = pj.BatchPlan(its)
        dflt_graph = dflt.capture()
        tuned, rep = autotune.autotune_batch(its, use_cache=False)
        tuned_graph = tuned.capture()
        out = {"requests": len(its), "total_states": n_states,
               "plain_sequential": {"ms": timed(plain), "launches": len(its), "kernels": "specialised per model"},
               "plain_graph": {"ms": timed(plain_graph.replay), "launches": len(its)},
               "batched_default": {"ms": timed(dflt.run), "graph_ms": timed(dflt_graph.replay), "launches": 1,
                                   "tiles": dflt.n_tiles, "kernel": "data-driven"},
               "batched_tuned": {"ms": timed(tuned.run), "graph_ms": timed(tuned_graph.replay), "launches": 1,
                                 "tiles": tuned.n_tiles, "choice": rep["choice"], "item_shapes": rep["item_shapes"],
                                 "tuning_ms": rep["timings"], "specialised_ms": rep["specialised_ms"],
                                 "specialised": rep["specialised"]}}
        for k in ("plain_sequential", "batched_default", "batched_tuned"):
            out[k]["jacobians_per_s"] = n_states / (out[k]["ms"] * 1e-3)
        del dflt, dflt_graph, tuned, tuned_graph, plain_graph
        return out

    out = {"mix": {synth.CONFIGS[c]["name"]: n for c, n in BATCH_MIX}}
    out.update(forms(items, total))

    # many small batches (the form's use: 64 requests of 16-1,024 states over the four models), one
    # persistent launch against 64 launches, plain or replayed from a graph
    rng = np.random.default_rng(17)
    small, stotal = [], 0
    for x in range(64):
        g = items[x % 4][0]
        n = int(np.exp(rng.uniform(np.log(16), np.log(1024))))
        N = g.n_species
        T, P, Y = synth.generate_states(N, n, seed=3000 + x)
        Td, Pd, Yd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, Y))
        small.append((g, Td, Pd, Yd, torch.empty((n, N + 1, N + 1), dtype=torch.float64, device="cuda")))
        stotal += n
    out["many_small"] = forms(small, stotal)
    del items, small, flush
    torch.cuda.empty_cache()
    return out


def _request_trace(models, n_req, seed):
    """Requests drawn uniformly from the models, each with log-uniform 1..4096 states (host arrays)."""
    rng = np.random.default_rng(seed)
    names = sorted(models)
    out = []
    for k in range(n_req):
        name = names[int(rng.integers(0, len(names)))]
        n = int(np.floor(np.exp(rng.uniform(0.0, np.log(4097.0)))))
        n = max(1, min(4096, n))
        out.append((name, *synth.generate_states(models[name].n_species, n, seed=seed * 100003 + k)))
    return out


def serving_form(seed: int = 7, open_loop_s: float = 2.0):
    """The serving form: continuous batching over the four resident models, against the plain
    per-mechanism launch (one request at a time, no merging, no overlap) on the same requests.
    Capacity = closed-loop throughput of a fixed trace (median of three runs); then Poisson arrivals
    at 0.5x and 0.8x that capacity (requests/s), with p50/p99 latency (submit -> result in device
    memory); then the same
    with every result copied to host memory (submit -> result in host memory) at half of the
    capacity measured with the copies. Requests above about 1 ms of GPU time are cut into chunks
    (the server's default); the plain per-request baseline cuts nothing. Every server first serves
    40 untimed warm-up requests (a long-running server is warm)."""
    import torch
    import paper_1605_03262_b300 as pj
    from paper_1605_03262_b300.serving import Server, latency_summary
    models = {}
    for cfg in (0, 1, 2, 3):
        blob = synth.to_bytes(synth.config_model(cfg))
        g = pj.Model(blob)
        autotune.autotune(g, blob, use_cache=False)
        specialise(g)
        models[synth.CONFIGS[cfg]["name"]] = g

    def run(trace, arrivals, warm=None, **kw):
        with Server(models, discard_results=True, **kw) as srv:
            if warm:                          # a running server is warm: its allocator and streams
                for f in [srv.submit(name, T, P, Y) for name, T, P, Y in warm]:
                    f.result(timeout=300)
                srv.stats.update({k: 0 for k in srv.stats})
            t0 = time.perf_counter()
            futs = []
            for (name, T, P, Y), ta in zip(trace, arrivals):
                dt = t0 + ta - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                futs.append(srv.submit(name, T, P, Y))
            for f in futs:
                f.result(timeout=300)
            wall = time.perf_counter() - t0
            stats = dict(srv.stats)
        states = sum(len(r[1]) for r in trace)
        out = {"requests": len(trace), "states": states, "wall_s": wall, "jacobians_per_s": states / wall}
        out.update(latency_summary([f.request for f in futs]))
        out["server"] = stats
        return out

    torch.cuda.synchronize()
    cap_trace = _request_trace(models, 160, seed)
    warm = _request_trace(models, 40, seed + 999)            # each server sees these first, untimed
    # capacity: the median of three closed-loop runs (one run of this 0.1 s trace varies by 10-20 %)
    caps = sorted((run(cap_trace, [0.0] * len(cap_trace), warm) for _ in range(3)), key=lambda r: r["wall_s"])
    cap = dict(caps[1], runs_jacobians_per_s=[c["jacobians_per_s"] for c in caps])
    cap_plain = run(cap_trace, [0.0] * len(cap_trace), warm, max_inflight=1, max_batch_states=1, chunk_ms=None)
    req_rate = cap["requests"] / cap["wall_s"]
    res = {"capacity_closed_loop": cap, "plain_per_request_closed_loop": cap_plain, "offered": {}}
    rng = np.random.default_rng(seed + 1)
    for frac in (0.5, 0.8):
        lam = frac * req_rate
        n_req = max(20, int(lam * open_loop_s))
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n_req))
        trace = _request_trace(models, n_req, seed + int(frac * 100))
        res["offered"]["%.1fx" % frac] = {
            "request_rate_per_s": lam,
            "continuous_batching": run(trace, arrivals, warm),
            "plain_per_request": run(trace, arrivals, warm, max_inflight=1, max_batch_states=1, chunk_ms=None),
        }
    # latency to results in host memory: the device-to-host copy (PCIe, ~56 GB/s) bounds that
    # capacity, so the open-loop run offers half of the capacity measured with the copies
    cap_host = run(cap_trace, [0.0] * len(cap_trace), warm, host_results=True)
    res["capacity_closed_loop_host"] = cap_host
    lam = 0.5 * cap_host["requests"] / cap_host["wall_s"]
    n_req = max(20, int(lam * open_loop_s))
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n_req))
    trace = _request_trace(models, n_req, seed + 70)
    res["offered_host"] = {"0.5x": {"request_rate_per_s": lam, "continuous_batching": run(trace, arrivals, warm,
                                                                                          host_results=True)}}
    torch.cuda.empty_cache()
    return res


def e2e_host(g, T, P, Y, steps):
    """End to end through the C ABI on pinned host buffers (copies inside the timed region)."""
    import torch
    n, N = Y.shape
    Th, Ph, Yh = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (T, P, Y))
    Jh = torch.empty((n, N + 1, N + 1), dtype=torch.float64).pin_memory()
    g.eval_jacobian_host(Th, Ph, Yh, Jh)      # warm-up (allocates staging)
    times = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.eval_jacobian_host(Th, Ph, Yh, Jh)
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    return {"value": n / t, "unit": UNIT, "h2d_bytes_per_step": int(n * (N + 2) * 8),
            "d2h_bytes_per_step": int(n * (N + 1) ** 2 * 8), "s_per_step": t}


EPS = 2.0 ** -52


def parity_report(gpu, ora, scale):
    """Tolerance report of the GPU Jacobians against the oracle's on the same states.

    Bar per entry: |x_gpu - x_oracle| <= 1e-10 max(|x_oracle|, 1e-20) + 64 eps S, S the oracle's sum
    of the absolute values of the terms of that entry. strict_fail counts entries that miss the
    plain 1e-10 relative bar (they pass only through the 64 eps S term, which covers the rounding
    of a cancelled sum), with the largest condition number kappa = S / |x| among them; well_cond
    are the entries with kappa <= 4500, where the bar is the plain relative one; bad = entries
    outside the bar (0 for parity). E_rel is the paper's per-state error norm (Section 5.1, Eq.
    e:error_norm): the Frobenius norm of elementwise relative errors over entries with
    |J| >= ||J||_F / 1e20; E_rel_well_cond_max is the largest E_rel over the well-conditioned
    entries alone (in an entry with kappa near 1/eps both sides hold rounding noise, which E_rel
    counts at full weight)."""
    gpu, ora, scale = (np.asarray(x, dtype=np.float64) for x in (gpu, ora, scale))
    finite = np.isfinite(gpu) & np.isfinite(ora)
    err = np.abs(gpu - ora)
    rel_bar = 1e-10 * np.maximum(np.abs(ora), 1e-20)
    ok = finite & (err <= rel_bar + 64.0 * EPS * scale)
    strict = finite & (err <= rel_bar)
    with np.errstate(over="ignore", divide="ignore", invalid="ignore"):
        kappa = np.where(np.abs(ora) > 0, scale / np.maximum(np.abs(ora), 1e-300), 0.0)
        rel = np.where(np.abs(ora) > 1e-20, err / np.maximum(np.abs(ora), 1e-20), 0.0)
    well = (kappa <= 4500.0) & (np.abs(ora) >= 1e-20)
    sf = ~strict & finite
    erel, erel_w = [], []
    for g_, o_, w_ in zip(gpu, ora, well):
        m = (np.abs(o_) >= np.linalg.norm(o_) / 1e20) & (o_ != 0)
        erel.append(float(np.linalg.norm((g_[m] - o_[m]) / o_[m])))
        m &= w_
        erel_w.append(float(np.linalg.norm((g_[m] - o_[m]) / o_[m])))
    erel, erel_w = np.array(erel), np.array(erel_w)
    return {"states": int(gpu.shape[0]), "entries": int(ora.size), "bad": int((~ok).sum()),
            "nonfinite": int((~finite).sum()), "strict_fail": int(sf.sum()),
            "strict_fail_max_kappa": float(kappa[sf].max()) if sf.any() else 0.0,
            "well_cond": int(well.sum()), "well_cond_max_rel": float(rel[well].max()) if well.any() else 0.0,
            "E_rel_median": float(np.median(erel)), "E_rel_max": float(erel.max()),
            "E_rel_well_cond_max": float(erel_w.max())}


def cpu_baseline(cfg, T, P, Y, sample=None, budget_s=12.0):
    """The oracle as it stands, on the host cores, on a bounded sample of the same workload (the
    first states of the batch the GPU evaluated), then on one core. With sample = (indices, GPU
    Jacobians of those states from the timed launch), the oracle's Jacobians of those states (with
    their rounding scales) give the parity report of that launch."""
    import oracle
    model = synth.config_model(cfg)
    om = oracle.load_model(synth.to_bytes(model))
    cores = oracle.max_threads()
    n0 = min(len(T), 4 * cores)
    t0 = time.perf_counter()
    om.jacobian(T[:n0], P[:n0], Y[:n0])
    per = (time.perf_counter() - t0) / n0
    ns = int(max(min(cores, len(T)), min(len(T), budget_s / max(per, 1e-9))))
    t0 = time.perf_counter()
    om.jacobian(T[:ns], P[:ns], Y[:ns])
    dt = time.perf_counter() - t0
    # the same oracle on one core, on a shorter sample
    oracle.set_threads(1)
    try:
        n1 = int(max(1, min(ns, budget_s / 4 / max(per * cores, 1e-9))))
        t1 = time.perf_counter()
        om.jacobian(T[:n1], P[:n1], Y[:n1])
        dt1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(cores)
    out = {"value": ns / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "first %d of the %d states of %s, oracle FP64 C with OpenMP over states"
                     % (ns, len(T), synth.CONFIGS[cfg]["name"]),
           "seconds": dt,
           "one_core": {"value": n1 / dt1, "unit": UNIT, "cores": 1, "sample": "first %d states" % n1,
                        "seconds": dt1}}
    if sample is not None:
        idx, Jg = sample
        Jo, _, Js, _ = om.jacobian(T[idx], P[idx], Y[idx], with_scale=True)
        out["parity"] = parity_report(Jg, Jo, Js)
    return out


def _sig(x, d=4):
    """x rounded to d significant digits (compact JSON)."""
    if x is None or not isinstance(x, (int, float)) or x == 0 or not math.isfinite(x):
        return x
    return float("%.*g" % (d, x))


def compact_config(res: dict, cpu: dict) -> dict:
    """One model's numbers for the JSON line: throughput, roofline fraction, step times, launch shape,
    the oracle on the host cores and the parity report of the timed launch."""
    lc = res["launch"]
    out = {"states": res["n_states"], "jacobians_per_s": _sig(res["jacobians_per_s"]),
           "frac": _sig(res["roofline"]["frac"], 3), "ms_median": _sig(res["ms_median"]),
           "ms_min": _sig(res["ms_min"]),
           "launch": "%dx%dx%d" % (lc["warps_per_state"], lc["states_per_cta"], lc["ctas_per_sm"]),
           "kernel": "specialised" if res["kernel"].startswith("specialised") else "data-driven"}
    if cpu:
        out["oracle_jacobians_per_s"] = _sig(cpu["value"])
        out["oracle_cores"] = cpu["cores"]
        if "parity" in cpu:
            p = cpu["parity"]
            out["parity"] = {k: (_sig(v, 3) if isinstance(v, float) else v) for k, v in p.items()}
    return out


def compact_forms(batched, serving, dyf, cvf, fd, concf) -> dict:
    """Headline numbers of the batched, serving, source-term, constant-volume, finite-difference and
    concentration-basis measurements (the full records go to the detail file)."""
    out = {}
    if batched:
        def one(b):
            return {"plain": _sig(b["plain_sequential"]["ms"]), "plain_graph": _sig(b["plain_graph"]["ms"]),
                    "default": _sig(b["batched_default"]["ms"]), "default_graph": _sig(b["batched_default"]["graph_ms"]),
                    "tuned": _sig(b["batched_tuned"]["ms"]), "tuned_graph": _sig(b["batched_tuned"]["graph_ms"]),
                    "tuned_choice": b["batched_tuned"]["choice"]}
        out["batched"] = {"mix_ms": one(batched), "small64_ms": one(batched["many_small"])}
    if serving:
        sv = {"capacity_jacobians_per_s": _sig(serving["capacity_closed_loop"]["jacobians_per_s"]),
              "plain_jacobians_per_s": _sig(serving["plain_per_request_closed_loop"]["jacobians_per_s"])}
        for k, v in serving["offered"].items():
            cb, pl = v["continuous_batching"], v["plain_per_request"]
            sv[k] = {"p50_ms": _sig(cb["p50_ms"], 3), "p99_ms": _sig(cb["p99_ms"], 3),
                     "plain_p50_ms": _sig(pl["p50_ms"], 3), "plain_p99_ms": _sig(pl["p99_ms"], 3)}
        if "capacity_closed_loop_host" in serving:
            h = serving["offered_host"]["0.5x"]["continuous_batching"]
            sv["host"] = {"capacity_jacobians_per_s": _sig(serving["capacity_closed_loop_host"]["jacobians_per_s"]),
                          "0.5x_p50_ms": _sig(h["p50_ms"], 3), "0.5x_p99_ms": _sig(h["p99_ms"], 3)}
        out["serving"] = sv
    if dyf:
        out["dydt_evals_per_s"] = {k: _sig(v["evaluations_per_s"], 3) for k, v in dyf.items()}
    if cvf:
        out["cv_over_cp_time"] = {k: _sig(v["cv_over_constant_pressure"], 3) for k, v in cvf.items()}
    if fd:
        out["fd_over_analytic_time"] = {k: _sig(v["fd_over_analytic"], 3) for k, v in fd.items()}
    if concf:
        out["conc_over_cp_time"] = {k: _sig(v["conc_over_constant_pressure"], 3) for k, v in concf.items()}
    return out


def detail_path(args):
    """Where the full measurement records go: --detail, else bench_detail.json in the working
    directory."""
    return args.detail if args.detail else os.path.join(os.getcwd(), "bench_detail.json")


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    cal = calibrate()
    gpu_index = torch.cuda.current_device()
    _barrier(ws)
    with ClockSampler(gpu_index) as clk:
        res, ctx = run_config(HEADLINE_CFG, args.steps, args.warmup, rank, cal,
                              launch=tuple(int(x) for x in args.launch.split(",")) if args.launch else None)
    clocks = clk.summary()
    g, model, T, P, Y = ctx[:5]
    torch.cuda.synchronize()
    _barrier(ws)
    ms_max = _max_over_ranks(ws, res["ms_per_step"])
    n_total = _sum_over_ranks(ws, float(res["n_states"]))
    value = n_total / (ms_max * 1e-3)
    e2e = e2e_host(g, T, P, Y, max(1, min(args.steps, 3))) if not args.no_e2e else None
    if e2e is not None and ws > 1:
        e2e["value"] = _sum_over_ranks(ws, e2e["value"])
    headline = synth.CONFIGS[HEADLINE_CFG]["name"]
    per_config, states = {headline: res}, {headline: (T, P, Y)}
    del ctx, g
    if not args.headline_only:
        for cfg in (0, 2, 3):
            r, c = run_config(cfg, max(3, args.steps // 2), args.warmup, rank, cal)
            per_config[synth.CONFIGS[cfg]["name"]] = r
            states[synth.CONFIGS[cfg]["name"]] = c[2:5]
            del c
            torch.cuda.empty_cache()
    batched = batched_form(max(3, args.steps // 2), args.warmup) if not args.headline_only else None
    fd = fd_form(per_config, 3, 1) if not (args.headline_only or args.no_fd) else None
    cvf = cv_form(per_config, max(3, args.steps // 2), args.warmup) if not args.headline_only else None
    dyf = dydt_form(per_config, max(3, args.steps // 2), args.warmup) if not args.headline_only else None
    concf = conc_form(per_config, max(3, args.steps // 2), args.warmup) if not args.headline_only else None
    serving = serving_form() if not (args.headline_only or args.no_serving) else None
    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    # the oracle on the host cores, per model, with the parity report of each timed launch
    cpu = {}
    if not args.no_cpu_baseline:
        for cfg in (0, 1, 2, 3):
            name = synth.CONFIGS[cfg]["name"]
            if name in per_config:
                cpu[name] = cpu_baseline(cfg, *states[name], sample=per_config[name]["_parity_sample"],
                                         budget_s=12.0 if cfg == HEADLINE_CFG else 4.0)
    roof = dict(res["roofline"])
    roof["traffic"] = stored_traffic(HEADLINE_CFG, res["n_states"])
    roof["traffic_unit"] = "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
    roof["algorithmic_bytes"] = res["n_states"] * (8 * (res["n_species"] + 1) ** 2 + 8 * (res["n_species"] + 2))
    roof["peak_source"] = "measured FP64 FMA throughput on this GPU in this run (libpjcalib)"
    # the line: the standard keys first, then the per-model numbers and the forms' headline numbers
    # (the end of the line is what a tail of the output keeps); full records in the detail file
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(HEADLINE_CFG), "model": headline,
                   "n_states_per_gpu": res["n_states"], "n_species": res["n_species"],
                   "n_reactions": res["n_reactions"], "parallelism": "states sharded over %d GPU(s)" % ws,
                   "l2": "flushed before every timed step (256 MB write)", "launch": res["launch"]},
        "roofline": roof,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "e2e": e2e,
        "calibration": {"fp64_tflops": _sig(cal["fp64_tflops"]), "store_gbs": _sig(cal["store_gbs"]),
                        "fma_per": {k: _sig(v, 3) for k, v in cal["ratios"].items()}},
    }
    if headline in cpu:
        line["cpu_baseline"] = {k: v for k, v in cpu[headline].items() if k != "parity"}
    line["forms"] = compact_forms(batched, serving, dyf, cvf, fd, concf)
    line["per_config"] = {name: compact_config(r, cpu.get(name)) for name, r in per_config.items()}
    dp = detail_path(args)
    if dp:
        detail = {"per_config": {k: {kk: vv for kk, vv in r.items() if kk != "_parity_sample"}
                                 for k, r in per_config.items()},
                  "cpu_baseline": cpu, "calibration": cal, "batched_form": batched, "fd_form": fd, "cv_form": cvf,
                  "dydt_form": dyf, "conc_form": concf, "serving_form": serving}
        with open(dp, "w") as f:
            json.dump(detail, f, indent=1)
        line["detail_file"] = os.path.relpath(dp, os.getcwd())
    print(json.dumps(line))
    sys.stdout.flush()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------------------------
# the reference arm: the oracle, timed on the host cores

def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cfg = HEADLINE_CFG
    model = synth.config_model(cfg)
    om = oracle.load_model(synth.to_bytes(model))
    cores = oracle.max_threads()
    T, P, Y = synth.config_states(cfg, 2 * cores)
    t0 = time.perf_counter()
    om.jacobian(T, P, Y)
    per = (time.perf_counter() - t0) / len(T)
    budget = 150.0 / max(1, args.steps + args.warmup)        # whole run within a few minutes
    ns = int(max(cores, min(synth.CONFIGS[cfg]["n_states"], budget / max(per, 1e-9))))
    T, P, Y = synth.config_states(cfg, ns)
    for _ in range(args.warmup):
        om.jacobian(T, P, Y)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        om.jacobian(T, P, Y)
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = ns / t
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": workload_name(cfg), "model": synth.CONFIGS[cfg]["name"],
                   "sample_states_per_step": ns},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "first %d of the %d states per step, oracle FP64 C with OpenMP over states"
                                   % (ns, synth.CONFIGS[cfg]["n_states"])},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# the autotuner's launch shapes of the four models (warps per state, states per CTA, CTAs per SM),
# fixed for profiling runs so that no tuning launches precede the profiled one
TUNED_SHAPES = {0: (1, 8, 2), 1: (2, 7, 1), 2: (4, 3, 1), 3: (16, 1, 1)}


def run_profile_batch(warmup: int, data_driven: bool = False):
    """--profile-batch -- the batched form for ncu: the 64 small requests of the benchmark's batched
    form (16-1,024 states each over the four models) as one plan of 512-thread CTAs with default
    tiles, its kernel specialised for the plan (--data-driven: the data-driven batched kernel);
    warm-up launches, then the profiled one."""
    import torch
    import paper_1605_03262_b300 as pj
    torch.cuda.set_device(0)
    models = []
    for cfg in (0, 1, 2, 3):
        g = pj.Model(synth.to_bytes(synth.config_model(cfg)))
        g.set_launch(*TUNED_SHAPES[cfg])
        models.append(g)
    rng = np.random.default_rng(17)
    items = []
    for x in range(64):
        g = models[x % 4]
        n = int(np.exp(rng.uniform(np.log(16), np.log(1024))))
        N = g.n_species
        T, P, Y = synth.generate_states(N, n, seed=3000 + x)
        Td, Pd, Yd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, Y))
        items.append((g, Td, Pd, Yd, torch.empty((n, N + 1, N + 1), dtype=torch.float64, device="cuda")))
    plan = pj.BatchPlan(items, threads_per_cta=512)
    if not data_driven:
        plan.specialize()
    for _ in range(warmup + 1):
        plan.run()
    torch.cuda.synchronize()
    print("profile case done: batched form, 64 requests, %d tiles, %s kernel" %
          (plan.n_tiles, "data-driven" if data_driven else "specialised"))


def run_profile_case(spec: str, warmup: int, data_driven: bool = False, conc: bool = False, dydt: bool = False):
    """--profile CFG:N[:WPS,GROUPS[,CTAS]] -- a small case for ncu: warm-up launches, then one Jacobian
    launch of the first N states of configuration CFG (inputs larger than L2 once N is a few
    thousand), at the given launch shape or else the autotuner's, with the kernel specialised for
    the model (the one the benchmark times; --data-driven for the other). The autotuner's own probe
    launches use a separate kernel instance count, so with an explicit shape the only launches
    are the warm-ups and the profiled one. --conc: the molar-concentration basis kernel instead;
    --dydt: the source-term kernel, at its own shape (the given one, else its tuner's)."""
    import torch
    import paper_1605_03262_b300 as pj
    parts = spec.split(":")
    cfg, n = int(parts[0]), int(parts[1])
    shape = tuple(int(x) for x in parts[2].split(",")) if len(parts) > 2 else None
    torch.cuda.set_device(0)
    model = synth.config_model(cfg)
    T, P, Y = synth.config_states(cfg, n, seed_offset=1000)
    blob = synth.to_bytes(model)
    g = pj.Model(blob)
    which = "dydt" if dydt else "jacobian"
    if shape:
        g.set_launch(shape[0], shape[1], shape[2] if len(shape) > 2 else 1, which=which)
    else:
        autotune.autotune(g, blob, which=which, use_cache=False)
    if not data_driven:
        specialise(g)
    if conc:
        Tc, Pc, Vc, nc = (torch.as_tensor(a, dtype=torch.float64, device="cuda")
                          for a in synth.config_conc_states(cfg, n))
        vals = torch.empty((n, len(g.conc_pattern()[1])), dtype=torch.float64, device="cuda")
        for _ in range(warmup + 1):
            g.eval_jacobian_conc(Tc, Pc, Vc, nc, out=vals)
        torch.cuda.synchronize()
        print("profile case done: concentration basis, cfg %d, %d states, launch %s" % (cfg, n, g.get_launch()))
        return
    Td, Pd, Yd = (torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in (T, P, Y))
    if dydt:
        F = torch.empty((n, model.n_species + 1), dtype=torch.float64, device="cuda")
        for _ in range(warmup + 1):
            g.eval_dydt(Td, Pd, Yd, out=F)
        torch.cuda.synchronize()
        print("profile case done: source terms, cfg %d, %d states, launch %s" % (cfg, n, g.get_launch("dydt")))
        return
    J = torch.empty((n, model.n_species + 1, model.n_species + 1), dtype=torch.float64, device="cuda")
    for _ in range(warmup + 1):
        g.eval_jacobian(Td, Pd, Yd, out=J)
    torch.cuda.synchronize()
    print("profile case done: cfg %d, %d states, launch %s" % (cfg, n, g.get_launch()))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--headline-only", action="store_true", help="skip the other model sizes")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-form measurement")
    ap.add_argument("--no-fd", action="store_true", help="skip the finite-difference comparison")
    ap.add_argument("--profile", default=None, metavar="CFG:N[:WPS,GROUPS[,CTAS]]", help="one small profiling case (for ncu)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="one batched launch of 64 small requests over the four models (for ncu)")
    ap.add_argument("--data-driven", action="store_true", help="with --profile: the data-driven kernel")
    ap.add_argument("--conc", action="store_true", help="with --profile: the molar-concentration basis kernel")
    ap.add_argument("--dydt", action="store_true", help="with --profile: the source-term kernel")
    ap.add_argument("--detail", default=None, metavar="PATH",
                    help="file for the full measurement records (default: bench_detail.json in the working "
                         "directory)")
    ap.add_argument("--launch", default=None, metavar="WPS,GROUPS,CTAS",
                    help="fixed launch shape of the headline model (skips the autotuner, e.g. for ncu runs)")
    args = ap.parse_args()
    if args.profile:
        return run_profile_case(args.profile, args.warmup, args.data_driven, args.conc, args.dydt)
    if args.profile_batch:
        return run_profile_batch(args.warmup, args.data_driven)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
