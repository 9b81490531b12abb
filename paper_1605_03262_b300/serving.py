"""Serving form: a continuous-batching loop for Jacobian requests over several resident models.

Requests (model name, T, P, Y) arrive at any time through :meth:`Server.submit`, which returns a
future. A scheduler thread runs iterations continuously:

* retire: iterations whose completion event has fired hand their results to the futures and
  give back their device memory and stream;
* admit: queued requests are taken in arrival order. By default an iteration merges queued
  requests of the head's model into one plain launch (up to ``max_batch_states`` states), which
  runs the model's own (specialised, if compiled) kernel; with ``mixed=True`` an iteration takes up
  to 64 queued requests of any of the models and evaluates them in one persistent batched launch
  (pj_batch_run_ws, with a workspace per stream). On a trace of requests of 1-4,096 states over
  four models (closed loop, 160 requests, three runs) the merged iterations served 1.29-1.42 M
  Jacobians/s and the mixed ones 0.83-1.18 M/s: the streams already overlap the iterations, and
  the no-allocation batched launch runs the data-driven kernel (group width and sizes at run
  time), not the model's specialised one. An iteration is admitted only while an in-flight slot is free and the device memory it
  holds (inputs, Jacobians, dydt) fits the HBM budget next to the iterations already in flight;
  otherwise it waits in the queue (no out-of-memory, no rejection). Iterations run on a pool of
  streams, so requests admitted while others are on the GPU overlap with them.

A request whose estimated GPU time exceeds ``chunk_ms`` is cut into chunks of about that time
(consecutive states; the per-state time of each model is measured when the server starts). The
server admits one chunk of such a request at a time, each launch writing its slice of the
request's output, and sends the request to the back of the queue after each chunk, so a small
request that arrives behind a large one waits for at most one chunk instead of the whole request.
The request completes when its last chunk has. States are evaluated independently, so a chunked
result is bitwise the unchunked one. A request that has started holds its device memory until
its last chunk, so when the head of the queue waits for memory, the started requests behind it
still get their chunks (they are what frees the memory).

An iteration costs the scheduler thread 0.3-0.5 ms of host time (packing inputs into pinned
staging, allocations, the launch): on the four-model trace at 1,600 requests/s the thread is about
half busy and the GPU a little less.

Model images stay resident for the server's lifetime. Each request's latency is measured from
:meth:`submit` to the completion event of its iteration (results in device memory), and, with
``host_results=True``, to the end of the copy to host memory. The evaluation itself is the
library's Jacobian kernel, so a request's result is the same (bitwise) alone and in the mix.
"""
from __future__ import annotations

import collections
import concurrent.futures
import threading
import time
from typing import Dict, List, Optional

import numpy as np

__all__ = ["Server", "Request"]


class Request:
    __slots__ = ("rid", "name", "T", "P", "Y", "n", "t_submit", "t_done", "future", "dydt", "chunks", "next",
                 "left", "out", "host", "bytes", "ready", "queued")

    def __init__(self, rid, name, T, P, Y, dydt, t_submit):
        self.rid, self.name, self.T, self.P, self.Y = rid, name, T, P, Y
        self.n = int(Y.shape[0])
        self.t_submit = t_submit
        self.t_done = None
        self.future: concurrent.futures.Future = concurrent.futures.Future()
        self.dydt = dydt
        self.chunks = None        # state ranges of a chunked request, else None
        self.next = 0             # next chunk to admit
        self.left = 0             # chunks not yet completed
        self.out = self.host = None   # device outputs, host outputs (chunked requests)
        self.bytes = 0
        self.ready = None         # event: the request's inputs are on the device (chunked requests)
        self.queued = True        # False once a merged launch has taken it


class _Slice:
    """States [a, b) of a request, as the input staging reads a request."""
    __slots__ = ("n", "T", "P", "Y")

    def __init__(self, r, a, b):
        self.n, self.T, self.P, self.Y = b - a, r.T[a:b], r.P[a:b], r.Y[a:b]


class _Iteration:
    __slots__ = ("reqs", "model", "stream", "event", "bytes", "J", "F", "offsets", "host", "results", "chunk",
                 "staged", "extra")

    def __init__(self):
        self.reqs, self.offsets, self.host, self.results, self.chunk = [], [], None, None, False
        self.staged = 0           # doubles of the stream's input staging buffer in use
        self.extra = []           # pinned buffers of inputs beyond it


class Server:
    """Continuous-batching Jacobian server on the current CUDA device.

    models: name -> paper_1605_03262_b300.Model (already loaded; their launch shapes are used).
    hbm_budget: bytes of device memory in-flight iterations may hold (default: half of the memory
    free at start, counting memory PyTorch's allocator holds unused as free).
    max_inflight: concurrent iterations (and streams). Each launch fills the GPU, so iterations
    beyond the few that keep it busy only wait in the device's own first-in, first-out queues,
    where the server can no longer order them (four-model trace at 1,600 requests/s: p99 13-19 ms
    with 3 in flight, 78 ms with 6, 96 ms with 2, where the GPU idled between iterations).
    max_batch_states: states merged into one launch (with chunking on, also at most one chunk's
    worth of the model's states, so that merged launches stay about chunk_ms long).
    host_results: copy results to host memory (numpy) before completing.
    chunk_requeue: where a chunked request goes back into the queue after each chunk (None: at its
    end; k: behind at most k queued requests).
    discard_results: complete futures with None and free the device results at once (throughput
    and latency measurement). The budget covers in-flight work: results handed to clients as
    device tensors are the clients' memory from then on."""

    def __init__(self, models: Dict[str, object], hbm_budget: Optional[int] = None, max_inflight: int = 3,
                 max_batch_states: int = 65536, host_results: bool = False, discard_results: bool = False,
                 mixed: bool = False, chunk_ms: Optional[float] = 1.0, chunk_requeue: Optional[int] = None):
        import torch
        self.torch = torch
        self.models = dict(models)
        self.device = torch.device("cuda", torch.cuda.current_device())
        free, _ = torch.cuda.mem_get_info(self.device)
        free += torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        self.hbm_budget = int(hbm_budget) if hbm_budget is not None else int(free // 2)
        self.max_inflight = int(max_inflight)
        self.max_batch_states = int(max_batch_states)
        self.host_results = bool(host_results)
        self.discard_results = bool(discard_results)
        # arrival order of queued requests (entries a merged launch took are dropped lazily), and,
        # per model, the queued requests that are not cut into chunks (what a merge takes)
        self._queue: collections.deque = collections.deque()
        self._by_model = {name: collections.deque() for name in self.models}
        self._inflight: List[_Iteration] = []
        self._streams = [torch.cuda.Stream(device=self.device) for _ in range(self.max_inflight)]
        self._free_streams = list(self._streams)
        self.mixed = bool(mixed)
        self._ws = {}
        if self.mixed:                    # one batched-launch workspace per stream
            from . import batch_workspace_bytes
            nb = batch_workspace_bytes()
            self._ws = {id(st): torch.empty(nb, dtype=torch.uint8, device=self.device) for st in self._streams}
        self._held = 0
        self._cv = threading.Condition()
        self._stop = False
        self._drain = True
        self.error: Optional[BaseException] = None
        self._thread: Optional[threading.Thread] = None
        self._next_id = 0
        self.chunk_ms = chunk_ms if (chunk_ms and not self.mixed) else None
        self.chunk_requeue = chunk_requeue
        self._lib = None
        self.state_ms: Dict[str, float] = {}      # measured GPU time per state, per model
        self._stage = {}                          # per stream: pinned host staging (discarded host results)
        self._in_stage = {id(st): torch.empty(self.IN_STAGE_DOUBLES, dtype=torch.float64, pin_memory=True)
                          for st in self._streams}   # per stream: pinned staging of host inputs
        self.stats = {"iterations": 0, "requests": 0, "states": 0, "max_inflight_seen": 0, "waits_for_memory": 0,
                      "merged_requests": 0, "chunked_requests": 0, "chunks": 0}

    # -- client side ---------------------------------------------------------------------------
    def submit(self, name: str, T, P, Y, dydt: bool = False) -> concurrent.futures.Future:
        """Queue one request (host or device float64 arrays). The future's result is the Jacobian
        (n, N+1, N+1) as a CUDA tensor (or numpy array with host_results), or (J, dydt)."""
        t_submit = time.perf_counter()
        if name not in self.models:
            raise KeyError("unknown model %r" % name)
        if self.error is not None:
            raise RuntimeError("server failed") from self.error
        need = self._bytes(self.models[name], int(Y.shape[0]))
        if need > self.hbm_budget:
            raise ValueError("request needs %d bytes of device memory, above the server's budget %d"
                             % (need, self.hbm_budget))
        with self._cv:
            req = Request(self._next_id, name, T, P, Y, dydt, t_submit)
            req.future.request = req          # lets clients read the request's timings
            cs = self._chunk_states(name)
            if cs and req.n > cs:
                k = -(-req.n // cs)
                edges = [req.n * x // k for x in range(k + 1)]
                req.chunks = list(zip(edges[:-1], edges[1:]))
                req.left = k
            self._next_id += 1
            self._queue.append(req)
            if req.chunks is None and not self.mixed:
                self._by_model[name].append(req)
            self._cv.notify()
        return req.future

    def _inputs_for(self, it, reqs, N):
        """Device (T, P, Y) of the requests, in order, filled on the iteration's stream.

        Host inputs (numpy arrays or CPU tensors) are packed as [T | P | Y] into the stream's
        pinned staging buffer (numpy copies on this thread) and sent with one asynchronous copy: a
        copy from pageable memory would block the scheduler thread for its whole transfer, which
        cost the four-model trace about 40 % of its closed-loop throughput, and each further
        copy or allocation costs the thread time a small request's launch does not have. Device
        inputs are used as they are (one request) or concatenated on the device."""
        torch = self.torch
        f64 = torch.float64
        n = sum(r.n for r in reqs)
        on_dev = [isinstance(x, torch.Tensor) and x.is_cuda for r in reqs for x in (r.T, r.P, r.Y)]
        if all(on_dev):
            parts = [[r.T.to(f64).reshape(-1) for r in reqs], [r.P.to(f64).reshape(-1) for r in reqs],
                     [r.Y.to(f64) for r in reqs]]
            if len(reqs) == 1:
                return tuple(x[0].contiguous() for x in parts)
            return tuple(torch.cat(x) for x in parts)
        total = n * (N + 2)
        buf = self._in_stage[id(it.stream)]
        if it.staged + total > buf.numel():      # beyond the staging buffer: a pinned buffer of its own
            h = torch.empty(total, dtype=f64, pin_memory=True)
            it.extra.append(h)
        else:
            h = buf[it.staged: it.staged + total]
            it.staged += total
        hn = h.numpy()
        Th, Ph, Yh = hn[:n], hn[n:2 * n], hn[2 * n:].reshape(n, N)
        a = 0
        for r in reqs:
            b = a + r.n
            for dst, x in ((Th, r.T), (Ph, r.P), (Yh, r.Y)):
                if isinstance(x, torch.Tensor):
                    x = x.cpu()                  # (a device input among host ones: rare)
                dst[a:b] = np.asarray(x).reshape(dst[a:b].shape)
            a = b
        d = torch.empty(total, dtype=f64, device=self.device)
        d.copy_(h, non_blocking=True)
        return d[:n], d[n:2 * n], d[2 * n:].view(n, N)

    def _chunk_states(self, name: str) -> int:
        """States per chunk of a request to this model (0: requests are not cut)."""
        if not self.chunk_ms or name not in self.state_ms:
            return 0
        return max(1, int(self.chunk_ms / self.state_ms[name]))

    def calibrate(self, n_states: int = 2048) -> Dict[str, float]:
        """Measure each model's GPU time per state (a warm launch of a synthetic batch that fills
        the GPU), which sets the chunk sizes."""
        torch = self.torch
        from . import synth
        for name, m in self.models.items():
            N = m.n_species
            T, P, Y = (torch.as_tensor(a, dtype=torch.float64, device=self.device)
                       for a in synth.generate_states(N, n_states, seed=4242))
            J = torch.empty((n_states, N + 1, N + 1), dtype=torch.float64, device=self.device)
            m.eval_jacobian(T, P, Y, out=J)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            m.eval_jacobian(T, P, Y, out=J)
            e1.record()
            torch.cuda.synchronize()
            self.state_ms[name] = e0.elapsed_time(e1) / n_states
            del J, T, P, Y
        return dict(self.state_ms)

    def start(self) -> "Server":
        if self.chunk_ms and not self.state_ms:
            self.calibrate()
        if self._thread is None:
            self._stop = False
            self._thread = threading.Thread(target=self._loop, name="pyjac-b300-server", daemon=True)
            self._thread.start()
        return self

    def stop(self, drain: bool = True) -> None:
        if self._thread is None:
            return
        with self._cv:
            self._stop = True
            self._drain = drain
            self._cv.notify()
        self._thread.join()
        self._thread = None

    def __enter__(self):
        return self.start()

    def __exit__(self, *exc):
        self.stop()

    # -- scheduler -----------------------------------------------------------------------------
    @staticmethod
    def _bytes(model, n: int) -> int:
        N = model.n_species
        return 8 * n * ((N + 1) ** 2 + 2 * (N + 1) + 2)

    def _head(self) -> Optional[Request]:
        """Under the lock: the first queued request (dropping entries a merged launch took)."""
        q = self._queue
        while q and not q[0].queued:
            q.popleft()
        return q[0] if q else None

    def _loop(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        error = None
        try:
            while True:
                progressed = self._retire()
                with self._cv:
                    if self._stop and (not self._drain or (self._head() is None and not self._inflight)):
                        break
                progressed |= self._admit()
                if not progressed:                    # (also while the head waits for memory)
                    with self._cv:
                        self._cv.wait(timeout=0.0002 if self._inflight else 0.05)
        except BaseException as exc:          # a failed launch or allocation must not strand clients
            error = exc
        # fail whatever is left: queued requests (stop without drain, or an error) and, after an
        # error, the requests of iterations that will not be retired
        with self._cv:
            self.error = error
            pending = [r for r in self._queue if r.queued]
            self._queue.clear()
        if error is not None:
            for it in self._inflight:
                pending += it.reqs
            self._inflight = []
        for r in pending:
            if not r.future.done():
                r.future.set_exception(error if error is not None else RuntimeError("server stopped"))

    def _retire(self) -> bool:
        done = [it for it in self._inflight if it.event.query()]
        for it in done:
            self._inflight.remove(it)
            t = time.perf_counter()
            if it.chunk:                          # one chunk of a request: complete it after its last
                r = it.reqs[0]
                r.left -= 1
                if r.left == 0:
                    r.t_done = t
                    if self.discard_results:
                        r.future.set_result(None)
                    else:
                        J, F = r.host if self.host_results else r.out
                        if self.host_results:
                            J, F = J.numpy(), F.numpy() if F is not None else None
                        r.future.set_result((J, F) if r.dydt else J)
                    r.out = r.host = r.ready = None
                    self._held -= r.bytes
                self._free_streams.append(it.stream)
                continue
            for x, r in enumerate(it.reqs):
                r.t_done = t
                if self.discard_results:
                    r.future.set_result(None)
                    continue
                if it.results is not None:        # a mixed iteration: one output per request
                    J, F = it.results[x]
                    r.future.set_result((J, F) if r.dydt else J)
                    continue
                a, b = it.offsets[x]
                if self.host_results:
                    J = it.host[0][a:b]
                    res = (J, it.host[1][a:b]) if r.dydt else J
                else:
                    J = it.J[a:b]
                    res = (J, it.F[a:b]) if r.dydt else J
                r.future.set_result(res)
            self._held -= it.bytes
            self._free_streams.append(it.stream)
        return bool(done)

    def _admit(self) -> bool:
        return self._admit_mixed() if self.mixed else self._admit_merged()

    def _admit_mixed(self) -> bool:
        """Iterations of up to 64 queued requests of any models, one batched launch each."""
        from . import run_batch
        torch = self.torch
        admitted = False
        while True:
            with self._cv:
                if self._head() is None or len(self._inflight) >= self.max_inflight or not self._free_streams:
                    return admitted
                take, n, need = [], 0, 0
                for r in self._queue:
                    if not r.queued:
                        continue
                    b = self._bytes(self.models[r.name], r.n)
                    if take and (len(take) == 64 or n + r.n > self.max_batch_states or
                                 self._held + need + b > self.hbm_budget):
                        break
                    take.append(r)
                    n += r.n
                    need += b
                if self._held + need > self.hbm_budget:
                    self.stats["waits_for_memory"] += 1
                    return admitted
                for r in take:
                    r.queued = False
            it = _Iteration()
            it.reqs, it.model, it.bytes = take, None, need
            it.stream = self._free_streams.pop()
            self._held += need
            items, results = [], []
            with torch.cuda.stream(it.stream):
                for r in take:
                    model = self.models[r.name]
                    N = model.n_species
                    T, P, Y = self._inputs_for(it, [r], N)
                    J = torch.empty((r.n, N + 1, N + 1), dtype=torch.float64, device=self.device)
                    F = torch.empty((r.n, N + 1), dtype=torch.float64, device=self.device) if r.dydt else None
                    items.append((model, T, P, Y, J) + ((F,) if F is not None else ()))
                    results.append((J, F))
                run_batch(items, workspace=self._ws[id(it.stream)], stream=it.stream)
                if self.host_results:
                    hres = []
                    for J, F in results:
                        Jh = self._copy_to_host(it.stream, J)
                        Fh = self._copy_to_host(it.stream, F) if F is not None else None
                        hres.append((Jh.numpy() if Jh is not None else None, Fh.numpy() if Fh is not None else None))
                    results = hres
                it.results = results
                it.event = torch.cuda.Event()
                it.event.record(it.stream)
            self._inflight.append(it)
            self.stats["iterations"] += 1
            self.stats["requests"] += len(take)
            self.stats["merged_requests"] += len(take) - 1
            self.stats["states"] += n
            self.stats["max_inflight_seen"] = max(self.stats["max_inflight_seen"], len(self._inflight))
            admitted = True

    STAGE_DOUBLES = 1 << 24             # 128 MB of pinned staging per stream (discarded host results)
    IN_STAGE_DOUBLES = 1 << 22          # 32 MB of pinned staging per stream (host inputs of an iteration)

    def _copy_to_host(self, stream, src):
        """Copy a device result to host memory on the stream: into a fresh pinned buffer that is
        returned (results handed to the client), or, when results are discarded, piece by piece
        through the stream's fixed pinned staging buffer (the copy takes its PCIe time, the host
        memory stays bounded); returns None then."""
        torch = self.torch
        if not self.discard_results:
            h = torch.empty(src.shape, dtype=torch.float64, pin_memory=True)
            h.copy_(src, non_blocking=True)
            return h
        buf = self._stage.get(id(stream))
        if buf is None:
            buf = torch.empty(self.STAGE_DOUBLES, dtype=torch.float64, pin_memory=True)
            self._stage[id(stream)] = buf
        flat = src.reshape(-1)
        for a in range(0, flat.numel(), buf.numel()):
            b = min(flat.numel(), a + buf.numel())
            buf[: b - a].copy_(flat[a:b], non_blocking=True)
        return None

    def _admit_chunk(self, r: Request, model) -> None:
        """One chunk of a chunked request on a free stream, into its slice of the request's output
        (allocated, for the whole request, at its first chunk). Each chunk stages and copies only
        its own inputs, so that the first chunk of a large request does not hold the scheduler
        for the copy of all of them."""
        torch = self.torch
        a, b = r.chunks[r.next]
        it = _Iteration()
        it.reqs, it.model, it.bytes, it.chunk = [r], model, 0, True
        it.stream = self._free_streams.pop()
        N = model.n_species
        with torch.cuda.stream(it.stream):
            if r.next == 0:
                r.bytes = self._bytes(model, r.n)
                self._held += r.bytes
                J = torch.empty((r.n, N + 1, N + 1), dtype=torch.float64, device=self.device)
                F = torch.empty((r.n, N + 1), dtype=torch.float64, device=self.device) if r.dydt else None
                r.out = (J, F)
                if self.host_results and not self.discard_results:
                    r.host = (torch.empty((r.n, N + 1, N + 1), dtype=torch.float64, pin_memory=True),
                              torch.empty((r.n, N + 1), dtype=torch.float64, pin_memory=True) if r.dydt else None)
                r.ready = torch.cuda.Event()
                r.ready.record(it.stream)                  # the outputs' memory is this stream's
                self.stats["chunked_requests"] += 1
            else:
                it.stream.wait_event(r.ready)             # later chunks run on other streams
            T, P, Y = self._inputs_for(it, [_Slice(r, a, b)], N)
            J, F = r.out
            self._launch(model, T, P, Y, J[a:b], F[a:b] if F is not None else None, it.stream)
            if self.host_results:
                if self.discard_results:                  # the copy counts, its result is dropped
                    self._copy_to_host(it.stream, J[a:b])
                else:
                    r.host[0][a:b].copy_(J[a:b], non_blocking=True)
                    if F is not None:
                        r.host[1][a:b].copy_(F[a:b], non_blocking=True)
            it.event = torch.cuda.Event()
            it.event.record(it.stream)
        r.next += 1
        self._inflight.append(it)
        self.stats["iterations"] += 1
        self.stats["chunks"] += 1
        if r.next == 1:
            self.stats["requests"] += 1
            self.stats["states"] += r.n
        self.stats["max_inflight_seen"] = max(self.stats["max_inflight_seen"], len(self._inflight))

    def _launch(self, model, T, P, Y, J, F, stream) -> None:
        """The model's Jacobian launch on tensors this server built (float64, contiguous, on its
        device), through the C ABI without the binding's argument checks: on small requests
        those checks cost the scheduler thread about as much as the launch itself."""
        from . import _check, library
        lib = self._lib
        if lib is None:
            lib = self._lib = library()
        n = int(T.shape[0])
        _check(lib.pj_eval_jacobian(model._h, n, T.data_ptr(), P.data_ptr(), Y.data_ptr(), Y.stride(0),
                                    J.data_ptr(), J.stride(0), F.data_ptr() if F is not None else None,
                                    F.stride(0) if F is not None else 0, stream.cuda_stream))

    def _requeue(self, r: Request) -> None:
        """Under the lock: a chunked request with chunks left goes back into the queue, at its end
        or, with chunk_requeue = k, behind at most k queued requests."""
        if self.chunk_requeue is None or len(self._queue) <= self.chunk_requeue:
            self._queue.append(r)
        else:
            self._queue.insert(self.chunk_requeue, r)

    def _take_started(self) -> Optional[Request]:
        """Under the lock, when the queue's head waits for memory: the first queued request that
        already runs in chunks, taken out of the queue (and put back at its end if chunks remain
        after the next). Its next chunk needs no new memory, and only its completion gives memory
        back, so it must not wait behind the head: with chunks rotating through the queue, a head
        that blocked them could wait forever."""
        for r in self._queue:
            if r.queued and r.chunks is not None and r.next > 0:
                self._queue.remove(r)
                if r.next + 1 < len(r.chunks):
                    self._requeue(r)
                return r
        return None

    def _admit_merged(self) -> bool:
        torch = self.torch
        admitted = False
        while True:
            with self._cv:
                head = self._head()
                if head is None or len(self._inflight) >= self.max_inflight or not self._free_streams:
                    return admitted
                model = self.models[head.name]
                resume = None
                if head.chunks is not None:
                    if head.next == 0 and self._held + self._bytes(model, head.n) > self.hbm_budget:
                        self.stats["waits_for_memory"] += 1
                        resume = self._take_started()
                        if resume is None:
                            return admitted
                    else:
                        self._queue.popleft()
                        if head.next + 1 < len(head.chunks):
                            self._requeue(head)           # its next chunk after others queued now
                        resume = head
                else:
                    # merge queued requests of the head's model, in arrival order, up to the state
                    # cap (and, with chunking, up to one chunk of GPU time)
                    cap = self.max_batch_states
                    cs = self._chunk_states(head.name)
                    if cs:
                        cap = min(cap, max(cs, head.n))
                    same = self._by_model[head.name]     # its first entry is the head
                    take, n = [], 0
                    for r in same:
                        if take and n + r.n > cap:
                            break
                        take.append(r)
                        n += r.n
                    need = self._bytes(model, n)
                    if self._held + need > self.hbm_budget and len(take) > 1:   # the head alone
                        take, n = [head], head.n
                        need = self._bytes(model, n)
                    if self._held + need > self.hbm_budget:
                        self.stats["waits_for_memory"] += 1
                        resume = self._take_started()
                        if resume is None:
                            return admitted
                    else:
                        for r in take:
                            same.popleft()
                            r.queued = False
            if resume is not None:
                self._admit_chunk(resume, self.models[resume.name])
                admitted = True
                continue
            it = _Iteration()
            it.reqs, it.model, it.bytes = take, model, need
            it.stream = self._free_streams.pop()
            self._held += need
            N = model.n_species
            with torch.cuda.stream(it.stream):
                T, P, Y = self._inputs_for(it, take, N)
                a = 0
                for r in take:
                    it.offsets.append((a, a + r.n))
                    a += r.n
                it.J = torch.empty((n, N + 1, N + 1), dtype=torch.float64, device=self.device)
                want_f = any(r.dydt for r in take)
                it.F = torch.empty((n, N + 1), dtype=torch.float64, device=self.device) if want_f else None
                self._launch(model, T, P, Y, it.J, it.F, it.stream)
                if self.host_results:
                    Jh = self._copy_to_host(it.stream, it.J)
                    Fh = self._copy_to_host(it.stream, it.F) if it.F is not None else None
                    it.host = (Jh.numpy() if Jh is not None else None, Fh.numpy() if Fh is not None else None)
                    it.J = it.F = None
                it.event = torch.cuda.Event()
                it.event.record(it.stream)
            self._inflight.append(it)
            self.stats["iterations"] += 1
            self.stats["requests"] += len(take)
            self.stats["merged_requests"] += len(take) - 1
            self.stats["states"] += n
            self.stats["max_inflight_seen"] = max(self.stats["max_inflight_seen"], len(self._inflight))
            admitted = True


def latency_summary(requests: List[Request]) -> dict:
    lat = np.array([r.t_done - r.t_submit for r in requests if r.t_done is not None]) * 1e3
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max())}
