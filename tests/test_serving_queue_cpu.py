"""The serving loop's queue logic on the host (no GPU): which request goes next when the head of
the queue waits for memory, where a chunked request goes back into the queue, and how entries a
merged launch took are dropped from the arrival order."""
import collections

import numpy as np

from paper_1605_03262_b300.serving import Request, Server


def _req(rid, name="m", n=10, chunks=None, nxt=0):
    r = Request(rid, name, None, None, np.zeros((n, 1)), False, 0.0)
    if chunks:
        r.chunks = [(k * n // chunks, (k + 1) * n // chunks) for k in range(chunks)]
        r.left = chunks
        r.next = nxt
    return r


def _server(requeue=None):
    srv = Server.__new__(Server)          # the queue logic only: no streams, no device
    srv._queue = collections.deque()
    srv._by_model = {"m": collections.deque()}
    srv.chunk_requeue = requeue
    return srv


def test_a_started_chunked_request_goes_ahead_of_a_head_waiting_for_memory():
    srv = _server()
    waiting = _req(0, chunks=3)               # not started: would need new memory
    small = _req(1)
    started = _req(2, chunks=4, nxt=1)        # started: holds its memory until its last chunk
    srv._queue.extend([waiting, small, started])
    got = srv._take_started()
    assert got is started
    # it went back to the end of the queue for its remaining chunks
    assert list(srv._queue) == [waiting, small, started]
    assert srv._take_started() is started
    # with no started request behind the head, nothing goes ahead of it
    srv2 = _server()
    srv2._queue.extend([_req(0, chunks=3), _req(1)])
    assert srv2._take_started() is None


def test_the_last_chunk_of_a_started_request_leaves_the_queue():
    srv = _server()
    last = _req(0, chunks=2, nxt=1)           # its next chunk is its last
    srv._queue.extend([_req(1, chunks=2), last])
    assert srv._take_started() is last
    assert last not in srv._queue


def test_chunk_requeue_position():
    r = _req(9, chunks=3, nxt=1)
    srv = _server()
    srv._queue.extend([_req(k) for k in range(5)])
    srv._requeue(r)
    assert srv._queue[-1] is r                # default: the end of the queue
    srv = _server(requeue=2)
    others = [_req(k) for k in range(5)]
    srv._queue.extend(others)
    srv._requeue(r)
    assert list(srv._queue).index(r) == 2     # behind at most two queued requests
    srv = _server(requeue=8)
    srv._queue.extend([_req(k) for k in range(3)])
    srv._requeue(r)
    assert srv._queue[-1] is r                # a short queue: its end


def test_the_head_skips_entries_a_merged_launch_took():
    srv = _server()
    a, b, c = _req(0), _req(1), _req(2)
    srv._queue.extend([a, b, c])
    a.queued = False                          # taken by a merge
    b.queued = False
    assert srv._head() is c
    assert list(srv._queue) == [c]
    c.queued = False
    assert srv._head() is None
