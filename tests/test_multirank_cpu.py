"""Multi-GPU host logic of bench.py on CPU: two gloo ranks (no GPU, no collective on the data path;
the only reductions are the job's step time and state count)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t = 10.0 + 5.0 * rank                       # per-rank step time (ms)
    n = 100.0 * (rank + 1)
    T, P, Y = bench.shard_states(0, rank, 16)
    out[rank] = (bench._max_over_ranks(ws, t), bench._sum_over_ranks(ws, n), float(T[0]), float(Y[0, 0]))
    bench._barrier(ws)
    dist.destroy_process_group()


def test_two_ranks_reduce_time_and_states_and_draw_distinct_batches():
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0         # max step time over ranks
    assert res[0][1] == res[1][1] == 300.0        # states of the whole job
    assert res[0][2] != res[1][2] and res[0][3] != res[1][3]   # each rank owns its own states
