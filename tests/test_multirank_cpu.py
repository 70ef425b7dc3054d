"""The benchmark's multi-rank path on CPU: two gloo ranks, each serving its own stream.

Independent solves shard with no collective on the data path; the ranks only combine their
timings and work at the end (slowest rank's time, summed entries).
"""
import os
import socket

import pytest
import torch
import torch.distributed as td
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import argparse
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    t_step = 1.0 + rank            # rank 1 is the slower one
    entries = 1e12 * (rank + 1)
    res = bench.combine_over_ranks(td, "cpu", t_step, entries, 2.0 + rank, 5e11 * (rank + 1))
    args = argparse.Namespace(requests=8, seed=2609, rate=32.0, burst=False)
    reqs, _ = bench.make_stream(args, rank)
    out.put((rank, res, [(r.s, r.seed) for r in reqs]))
    td.destroy_process_group()


def test_two_gloo_ranks_combine_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (res, rq)) for r, res, rq in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        t, e, t2, e2 = got[r][0]
        assert t == 2.0 and e == 3e12 and t2 == 3.0 and e2 == 1.5e12
    assert got[0][1] != got[1][1]  # each rank serves a different seeded stream
