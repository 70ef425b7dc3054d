"""Row-sharded execution, host side (CPU only, two gloo ranks): the slice partition and the exchange
of packed operands and certificate partial sums that ``paper_2609_33814_b300.shard`` runs between
half-sweeps.  The GPU test ``test_shard_gpu.py`` runs the same driver on real slice states."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

P = pytest.importorskip("paper_2609_33814_b300")


@pytest.mark.parametrize("np_,world", [(2304, 2), (1500, 2), (4096, 3), (10_000_000, 4), (513, 2)])
def test_slices_partition_the_points(np_, world):
    got = [P.shard_range(np_, r, world) for r in range(world)]
    assert got[0][0] == 0 and got[-1][1] == np_
    for (a0, a1), (b0, b1) in zip(got, got[1:]):
        assert a1 == b0                      # contiguous, disjoint
    for p0, p1 in got:
        assert p0 % 512 == 0 and p1 > p0     # whole 512-point units (a multiple of every point block)
    units = [(p1 - p0 + 511) // 512 for p0, p1 in got]
    assert max(units) - min(units) <= 1      # balanced


class _FakeSlice:
    """A slice state without a GPU: its pack slice is recognisable bytes, puts are recorded."""

    def __init__(self, rank, world):
        self.rank, self.world = rank, world
        self.put = {}

    def pack_bytes(self, side, rank):
        return 100 + 37 * rank + side

    def pack_get(self, side):
        return np.full(self.pack_bytes(side, self.rank), 10 * self.rank + side, np.uint8)

    def pack_put(self, side, rank, buf):
        self.put[(side, rank)] = buf.copy()

    def cert_partials(self):
        r = self.rank + 1.0
        return np.array([r, 2 * r, 3 * r, 0.5 * r, 0.01])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2609_33814_b300 import shard
    st = _FakeSlice(rank, world)
    for side in (0, 1):
        shard.exchange(st, side)
    U, L, eps = shard.certificate(st, omega=2.0)
    q.put((rank, {k: (v.size, int(v[0]), int(v.max())) for k, v in st.put.items()}, U, L, eps))
    td.destroy_process_group()


def test_exchange_and_certificate_over_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        r, puts, U, L, eps = q.get(timeout=120)
        got[r] = (puts, U, L, eps)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        puts, U, L, eps = got[r]
        other = 1 - r
        # every other rank's slice arrives whole (its own size, its own bytes), none of its own
        assert set(puts) == {(0, other), (1, other)}
        for side in (0, 1):
            size, first, top = puts[(side, other)]
            assert size == 100 + 37 * other + side and first == top == 10 * other + side
        # L = sum <r,f> + sum <c,g>, U = sum <t,w> + omega sum delta over the ranks
        assert L == pytest.approx((1 + 2) * 3.0) and U == pytest.approx((1 + 2) * 3.0 + 2.0 * 0.5 * 3.0)
        assert eps == pytest.approx(0.01)
