"""Host side of segment sharding (Sec. 7, redundant coarse-grid solves) on
CPU: two gloo ranks, one process each, as torchrun would launch them.

- The exchange: each rank owns half of the 512 segments of the 256^3
  benchmark geometry and fills only its segments' genuine cells of the two
  transition-level arrays (32^3 doubles each, 512 KB together); after
  srfmg.exchange_sum with an all-reduce over gloo both ranks hold exactly
  the whole arrays.
- The driver: srfmg.solve_staged calls stage_down(k), the exchange and
  stage_up(k) for k = 1..K in that order on a stand-in handle whose
  stage_up checks that it sees the sum over both ranks."""
import os
import socket

import numpy as np
import pytest

N0, S0, NSD = 32, 4, 8   # transition level 32^3, 4^3 genuine cells per segment, 8^3 segments


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def owned_mask(first, count):
    """genuine transition-level cells of segments first .. first+count-1 (x fastest)"""
    m = np.zeros((N0, N0, N0), dtype=bool)
    for i in range(first, first + count):
        px, py, pz = i % NSD, (i // NSD) % NSD, i // (NSD * NSD)
        m[pz * S0:(pz + 1) * S0, py * S0:(py + 1) * S0, px * S0:(px + 1) * S0] = True
    return m


def whole(k):
    """the values every cell should end with after stage k's exchange"""
    rng = np.random.default_rng(k)
    return rng.standard_normal((2, N0, N0, N0))


class StandIn:
    """Records the stage calls of one rank's handle; its exchange arrays get
    that rank's cells of whole(k)."""

    def __init__(self, rank, world, K, log):
        from paper_1406_7808_gb300 import srfmg
        first, count = srfmg.segment_range(NSD ** 3, rank, world)
        self.mask = owned_mask(first, count)
        self.K, self.log = K, log
        import torch
        self.bufs = (torch.zeros(N0 ** 3, dtype=torch.float64),
                     torch.zeros(N0 ** 3, dtype=torch.float64))

    def stage_down(self, f, k):
        self.log.append(("down", k))
        w = whole(k)
        for b, v in zip(self.bufs, w):
            b.copy_(__import__("torch").from_numpy(np.where(self.mask, v, 0.0).ravel()))

    def stage_buffers(self):
        return self.bufs

    def stage_up(self, f, k, out):
        w = whole(k)
        ok = all(np.array_equal(b.numpy(), v.ravel()) for b, v in zip(self.bufs, w))
        self.log.append(("up", k, ok))


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1406_7808_gb300 import srfmg

    def allreduce(ts):
        for t in ts:
            dist.all_reduce(t)

    # the exchange alone, on the benchmark's segment split
    first, count = srfmg.segment_range(NSD ** 3, rank, world)
    m = owned_mask(first, count)
    w = whole(7)
    bufs = [tuple(torch.from_numpy(np.where(m, v, 0.0).ravel()) for v in w)]
    srfmg.exchange_sum(bufs, allreduce)
    exchange_ok = all(np.array_equal(b.numpy(), v.ravel()) for b, v in zip(bufs[0], w))
    # the driver with a stand-in handle, K = 3
    log = []
    srfmg.solve_staged([StandIn(rank, world, 3, log)], None, None, allreduce)
    dist.barrier()
    q.put((rank, exchange_ok, log, count))
    dist.destroy_process_group()


def test_two_rank_exchange_and_driver_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[3] for r in results] == [256, 256]
    for rank, exchange_ok, log, _ in results:
        assert exchange_ok
        assert log == [("down", 1), ("up", 1, True), ("down", 2), ("up", 2, True),
                       ("down", 3), ("up", 3, True)]


def test_segment_ranges_cover_once():
    from paper_1406_7808_gb300 import srfmg
    for nsegs, world in [(512, 2), (512, 3), (64, 8), (16, 5), (7, 7)]:
        seen = []
        for r in range(world):
            first, count = srfmg.segment_range(nsegs, r, world)
            seen += list(range(first, first + count))
            assert count in (nsegs // world, nsegs // world + 1)
        assert seen == list(range(nsegs))
    assert srfmg.segment_count(256, 32) == 512
    assert srfmg.segment_count(16, 8, (2, 1, 1)) == 16   # the paper's 4 x 2 x 2 layout


def test_exchange_sum_local_handles():
    import torch
    from paper_1406_7808_gb300 import srfmg
    a = (torch.tensor([1.0, 0.0, 0.0]), torch.tensor([0.0, -2.0, 0.0]))
    b = (torch.tensor([0.0, 3.0, 0.0]), torch.tensor([0.0, 0.0, 5.0]))
    srfmg.exchange_sum([a, b])
    for t in (a, b):
        assert t[0].tolist() == [1.0, 3.0, 0.0] and t[1].tolist() == [0.0, -2.0, 5.0]
