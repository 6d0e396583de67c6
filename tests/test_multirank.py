"""Host logic of the benchmark's multi-GPU mode, on CPU with the gloo backend
and two ranks (one process per rank, as torchrun launches them): the
problem is not sharded -- every rank solves its own replica (its own seed)
and the job's time is the slowest rank's, so the reported rate is
world x the per-rank cells / that time.  The reference arm runs on rank 0
only; the other ranks exit at once without output."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(1.5 + rank, world, device="cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(rank))
    dist.barrier()
    q.put((rank, slowest, seeds))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, seeds in results:
        assert slowest == 2.5          # the slower rank's time on every rank
        assert seeds == [0, 1]         # distinct replicas


def test_job_rate():
    import bench
    # two replicas of 256^3 cells in 10 ms: twice one replica's rate
    assert bench.job_rate(256 ** 3, 2, 0.01) == pytest.approx(2 * 256 ** 3 / 0.01)
    assert bench.max_over_ranks(3.0, 1) == 3.0


def test_reference_arm_on_other_ranks_is_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], cwd=ROOT, env=env,
                       capture_output=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == b""
