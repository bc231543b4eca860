"""bench.py's multi-rank logic on CPU: two gloo ranks (world size 2).

Each rank decomposes its own batch (weak scaling); the only collective is the
max-reduce of the timed seconds, and the reported value counts every rank's
samples over the slowest rank's time.  Also checks that the ranks' batches are
different signals (rank r takes signals r*B .. r*B+B-1 of the workload).
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1802_01359_gb300 import signals
    my_seconds = [1.25, 2.5][rank]
    t = bench.max_over_ranks(my_seconds, dist, "cpu")
    rate = bench.whole_job_rate(1000, world, t)
    wid = getattr(signals, bench.UNIFORM[bench.DEFAULT_WORKLOAD][0])
    first = signals.component_signal(wid, bench.first_signal(bench.DEFAULT_WORKLOAD, rank), 256)
    q.put((rank, t, rate, first))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        r, t, rate, first = q.get(timeout=120)
        got[r] = (t, rate, first)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        t, rate, _ = got[r]
        assert t == 2.5                      # the slowest rank's seconds, on every rank
        assert rate == pytest.approx(2 * 1000 / 2.5)
    assert not np.array_equal(got[0][2], got[1][2])   # disjoint batches


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.whole_job_rate(500, 1, 2.0) == 250.0
    assert bench.first_signal("batch4096", 3) == 3 * 65536
    assert bench.first_signal("long", 3) == 0
