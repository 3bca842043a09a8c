"""The multi-GPU bench's host logic on CPU ranks (gloo, world size 2).

Toys are independent, so the batch shards with no exchange step: each rank draws its own toys
from a seed range of its own, times its own step, and the job's time is the slowest rank's.  Two
gloo ranks check that the ranks' toy batches differ, that every rank receives the maximum of the
ranks' step times, and the whole-job rate."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        T = 3
        _, b = bench.make_inputs(T, bench.rank_toy_seed(rank, T))
        digest = torch.tensor([float(b["counts"].sum()), float(b["windows"].sum())], dtype=torch.float64)
        all_digests = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(all_digests, digest)
        dist.barrier()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
        out.put((rank, [d.tolist() for d in all_digests], ms, bench.job_rate(world, T, ms),
                 int(b["windows"].min()), int(b["windows"].max())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_toys_and_time_the_slowest():
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, d0, ms0, v0, lo0, hi0), (r1, d1, ms1, v1, lo1, hi1) = res
    assert (r0, r1) == (0, 1)
    assert d0 == d1                      # both ranks see the same gathered digests
    assert d0[0] != d0[1]                # ... and the ranks' toy batches differ
    assert ms0 == ms1 == 15.0            # every rank gets the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 3 / 15e-3)
    assert min(lo0, lo1) >= 0 and max(hi0, hi1) <= 1200
