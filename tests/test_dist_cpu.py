"""The multi-process (N > 1) bench path on CPU ranks (gloo, world size 2):
every rank draws its own collection (independent problems, no collective on
the data path) and the whole-job number is the summed work over the slowest
rank's time."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.dist_env() == (world, rank, rank)
    off, ids, cfg = bench.make_workload("ancestral64", rank)
    # the slowest rank's time, the summed work
    ms, work = bench.aggregate_over_ranks(10.0 * (rank + 1), 100.0 + rank)
    out.put((rank, ms, work, int(off[-1]), int(ids[:64].sum() % (1 << 62))))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(240)
def test_two_gloo_ranks_draw_independent_problems_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=200) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, w0, n0, h0), (r1, ms1, w1, n1, h1) = res
    assert (r0, r1) == (0, 1)
    assert ms0 == ms1 == 20.0          # max over ranks
    assert w0 == w1 == 201.0           # sum over ranks
    assert (n0, h0) != (n1, h1)        # each rank its own collection


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(12.5, 7.0) == (12.5, 7.0)
