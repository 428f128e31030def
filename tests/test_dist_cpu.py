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


def _part_rank(rank, world, port, out):
    """Rank r takes part r of the collection's row batches (the rule of
    jsim_all_pairs_part), counts its pairs with the oracle over the values in
    its batches, and the counts are summed across ranks with one all-reduce
    (the exchange step of a split contraction)."""
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1911_04200_gb300 import jsim, synth
    off, ids = synth.ancestral64()
    mt = 1 << 14
    nz = [i for i in range(len(off) - 1) if off[i + 1] > off[i]]
    minid = min(int(ids[off[i]]) for i in nz)
    maxid = max(int(ids[off[i + 1] - 1]) for i in nz)
    b0, b1 = jsim.partition_batches(minid, maxid, mt, world)[rank]
    lo, hi = b0 * mt, b1 * mt
    segs = [ids[int(off[i]):int(off[i + 1])] for i in range(len(off) - 1)]
    part = [s[(s >= lo) & (s < hi)] for s in segs]
    poff = np.zeros(len(part) + 1, dtype=np.uint64)
    poff[1:] = np.cumsum([len(s) for s in part])
    pids = np.concatenate(part).astype(np.uint64)
    C, _, _ = oracle.all_pairs(poff, pids)
    t = torch.from_numpy(C.astype(np.int64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    out.put((rank, t.numpy().astype(np.uint64), (lo, hi)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(240)
def test_split_contraction_over_two_gloo_ranks_sums_to_the_whole():
    """C is additive over row batches (Eq. 4): two CPU ranks each count the
    pairs of one part of the batches, one all-reduce sums them, and the sum
    is the whole collection's C; the parts tile the value range."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1911_04200_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_part_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=200) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, C0, r0), (_, C1, r1) = res
    np.testing.assert_array_equal(C0, C1)            # every rank holds the sum
    assert r0[1] == r1[0] and r0[0] < r0[1] < r1[1]  # contiguous, disjoint parts
    off, ids = synth.ancestral64()
    Cw, _, _ = oracle.all_pairs(off, ids)
    np.testing.assert_array_equal(C0, Cw)


def test_partition_rule_tiles_the_batches():
    sys.path.insert(0, ROOT)
    from paper_1911_04200_gb300 import jsim
    for minid, maxid, mt in ((0, 10**6, 1 << 14), (5, 5, 64), (2**40, 2**41, 1 << 28), (0, 2**64 - 1, 1 << 28)):
        first, last = minid // mt, maxid // mt
        for parts in (1, 2, 3, 7, 64):
            pb = jsim.partition_batches(minid, maxid, mt, parts)
            assert len(pb) == parts and pb[0][0] == first and pb[-1][1] == last + 1
            assert all(a <= b for a, b in pb) and all(pb[k][1] == pb[k + 1][0] for k in range(parts - 1))
            sizes = [b - a for a, b in pb]
            assert max(sizes) - min(sizes) <= 1


def test_partition_rule_is_the_library_rule_with_the_automatic_batch_size():
    """The split is computed by the library (jsim_partition_batches), with the
    automatic batch size of a plain call: 2^28 rows for a 2^32 span (16
    batches), the span itself rounded up to a power of two when smaller."""
    import ctypes
    sys.path.insert(0, ROOT)
    from paper_1911_04200_gb300 import jsim
    lib = jsim.load()
    b0, b1, mt = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    assert lib.jsim_partition_batches(0, 2**32 - 1, 0, 0, 1, ctypes.byref(b0), ctypes.byref(b1), ctypes.byref(mt)) == 0
    assert (b0.value, b1.value, mt.value) == (0, 16, 1 << 28)
    assert lib.jsim_partition_batches(100, 5000, 0, 1, 2, ctypes.byref(b0), ctypes.byref(b1), ctypes.byref(mt)) == 0
    assert mt.value == 8192 and (b0.value, b1.value) == (0, 1)
    assert jsim.partition_batches(0, 2**32 - 1, 0, 4) == [(0, 4), (4, 8), (8, 12), (12, 16)]
    for bad in ((0, 10, 0, 2, 2), (0, 10, 0, 0, 0), (10, 0, 0, 0, 1), (0, 10, 100, 0, 1)):
        assert lib.jsim_partition_batches(*bad, None, None, None) == 1
