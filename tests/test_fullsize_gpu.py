"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times: the whole result against digests of the oracle's result
(computed once by tests/golden/make_full_size_hashes.py, which calls only the
oracle), sampled pairs the oracle computes one by one (merge counts and
binary64 J), every size, and the invariants that hold at any size (symmetry,
C_ii = |X_i|, C_ij <= min, J_ii = 1, 0 <= J <= 1).  Integers and correctly
rounded quotients: tolerance zero."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size_sha256.json")


def golden(name):
    with open(GOLDEN) as f:
        return json.load(f)[name]


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def check_digests(name, off, ids, C, s, J):
    """The whole result against the oracle's, by SHA-256 of C (uint32), sizes
    (uint64) and the bit patterns of J, stored by
    tests/golden/make_full_size_hashes.py (which calls only the oracle)."""
    g = golden(name)
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(off, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(ids, dtype="<u8").tobytes())
    assert h.hexdigest() == g["input_sha256"], "the generator drew another collection"
    assert sha(np.asarray(C).astype(np.uint32)) == g["C_u32_sha256"]
    assert sha(np.asarray(s).astype(np.uint64)) == g["sizes_u64_sha256"]
    assert sha(np.asarray(J).view(np.uint64)) == g["J_f64_sha256"]

pytestmark = pytest.mark.gpu


def check_sampled(off, ids, C, sizes, J, pairs=384, seed=5):
    n = len(off) - 1
    np.testing.assert_array_equal(sizes, oracle.sizes_of(off, ids))
    C = C.astype(np.uint64)
    # invariants over the whole matrix
    np.testing.assert_array_equal(C, C.T)
    np.testing.assert_array_equal(J.view(np.uint64), J.T.view(np.uint64))
    np.testing.assert_array_equal(np.diag(C), sizes)
    assert np.all(C <= np.minimum(sizes[:, None], sizes[None, :]))
    assert np.all((J >= 0.0) & (J <= 1.0))
    assert np.all(np.diag(J) == 1.0)
    # sampled pairs against the plain merge
    rng = np.random.default_rng(seed)
    pi = rng.integers(0, n, pairs).astype(np.uint64)
    pj = rng.integers(0, n, pairs).astype(np.uint64)
    Co, Jo = oracle.pairs(off, ids, pi, pj)
    np.testing.assert_array_equal(C[pi, pj], Co)
    np.testing.assert_array_equal(J[pi, pj].view(np.uint64), Jo.view(np.uint64))


@pytest.fixture(scope="module")
def clade1024():
    return synth.clade1024()


@pytest.mark.timeout(900)
def test_clade1024_full_size(gpu, clade1024):
    """The benchmark's workload (1024 samples, 1.3e9 values) with the automatic
    product (SM pairs) and with the two-or-more filter: sampled parity, and the
    two runs byte-identical."""
    off, ids = clade1024
    with jsim.Context(id_bits=32) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        assert ctx.stats()["variant"] == "tc2"
    check_sampled(off, ids, C, s, J)
    check_digests("clade1024", off, ids, C, s, J)
    with jsim.Context(id_bits=32, filter_min=2) as ctx:
        C2, s2, J2 = ctx.all_pairs(off, ids)
    np.testing.assert_array_equal(C2, C)
    np.testing.assert_array_equal(s2, s)
    np.testing.assert_array_equal(J2.view(np.uint64), J.view(np.uint64))


@pytest.mark.timeout(900)
def test_clade1024_device_input_whole_result(gpu, clade1024):
    """Device-resident input (the benchmark's timed call: plain row batches,
    no streaming) gives the oracle's whole result, by digest."""
    import torch
    off, ids = clade1024
    d_off = torch.from_numpy(off.view(np.int64)).cuda()
    d_ids = torch.from_numpy(ids.view(np.int64)).cuda()
    with jsim.Context(id_bits=32) as ctx:
        C, s, J = ctx.all_pairs(d_off, d_ids)
        torch.cuda.synchronize()
        C = C.view(torch.int32).cpu().numpy().view(np.uint32)
        s = s.view(torch.int64).cpu().numpy().view(np.uint64)
        J = J.cpu().numpy()
    check_digests("clade1024", off, ids, C, s, J)


def test_ancestral64_whole_result_digest(gpu):
    off, ids = synth.ancestral64()
    with jsim.Context() as ctx:
        C, s, J = ctx.all_pairs(off, ids)
    check_digests("ancestral64", off, ids, C, s, J)


@pytest.mark.timeout(900)
def test_batched_recipe_full_size_subset(gpu):
    """The first 12 collections of the 200-collection recipe at full size
    (n ~ U{8..512}, sizes log-normal median 2e5 in [1e4, 5e6]) through one
    batched call."""
    cols = synth.batched_collections(count=12)
    with jsim.Context(id_bits=32) as ctx:
        outs = ctx.all_pairs_batched(cols)
    for (off, ids), (C, s, J) in zip(cols, outs):
        check_sampled(off, ids, C, s, J, pairs=128)


@pytest.mark.timeout(1200)
def test_serving_full_size_sampled(gpu):
    """The serving workload at full size (2048 reference samples of median
    1e6 values: a 171 GB resident index): one request of 6 query samples,
    whose counts and J against 48 sampled reference samples are merged by
    the oracle; invariants over every reference column."""
    roff, rids = synth.serving_reference()
    qoff, qids = synth.serving_queries(0, 6)
    n_ref = len(roff) - 1
    with jsim.Context(id_bits=32) as ctx:
        with jsim.Index(ctx, roff, rids, max_batch_samples=64, max_batch_values=int(qoff[-1])) as ix:
            r = ix.submit(qoff, qids)
            C, qs, J = r.wait()
            r.free()
            rsz = ix.ref_sizes()
    C = C.astype(np.uint64)
    np.testing.assert_array_equal(qs, oracle.sizes_of(qoff, qids))
    assert np.all(C <= np.minimum(qs[:, None], np.asarray(rsz, dtype=np.uint64)[None, :]))
    assert np.all((J >= 0.0) & (J <= 1.0))
    cols = np.sort(np.random.default_rng(9).choice(n_ref, 48, replace=False))
    segs = [rids[int(roff[j]):int(roff[j + 1])] for j in cols]
    soff = np.zeros(len(segs) + 1, dtype=np.uint64)
    soff[1:] = np.cumsum([len(s) for s in segs])
    Co, qso, Jo = oracle.cross(qoff, qids, soff, np.concatenate(segs))
    np.testing.assert_array_equal(C[:, cols], Co)
    np.testing.assert_array_equal(J[:, cols].view(np.uint64), Jo.view(np.uint64))


@pytest.mark.timeout(1800)
def test_streamed_full_size_sampled(gpu):
    """The out-of-HBM workload at full size (4096 samples, median 2e6 values
    in [0, 2^40), about 1.1e10 values = 88 GB of host memory, 64-bit counts)
    through the streamed call with the benchmark's 1 GiB staging: sampled
    pairs against the oracle's merges, and the invariants over the whole
    matrix."""
    off, ids = synth.clade4096()
    with jsim.Context(count_bits=64, id_bits=40) as ctx:
        C, s, J = ctx.all_pairs_streamed(off, ids, staging_bytes=1 << 30)
    check_sampled(off, ids, C, s, J, pairs=128)
