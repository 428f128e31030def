"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times: the whole result against digests of the oracle's result
(computed once by tests/golden/make_full_size_hashes.py, which calls only the
oracle), sampled pairs the oracle computes one by one (merge counts and
binary64 J), every size, and the invariants that hold at any size (symmetry,
C_ii = |X_i|, C_ij <= min, J_ii = 1, 0 <= J <= 1).  Integers and correctly
rounded quotients: tolerance zero."""
import ctypes
import hashlib
import importlib.util
import json
import os

import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size_sha256.json")
_spec = importlib.util.spec_from_file_location(
    "make_full_size_hashes", os.path.join(os.path.dirname(GOLDEN), "make_full_size_hashes.py"))
hashes = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(hashes)  # the digest script's own fingerprint of an input


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
    choice (the block-sparse product), the dense SM-pair product, and the
    two-or-more filter: sampled parity, whole-result digests, and all runs
    byte-identical."""
    import torch
    torch.cuda.empty_cache()  # host input this large takes the block-sparse route only with room on the device
    off, ids = clade1024
    with jsim.Context(id_bits=32) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        assert ctx.stats()["variant"] == "sparse"
    check_sampled(off, ids, C, s, J)
    check_digests("clade1024", off, ids, C, s, J)
    for kw in (dict(variant="tc2"), dict(filter_min=2), dict(filter_min=2, variant="tc2")):
        with jsim.Context(id_bits=32, **kw) as ctx:
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
    for variant in ("auto", "tc2"):
        with jsim.Context(id_bits=32, variant=variant) as ctx:
            C, s, J = ctx.all_pairs(d_off, d_ids)
            torch.cuda.synchronize()
            C = C.view(torch.int32).cpu().numpy().view(np.uint32)
            s = s.view(torch.int64).cpu().numpy().view(np.uint64)
            J = J.cpu().numpy()
        check_digests("clade1024", off, ids, C, s, J)


@pytest.mark.timeout(900)
def test_clade1024_pinned_host_input_whole_result(gpu, clade1024):
    """Page-locked host input (the benchmark's end-to-end call): the values
    are copied piece by piece while the block-sparse batch loop runs; the
    oracle's whole result, by digest, with both filters."""
    import torch
    torch.cuda.empty_cache()  # host input this large takes the block-sparse route only with room on the device
    off, ids = clade1024
    pin = torch.empty(len(ids), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    pin[:] = ids
    for kw in ({}, dict(filter_min=2)):
        with jsim.Context(id_bits=32, **kw) as ctx:
            C, s, J = ctx.all_pairs(off, pin)
            st = ctx.stats()
        assert st["variant"] == "sparse"
        assert st["h2d_pieces"] >= 3, "the input was not fed piece by piece"
        check_digests("clade1024", off, ids, C, s, J)


def test_ancestral64_whole_result_digest(gpu):
    off, ids = synth.ancestral64()
    with jsim.Context() as ctx:
        C, s, J = ctx.all_pairs(off, ids)
    check_digests("ancestral64", off, ids, C, s, J)


def batched_call_twice(ctx, dcols):
    """jsim_all_pairs_batched on device-resident collections with the same
    preallocated device outputs twice (capture, then replay of the CUDA
    graph); the results of the replay, on the host."""
    import torch
    k = len(dcols)
    dev = dcols[0][0].device
    ns = [o.numel() - 1 for o, _ in dcols]
    Cs = [torch.empty((n, n), dtype=torch.uint32, device=dev) for n in ns]
    Ss = [torch.empty(n, dtype=torch.uint64, device=dev) for n in ns]
    Js = [torch.empty((n, n), dtype=torch.float64, device=dev) for n in ns]
    sets = (jsim.Sets * k)()
    for c, (o, i) in enumerate(dcols):
        sets[c] = jsim.Sets(ns[c], o.data_ptr(), i.data_ptr() if i.numel() else None, jsim.MEM_DEVICE)
    arr = lambda L: (ctypes.c_void_p * k)(*[t.data_ptr() for t in L])
    Cp, Sp, Jp = arr(Cs), arr(Ss), arr(Js)
    lib = jsim.load()
    for _ in range(2):
        ctx._order()
        jsim._check(lib.jsim_all_pairs_batched(ctx._h, sets, k, Cp, Sp, Jp, jsim.MEM_DEVICE), ctx._h)
    torch.cuda.synchronize()
    return [(C.view(torch.int32).cpu().numpy().view(np.uint32), S.view(torch.int64).cpu().numpy().view(np.uint64),
             J.cpu().numpy()) for C, S, J in zip(Cs, Ss, Js)]


@pytest.mark.timeout(1500)
def test_batched_recipe_full_size_whole_results(gpu):
    """All 200 collections of the batched recipe at full size (n ~ U{8..512},
    sizes log-normal median 2e5 in [1e4, 5e6]: 53,900 samples, 1.8e10
    values) through batched calls on device-resident input (the graph
    replay, as the benchmark times it), in waves of 25 collections: C, sizes
    and J of every collection against digests of the oracle's results."""
    import torch
    g = golden("batched200")
    hC, hs, hJ, hfp = (hashlib.sha256() for _ in range(4))
    bad = []
    with jsim.Context(id_bits=32) as ctx:
        for w0 in range(0, g["collections"], 25):
            cols = [synth.batched_collection(k) for k in range(w0, min(w0 + 25, g["collections"]))]
            dcols = [(torch.from_numpy(o.view(np.int64)).cuda(), torch.from_numpy(i.view(np.int64)).cuda())
                     for o, i in cols]
            outs = batched_call_twice(ctx, dcols)
            del dcols
            for k, ((off, ids), (C, S, J)) in enumerate(zip(cols, outs)):
                hashes.fingerprint(off, ids, hfp)
                c32 = np.ascontiguousarray(C.astype("<u4"))
                hC.update(c32.tobytes())
                hs.update(np.ascontiguousarray(S, dtype="<u8").tobytes())
                hJ.update(np.ascontiguousarray(J.view(np.uint64), dtype="<u8").tobytes())
                one = hashlib.sha256()
                one.update(c32.tobytes())
                one.update(np.ascontiguousarray(S, dtype="<u8").tobytes())
                one.update(np.ascontiguousarray(J.view(np.uint64), dtype="<u8").tobytes())
                if one.hexdigest()[:16] != g["per_collection_sha256_16"][w0 + k]:
                    bad.append(w0 + k)
            del cols, outs
    assert hfp.hexdigest() == g["input_fingerprint_sha256"], "the generator drew other collections"
    assert not bad, "collections whose results differ from the oracle's: %s" % bad
    assert hC.hexdigest() == g["C_u32_sha256"]
    assert hs.hexdigest() == g["sizes_u64_sha256"]
    assert hJ.hexdigest() == g["J_f64_sha256"]


@pytest.mark.timeout(1500)
def test_serving_full_size_whole_results(gpu):
    """The serving workload at full size (2048 reference samples of median
    1e6 values: a 171 GB resident index): the first 256 query samples of the
    recipe, submitted at once as requests of U{1..64} samples (so the server
    batches them as they arrive), every result against digests of the
    oracle's merges of every query sample with every reference sample; and a
    sampled check of 48 reference columns for diagnosis."""
    g = golden("serve2048_q256")
    roff, rids = synth.serving_reference()
    qoff, qids = synth.serving_queries(0, g["queries"])
    assert hashes.fingerprint(roff, rids).hexdigest() == g["ref_fingerprint_sha256"]
    assert hashes.fingerprint(qoff, qids).hexdigest() == g["query_fingerprint_sha256"]
    n_ref, nq = len(roff) - 1, len(qoff) - 1
    rng = np.random.default_rng(21)
    cuts = [0]
    while cuts[-1] < nq:
        cuts.append(min(nq, cuts[-1] + int(rng.integers(1, 65))))
    C = np.zeros((nq, n_ref), dtype=np.uint32)
    qs = np.zeros(nq, dtype=np.uint64)
    J = np.zeros((nq, n_ref), dtype=np.float64)
    with jsim.Context(id_bits=32) as ctx:
        sizes = np.diff(qoff.astype(np.int64))
        with jsim.Index(ctx, roff, rids, max_batch_samples=64, max_batch_values=int(np.sort(sizes)[-64:].sum())) as ix:
            reqs = []
            for a, b in zip(cuts[:-1], cuts[1:]):
                o = (qoff[a:b + 1] - qoff[a]).astype(np.uint64)
                reqs.append((a, b, ix.submit(o, qids[int(qoff[a]):int(qoff[b])])))
            for a, b, r in reqs:
                Cr, qr, Jr = r.wait()
                r.free()
                C[a:b], qs[a:b], J[a:b] = Cr, qr, Jr
            rsz = ix.ref_sizes()
    assert sha(np.ascontiguousarray(rsz, dtype="<u8")) == g["ref_sizes_u64_sha256"]
    cols = np.sort(np.random.default_rng(9).choice(n_ref, 48, replace=False))
    segs = [rids[int(roff[j]):int(roff[j + 1])] for j in cols]
    soff = np.zeros(len(segs) + 1, dtype=np.uint64)
    soff[1:] = np.cumsum([len(x) for x in segs])
    Co, qso, Jo = oracle.cross(qoff[:7], qids[:int(qoff[6])], soff, np.concatenate(segs))
    np.testing.assert_array_equal(C[:6][:, cols], Co)
    np.testing.assert_array_equal(J[:6][:, cols].view(np.uint64), Jo.view(np.uint64))
    assert sha(np.ascontiguousarray(qs, dtype="<u8")) == g["qsizes_u64_sha256"]
    assert sha(np.ascontiguousarray(C, dtype="<u4")) == g["C_u32_sha256"]
    assert sha(np.ascontiguousarray(J.view(np.uint64), dtype="<u8")) == g["J_f64_sha256"]


@pytest.mark.timeout(1800)
def test_streamed_full_size_whole_results(gpu):
    """The out-of-HBM workload at full size (4096 samples, median 2e6 values
    in [0, 2^40), about 1.1e10 values = 88 GB of host memory, 64-bit counts)
    through the streamed call with the benchmark's 1 GiB staging: C (uint64),
    sizes and J against digests of the oracle's result (counted by rows of
    the indicator matrix, range by range), sampled pairs against the
    oracle's merges, and the invariants over the whole matrix."""
    g = golden("stream4096")
    off, ids = synth.clade4096()
    # the input's fingerprint, range by range as the oracle visited it
    h = hashlib.sha256()
    n = len(off) - 1
    for lo, hi in zip(g["ranges"][:-1], g["ranges"][1:]):
        a = np.array([np.searchsorted(ids[int(off[i]):int(off[i + 1])], lo) + int(off[i]) for i in range(n)])
        b = np.array([np.searchsorted(ids[int(off[i]):int(off[i + 1])], hi) + int(off[i]) for i in range(n)])
        po = np.zeros(n + 1, dtype=np.uint64)
        po[1:] = np.cumsum(b - a)
        h.update(np.ascontiguousarray(po, dtype="<u8").tobytes())
        for i in range(n):
            h.update(np.ascontiguousarray(ids[a[i]:b[i]][::hashes.FP_STRIDE], dtype="<u8").tobytes())
    assert h.hexdigest() == g["input_fingerprint_sha256"], "the generator drew another collection"
    with jsim.Context(count_bits=64, id_bits=40) as ctx:
        C, s, J = ctx.all_pairs_streamed(off, ids, staging_bytes=1 << 30)
    check_sampled(off, ids, C, s, J, pairs=128)
    # the whole result against the oracle's, counted range by range
    assert sha(np.ascontiguousarray(s, dtype="<u8")) == g["sizes_u64_sha256"]
    assert sha(np.ascontiguousarray(C, dtype="<u8")) == g["C_u64_sha256"]
    assert sha(np.ascontiguousarray(J.view(np.uint64), dtype="<u8")) == g["J_f64_sha256"]
