"""Distance and threshold outputs against the oracle.

The distance D = 1 - J is the binary64 subtraction 1.0 - J of the correctly
rounded J, so it is compared bit for bit with the oracle's; threshold lists
are compared as exact (i, j, value) sequences in row-major order."""
import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu


def same_bits(a, b):
    np.testing.assert_array_equal(np.asarray(a, dtype=np.float64).view(np.uint64),
                                  np.asarray(b, dtype=np.float64).view(np.uint64))


def collection(segs):
    offsets = np.zeros(len(segs) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([len(s) for s in segs])
    ids = np.concatenate([np.asarray(s, dtype=np.uint64) for s in segs]) if segs else np.zeros(0, np.uint64)
    return offsets, ids.astype(np.uint64)


def oracle_D(off, ids):
    C, s, _ = oracle.all_pairs(off, ids)
    return C, s, oracle.distance_matrix(C, s, s)


@pytest.mark.parametrize("filter_min", [1, 2])
def test_distance_plain_streamed_batched(gpu, filter_min):
    import torch
    c1 = synth.ancestral64()
    c2 = synth.clade1024(n=130, median=2e4)
    c3 = collection([[], [], [0, 5], [5], list(range(100)), list(range(50, 150)), [2**63]])
    refs = [oracle_D(*c) for c in (c1, c2, c3)]
    with jsim.Context(distance=True, filter_min=filter_min) as ctx:
        for c, (Co, so, Do) in zip((c1, c2, c3), refs):
            C, s, D = ctx.all_pairs(*c)
            np.testing.assert_array_equal(C.astype(np.uint64), Co)
            same_bits(D, Do)
            C, s, D = ctx.all_pairs_streamed(*c, staging_bytes=1 << 20)
            same_bits(D, Do)
            off, ids = c
            d_off = torch.from_numpy(off.view(np.int64)).cuda()
            d_ids = torch.from_numpy(ids.view(np.int64)).cuda()
            C, s, D = ctx.all_pairs(d_off, d_ids)
            same_bits(D.cpu().numpy(), Do)
        # the batched call plans one value span per collection (no 2^63 outlier)
        c4 = collection([[], [], [0, 5], [5], list(range(100)), list(range(50, 150)), [7, 10**6]])
        outs = ctx.all_pairs_batched([c1, c2, c4])
        for (C, s, D), (Co, so, Do) in zip(outs, refs[:2] + [oracle_D(*c4)]):
            same_bits(D, Do)
    # the similarity context still gives J, and D is exactly 1.0 - J
    with jsim.Context() as ctx:
        _, _, J = ctx.all_pairs(*c2)
    same_bits(1.0 - J, refs[1][2])


def test_distance_serving(gpu):
    roff, rids = synth.serving_reference(n=96, median=2e4)
    qoff, qids = synth.serving_queries(0, 12, n_ref=96, median=2e4)
    Co, qs, _ = oracle.cross(qoff, qids, roff, rids)
    rs = oracle.sizes_of(roff, rids)
    Do = oracle.distance_matrix(Co, qs, rs)
    with jsim.Context(id_bits=32, distance=True) as ctx:
        with jsim.Index(ctx, roff, rids, max_batch_samples=16, max_batch_values=1 << 22) as ix:
            r = ix.submit(qoff, qids)
            C, s, D = r.wait()
            r.free()
    np.testing.assert_array_equal(C.astype(np.uint64), Co)
    same_bits(D, Do)


def threshold_ref(M, tau, below=False):
    n = M.shape[0]
    sel = (M <= tau) if below else (M >= tau)
    sel &= np.triu(np.ones((n, n), dtype=bool), 1)
    i, j = np.nonzero(sel)  # row-major order
    return i.astype(np.uint64), j.astype(np.uint64), M[i, j]


@pytest.mark.parametrize("tau", [0.0, 0.05, 0.2, 0.5, 1.0, 1.5])
def test_threshold_host_matches_oracle_order(gpu, tau):
    off, ids = synth.clade1024(n=300, median=5e3)
    _, _, J = oracle.all_pairs(off, ids)
    ri, rj, rv = threshold_ref(J, tau)
    with jsim.Context() as ctx:
        pi, pj, val, cnt = ctx.threshold(J, tau)
        assert cnt == ri.size
        np.testing.assert_array_equal(pi, ri)
        np.testing.assert_array_equal(pj, rj)
        same_bits(val, rv)
        # a capacity below the count keeps the first pairs in order
        if cnt > 3:
            cap = cnt // 3
            pi, pj, val, cnt2 = ctx.threshold(J, tau, cap=cap)
            assert cnt2 == cnt and pi.size == cap
            np.testing.assert_array_equal(pi, ri[:cap])
            np.testing.assert_array_equal(pj, rj[:cap])
        # count only
        _, _, _, cnt3 = ctx.threshold(J, tau, cap=0)
        assert cnt3 == cnt


def test_threshold_device_and_distance(gpu):
    import torch
    off, ids = synth.ancestral64()
    C, s, _ = oracle.all_pairs(off, ids)
    D = oracle.distance_matrix(C, s, s)
    with jsim.Context(distance=True) as ctx:
        d_off = torch.from_numpy(off.view(np.int64)).cuda()
        d_ids = torch.from_numpy(ids.view(np.int64)).cuda()
        _, _, Dd = ctx.all_pairs(d_off, d_ids)
        for tau in (0.3, 0.6, 0.75):
            ri, rj, rv = threshold_ref(D, tau, below=True)
            pi, pj, val, cnt = ctx.threshold(Dd, tau, below=True)
            assert cnt == ri.size
            np.testing.assert_array_equal(pi.view(torch.int64).cpu().numpy().view(np.uint64), ri)
            np.testing.assert_array_equal(pj.view(torch.int64).cpu().numpy().view(np.uint64), rj)
            same_bits(val.cpu().numpy(), rv)


def test_threshold_edges_and_errors(gpu):
    with jsim.Context() as ctx:
        one = np.ones((1, 1))
        assert ctx.threshold(one, 0.5)[3] == 0
        n = 70
        J = np.full((n, n), 0.25)
        pi, pj, val, cnt = ctx.threshold(J, 0.25)
        assert cnt == n * (n - 1) // 2 and pi.size == cnt
        assert np.all(pi < pj)
        with pytest.raises(jsim.JsimError) as e:
            ctx.threshold(J, float("nan"))
        assert e.value.name == "JSIM_ERR_ARG"
        # still usable
        assert ctx.threshold(J, 0.3)[3] == 0
