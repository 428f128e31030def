"""Nearest neighbours (jsim_topk) against an ordering of the oracle's J:
largest J first, ties to the smaller index, the sample itself left out.
J is the oracle's bit-exact binary64, so the order is unique and compared
exactly."""
import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu


def topk_ref(J, k):
    n = J.shape[0]
    idx = np.empty((n, k), dtype=np.uint64)
    for i in range(n):
        j = np.arange(n)
        keep = j != i
        order = np.lexsort((j[keep], -J[i][keep]))  # last key primary: J descending, then index
        idx[i] = j[keep][order[:k]]
    return idx


def test_topk_ancestral64_host():
    off, ids = synth.ancestral64()
    C, s, J = oracle.all_pairs(off, ids)
    with jsim.Context() as ctx:
        for k in (1, 5, 63):
            idx, val = ctx.topk(J, k)
            np.testing.assert_array_equal(idx, topk_ref(J, k))
            np.testing.assert_array_equal(val.view(np.uint64),
                                          np.take_along_axis(J, idx.astype(np.int64), 1).view(np.uint64))


def test_topk_device_from_all_pairs_with_ties():
    import torch
    off, ids = synth.clade1024(n=300, median=5e3)
    # duplicate samples make exact ties in J
    segs = [ids[int(off[i]):int(off[i + 1])] for i in range(300)] + \
           [ids[int(off[i]):int(off[i + 1])] for i in (3, 3, 7)]
    off2 = np.zeros(len(segs) + 1, dtype=np.uint64)
    off2[1:] = np.cumsum([len(x) for x in segs])
    ids2 = np.concatenate(segs).astype(np.uint64)
    with jsim.Context(id_bits=32) as ctx:
        d_off = torch.from_numpy(off2.view(np.int64)).cuda()
        d_ids = torch.from_numpy(ids2.view(np.int64)).cuda()
        C, s, J = ctx.all_pairs(d_off, d_ids)
        idx, val = ctx.topk(J, 64)
        torch.cuda.synchronize()
        Jh = J.cpu().numpy()
        idxh = idx.view(torch.int64).cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(idxh, topk_ref(Jh, 64))
    Co, so, Jo = oracle.all_pairs(off2, ids2)
    np.testing.assert_array_equal(Jh.view(np.uint64), Jo.view(np.uint64))


def test_topk_errors():
    J = np.eye(4)
    with jsim.Context() as ctx:
        for k in (0, 4, 65):
            with pytest.raises(jsim.JsimError) as e:
                ctx.topk(J, k)
            assert e.value.name == "JSIM_ERR_ARG"
