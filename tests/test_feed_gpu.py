"""Page-locked host input to the plain all-pairs call on the block-sparse
path: the device reads the values in value-range pieces (one slice of every
sample per piece) while the batch loop runs on the pieces already there,
and the input is validated once it is all in.  Results are bit-identical to the same call
on device-resident input (which takes the windowed ingest where the fed call takes the
per-value one; itself checked against the oracle elsewhere) and
agree with the oracle on sampled pairs and every size; bad input (a descent
in a late piece, a value beyond id_bits) is reported before any output is
written; a collection where the automatic choice declines the block-sparse
product continues on the dense path after the last piece."""
import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu


def pinned(count):
    import torch
    return torch.empty(count, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)


def device_call(off, ids, **kw):
    import torch
    d_off = torch.from_numpy(off.view(np.int64)).cuda()
    d_ids = torch.from_numpy(ids.view(np.int64)).cuda()
    with jsim.Context(**kw) as ctx:
        C, s, J = ctx.all_pairs(d_off, d_ids)
        st = ctx.stats()
        torch.cuda.synchronize()
        dt = torch.int64 if kw.get("count_bits") == 64 else torch.int32
        ndt = np.uint64 if kw.get("count_bits") == 64 else np.uint32
        return (C.view(dt).cpu().numpy().view(ndt), s.view(torch.int64).cpu().numpy().view(np.uint64),
                J.cpu().numpy(), st)


def sampled(off, ids, C, s, J, pairs=256, distance=False):
    n = len(off) - 1
    np.testing.assert_array_equal(s, oracle.sizes_of(off, ids))
    rng = np.random.default_rng(3)
    pi = rng.integers(0, n, pairs).astype(np.uint64)
    pj = rng.integers(0, n, pairs).astype(np.uint64)
    Co, Jo = oracle.pairs(off, ids, pi, pj)
    np.testing.assert_array_equal(C[pi, pj].astype(np.uint64), Co)
    if not distance:
        np.testing.assert_array_equal(J[pi, pj].view(np.uint64), Jo.view(np.uint64))


@pytest.fixture(scope="module")
def clades():
    # 512 clade samples, about 1.2e8 values (0.95 GB): above the size from
    # which host input is fed piece by piece
    return synth.clade1024(n=512, median=1.6e5, alloc=pinned)


@pytest.mark.timeout(600)
@pytest.mark.parametrize("kw", [dict(), dict(variant="sparse", filter_min=2),
                                dict(variant="sparse", count_bits=64, distance=True),
                                dict(variant="sparse", batch_rows=1 << 24)])
def test_fed_input_equals_device_input(gpu, clades, kw):
    off, ids = clades
    assert ids.nbytes >= 512 << 20
    with jsim.Context(id_bits=32, **kw) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        st = ctx.stats()
    assert st["variant"] == "sparse"
    assert st["h2d_pieces"] >= 3, "the values were not fed piece by piece"
    assert st["h2d_bytes"] >= ids.nbytes
    # fed input takes the per-value ingest, device-resident input the
    # windowed one: the two ingests give the same words
    assert st["windows"] == 0
    Cd, sd, Jd, std = device_call(off, ids, id_bits=32, **kw)
    assert std["variant"] == "sparse" and std["windows"] > 0
    np.testing.assert_array_equal(C, Cd)
    np.testing.assert_array_equal(s, sd)
    np.testing.assert_array_equal(J.view(np.uint64), Jd.view(np.uint64))
    sampled(off, ids, C, s, J, distance=kw.get("distance", False))


@pytest.mark.timeout(600)
def test_fed_input_errors_write_nothing(gpu, clades):
    off, ids = clades
    n = len(off) - 1
    bad = pinned(len(ids))
    bad[:] = ids
    # a descent near the end of a sample: in the last pieces
    i = n // 2
    a, b = int(off[i]), int(off[i + 1])
    bad[b - 3], bad[b - 2] = bad[b - 2], bad[b - 3]
    outs = (np.full((n, n), 7, dtype=np.uint32), np.full(n, 7, dtype=np.uint64), np.full((n, n), -1.0))
    with jsim.Context(id_bits=32) as ctx:
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs(off, bad, out=outs)
        assert e.value.name == "JSIM_ERR_UNSORTED"
        # a value beyond id_bits, in the middle of a sample
        bad[b - 3], bad[b - 2] = bad[b - 2], bad[b - 3]
        bad[(a + b) // 2] = 1 << 40
        bad[(a + b) // 2 + 1 : b] = np.arange(1, b - (a + b) // 2, dtype=np.uint64) + (1 << 40)
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs(off, bad, out=outs)
        assert e.value.name == "JSIM_ERR_ID_RANGE"
        # the context keeps working
        C, s, J = ctx.all_pairs(off, ids)
    assert (outs[0] == 7).all() and (outs[1] == 7).all() and (outs[2] == -1.0).all()
    sampled(off, ids, C, s, J, pairs=64)


@pytest.mark.timeout(600)
def test_fed_input_auto_declines_to_dense(gpu):
    # Bernoulli rows: no sample order empties tensor-core blocks, so the
    # automatic choice goes on dense once every piece is in
    off, ids = synth.bernoulli(300, 1 << 25, 0.008, alloc=pinned)
    assert ids.nbytes >= 512 << 20
    kw = dict(id_bits=25, batch_rows=1 << 22)  # 8 row batches: fed in pieces
    with jsim.Context(**kw) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        st = ctx.stats()
    assert st["variant"] != "sparse"
    assert st["h2d_pieces"] >= 3
    Cd, sd, Jd, std = device_call(off, ids, **kw)
    assert std["variant"] == st["variant"]
    np.testing.assert_array_equal(C, Cd)
    np.testing.assert_array_equal(J.view(np.uint64), Jd.view(np.uint64))
    sampled(off, ids, C, s, J, pairs=64)
