"""GPU parity of the batched pattern: many independent collections per call,
each bit-exact against the CPU oracle (C, sizes, J)."""
import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu


def to_np(t):
    import torch
    if isinstance(t, np.ndarray):
        return t
    m = {torch.uint64: (torch.int64, np.uint64), torch.uint32: (torch.int32, np.uint32)}
    if t.dtype in m:
        sdt, ndt = m[t.dtype]
        return t.view(sdt).cpu().numpy().view(ndt)
    return t.cpu().numpy()


def assert_same(res, ref):
    C, s, J = (to_np(x) for x in res)
    Co, so, Jo = ref
    np.testing.assert_array_equal(s, so)
    np.testing.assert_array_equal(C.astype(np.uint64), Co)
    np.testing.assert_array_equal(J.view(np.uint64), Jo.view(np.uint64))


@pytest.fixture(scope="module")
def cols():
    """The batched recipe (n ~ U{8..512}, log-normal sizes, clade model) scaled so
    the oracle finishes in seconds, plus degenerate collections."""
    out = synth.batched_collections(count=10, n_lo=1, n_hi=300, median=4e3)
    out.append((np.zeros(4, np.uint64), np.zeros(0, np.uint64)))          # 3 empty samples
    out.append((np.array([0, 2], np.uint64), np.array([5, 9], np.uint64)))  # n = 1
    return out


@pytest.fixture(scope="module")
def refs(cols):
    return [oracle.all_pairs(o, i) for o, i in cols]


@pytest.mark.parametrize("variant,tile_n", [("auto", 0), ("tc", 256), ("tc", 128), ("auto", 128), ("popc", 0)])
def test_batched_host_io(gpu, cols, refs, variant, tile_n):
    """Every variant and both tensor tile shapes (128 x 256, and 128 x 128
    whose diagonal tiles unpack their rows once for both operands) on
    collections of 1 to 300 samples (one to three tiles, ragged)."""
    with jsim.Context(variant=variant, tile_n=tile_n) as ctx:
        outs = ctx.all_pairs_batched(cols)
        st = ctx.stats()
    if variant == "tc":
        assert st["tile_n"] == tile_n
    for res, ref in zip(outs, refs):
        assert_same(res, ref)


def test_batched_device_io_graph_replay(gpu, cols, refs):
    """Device inputs and outputs: the second call replays the captured graph;
    after the values change in place (same sizes) a replay gives the new result."""
    import torch
    dcols = [(torch.from_numpy(o.view(np.int64)).cuda(), torch.from_numpy(i.view(np.int64)).cuda())
             for o, i in cols]
    with jsim.Context() as ctx:
        first = ctx.all_pairs_batched(dcols)
        second = ctx.all_pairs_batched(dcols)
        torch.cuda.synchronize()
        for a, b, ref in zip(first, second, refs):
            assert_same(a, ref)
            assert_same(b, ref)
        # shift every value of collection 0 by one (sortedness and range kept)
        o0, i0 = cols[0]
        shifted = i0 + np.uint64(1)
        dcols[0][1].copy_(torch.from_numpy(shifted.view(np.int64)))
        third = ctx.all_pairs_batched(dcols)
        torch.cuda.synchronize()
        assert_same(third[0], oracle.all_pairs(o0, shifted))
        for a, ref in zip(third[1:], refs[1:]):
            assert_same(a, ref)


def test_batched_matches_plain_calls(gpu, cols):
    with jsim.Context(variant="tc") as ctx:
        outs = ctx.all_pairs_batched(cols)
        for (o, i), res in zip(cols, outs):
            plain = ctx.all_pairs(o, i)
            for a, b in zip(res, plain):
                np.testing.assert_array_equal(to_np(a).view(np.uint8), to_np(b).view(np.uint8))


def test_batched_errors(gpu):
    good = (np.array([0, 2], np.uint64), np.array([1, 2], np.uint64))
    bad = (np.array([0, 2], np.uint64), np.array([3, 2], np.uint64))
    with jsim.Context() as ctx:
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_batched([good, bad])
        assert e.value.name == "JSIM_ERR_UNSORTED"
        outs = ctx.all_pairs_batched([good])
        assert outs[0][2][0, 0] == 1.0


@pytest.mark.parametrize("variant", ["auto", "tc", "popc"])
def test_batched_two_or_more_filter(gpu, cols, refs, variant):
    with jsim.Context(variant=variant, id_bits=32, filter_min=2) as ctx:
        outs = ctx.all_pairs_batched(cols)
    for (C, s, J), ref in zip(outs, refs):
        assert_same((C, s, J), ref)


def test_batched_mixes_block_sparse_and_shared_launches(gpu):
    """With variant AUTO, collections of 256 to 2048 samples run as plain
    calls (the block-sparse product where the sketch says so) and the others
    share the batched launches: every result equals the oracle's, with host
    and device buffers, on a first call and on a replay."""
    import torch
    cols = [synth.clade1024(n=300, median=3e3), synth.clade1024(n=260, median=2e3, seed=77)]
    cols += synth.batched_collections(count=4, n_lo=5, n_hi=120, median=3e3)
    cols.insert(2, (np.zeros(3, np.uint64), np.zeros(0, np.uint64)))
    refs = [oracle.all_pairs(o, i) for o, i in cols]
    with jsim.Context(id_bits=32) as ctx:
        outs = ctx.all_pairs_batched(cols)
        st = ctx.stats()
    for res, ref in zip(outs, refs):
        assert_same(res, ref)
    assert st["bitops_done"] <= st["bitops_dense"]
    dcols = [(torch.from_numpy(o.view(np.int64)).cuda(), torch.from_numpy(i.view(np.int64)).cuda())
             for o, i in cols]
    with jsim.Context(id_bits=32) as ctx:
        for _ in range(2):
            outs = ctx.all_pairs_batched(dcols)
            torch.cuda.synchronize()
            for res, ref in zip(outs, refs):
                assert_same(res, ref)


def test_batched_mixed_input_error_in_a_large_collection(gpu):
    """An unsorted large collection (a plain call inside the batched call) is
    reported before anything runs, and the context keeps working."""
    import torch
    big_o, big_i = synth.clade1024(n=280, median=2e3)
    bad_i = big_i.copy()
    a, b = int(big_o[100]), int(big_o[101])
    bad_i[b - 3], bad_i[b - 2] = bad_i[b - 2], bad_i[b - 3]
    small = synth.batched_collections(count=2, n_lo=5, n_hi=60, median=2e3)
    dev = lambda o, i: (torch.from_numpy(o.view(np.int64)).cuda(), torch.from_numpy(i.view(np.int64)).cuda())
    with jsim.Context(id_bits=32) as ctx:
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_batched([dev(*small[0]), dev(big_o, bad_i), dev(*small[1])])
        assert e.value.name == "JSIM_ERR_UNSORTED"
        outs = ctx.all_pairs_batched([dev(*small[0]), dev(big_o, big_i)])
        torch.cuda.synchronize()
    assert_same(outs[0], oracle.all_pairs(*small[0]))
    assert_same(outs[1], oracle.all_pairs(big_o, big_i))
