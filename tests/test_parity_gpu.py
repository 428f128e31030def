"""GPU parity: the CUDA path through the C-ABI against the CPU oracles.

C, |X_i| and the filter/rank/packed words are integers and must match
bit for bit; J is the correctly rounded binary64 quotient of the same
integers, so it must match bit for bit as well (tolerance 0).
"""
import numpy as np
import pytest

import oracle
from oracle import packed
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu

VARIANTS = ["popc", "b1", "i8", "f8", "tc", "tc2"]


def collection(segs):
    offsets = np.zeros(len(segs) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([len(s) for s in segs])
    ids = np.concatenate([np.asarray(s, dtype=np.uint64) for s in segs]) if segs else np.zeros(0, np.uint64)
    return offsets, ids.astype(np.uint64)


def to_np(t):
    """torch CUDA/CPU tensor or ndarray -> ndarray (unsigned views kept)."""
    import torch
    if isinstance(t, np.ndarray):
        return t
    m = {torch.uint64: (torch.int64, np.uint64), torch.uint32: (torch.int32, np.uint32)}
    if t.dtype in m:
        sdt, ndt = m[t.dtype]
        return t.view(sdt).cpu().numpy().view(ndt)
    return t.cpu().numpy()


def assert_same(res, ref):
    C, sizes, J = res
    Co, so, Jo = ref
    np.testing.assert_array_equal(np.asarray(sizes, dtype=np.uint64), so)
    np.testing.assert_array_equal(np.asarray(C).astype(np.uint64), Co)
    # bit-exact binary64
    np.testing.assert_array_equal(np.asarray(J).view(np.uint64), Jo.view(np.uint64))


@pytest.fixture(scope="module")
def c1():
    return synth.ancestral64()


@pytest.fixture(scope="module")
def c1_ref(c1):
    return oracle.all_pairs(*c1)


@pytest.mark.parametrize("variant", VARIANTS)
def test_ancestral64_host_io(gpu, c1, c1_ref, variant):
    with jsim.Context(variant=variant) as ctx:
        assert_same(ctx.all_pairs(*c1), c1_ref)
        assert ctx.stats()["variant"] == variant


@pytest.mark.parametrize("batch_rows", [1 << 12, 1 << 16, 3 << 14, 1 << 20, 1 << 26])
def test_ancestral64_batch_invariance(gpu, c1, c1_ref, batch_rows):
    """Eq. 4: any row-batch size gives the same C (several batches, a ragged last one)."""
    with jsim.Context(batch_rows=batch_rows) as ctx:
        assert_same(ctx.all_pairs(*c1), c1_ref)
        st = ctx.stats()
        assert st["batch_rows"] == batch_rows
        assert (st["batches"] > 1) == (batch_rows < 2**20)


@pytest.mark.parametrize("count_bits,word_bits", [(64, 64), (32, 32), (64, 32)])
def test_ancestral64_widths(gpu, c1, c1_ref, count_bits, word_bits):
    with jsim.Context(count_bits=count_bits, word_bits=word_bits) as ctx:
        assert_same(ctx.all_pairs(*c1), c1_ref)


def test_ancestral64_device_io(gpu, c1, c1_ref):
    import torch
    off = torch.from_numpy(c1[0].view(np.int64)).cuda()
    ids = torch.from_numpy(c1[1].view(np.int64)).cuda()
    with jsim.Context() as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        torch.cuda.synchronize()
        res = (to_np(C), to_np(s), to_np(J))
    assert_same(res, c1_ref)


@pytest.mark.parametrize("n,median", [(130, 2e4), (1, 5e4), (257, 3e3)])
def test_clade_recipe_scaled(gpu, n, median):
    """The 1024-sample clade recipe at sizes the oracle finishes in seconds
    (ragged n spans several tiles and a partial one)."""
    off, ids = synth.clade1024(n=n, median=median)
    ref = oracle.all_pairs(off, ids)
    for v in VARIANTS:
        with jsim.Context(variant=v) as ctx:
            assert_same(ctx.all_pairs(off, ids), ref)


def test_edge_cases(gpu):
    segs = [[], [], [0], [0, 2**64 - 1], [5, 5, 5, 7], list(range(1000, 1300)), [2**63, 2**63 + 1],
            [2**64 - 1]]
    off, ids = collection(segs)
    ref = oracle.all_pairs(off, ids)
    with jsim.Context() as ctx:
        assert_same(ctx.all_pairs(off, ids), ref)
    # all empty
    off, ids = collection([[], [], []])
    with jsim.Context() as ctx:
        C, s, J = ctx.all_pairs(off, ids)
    assert np.all(C == 0) and np.all(s == 0) and np.all(J == 1.0)
    # n = 0
    with jsim.Context() as ctx:
        C, s, J = ctx.all_pairs(np.zeros(1, np.uint64), np.zeros(0, np.uint64))
    assert C.shape == (0, 0)


def test_errors(gpu):
    with jsim.Context() as ctx:
        off, ids = collection([[1, 2, 3], [4, 3]])
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs(off, ids)
        assert e.value.name == "JSIM_ERR_UNSORTED"
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs(np.array([1, 3], np.uint64), np.array([1, 2, 3], np.uint64))
        assert e.value.name == "JSIM_ERR_ARG"
    with jsim.Context(id_bits=20) as ctx:
        off, ids = collection([[1, 2**20], [4]])
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs(off, ids)
        assert e.value.name == "JSIM_ERR_ID_RANGE"
        # the context is still usable after an error
        off, ids = collection([[1, 2], [2, 3]])
        C, s, J = ctx.all_pairs(off, ids)
        assert C[0, 1] == 1 and J[0, 1] == 1 / 3


@pytest.mark.parametrize("lo,width", [(0, 1 << 20), (1 << 18, 1 << 16), (123 * 64, 64 * 1000)])
def test_pack_matches_packed_oracle(gpu, c1, lo, width):
    """Filter (Eq. 5), ranks (Eq. 6) and bitmask words against the step-by-step model."""
    off, ids = c1
    sub_off = off[:9]
    sub_ids = ids[:int(off[8])]
    ref = packed.run_batch(sub_off, sub_ids, lo, width, 64)
    with jsim.Context() as ctx:
        filt, words, R, sz = ctx.pack(sub_off, sub_ids, lo, width)
    assert R == ref["R"]
    fbits = np.unpackbits(filt.view(np.uint8), bitorder="little").astype(bool)
    np.testing.assert_array_equal(fbits, ref["f"])
    np.testing.assert_array_equal(words[:, :ref["words"].shape[1]], ref["words"])
    np.testing.assert_array_equal(sz, ref["ahat"])


def popcount_product_ref(X, W):
    return packed.popcount_product(np.ascontiguousarray(X[:, :W]))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,W,density", [(1, 1, 0.5), (64, 64, 0.5), (65, 70, 0.05), (130, 300, 1.0),
                                         (300, 129, 0.3), (200, 1000, 0.01), (128, 4096, 1.0)])
def test_product_random_bits(gpu, variant, n, W, density):
    """The semiring product alone (Eq. 7) on random packed words, all-ones included."""
    import torch
    rng = np.random.default_rng(n * 1000 + W)
    stride = W + 3
    bits = rng.random((n, stride * 64)) < density
    X = np.packbits(bits, axis=1, bitorder="little").view(np.uint64).copy()
    ref = popcount_product_ref(X, W)
    with jsim.Context(count_bits=64) as ctx:
        Xd = torch.from_numpy(X.view(np.int64)).cuda()
        C = ctx.product(Xd, n, W, stride, variant=variant)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_np(C), ref)


@pytest.mark.parametrize("variant", VARIANTS)
def test_product_all_ones_long(gpu, variant):
    """Adversarial exactness: all-ones rows over 2^23 bit-rows (every count is
    8388608; f32 accumulation must stay exact, so slices are capped)."""
    import torch
    n, W = 130, 1 << 17
    Xd = torch.full((n, W), -1, dtype=torch.int64, device="cuda")
    with jsim.Context(count_bits=64) as ctx:
        C = ctx.product(Xd, n, W, W, variant=variant)
        torch.cuda.synchronize()
    assert np.all(to_np(C) == W * 64)


@pytest.mark.parametrize("variant", VARIANTS[1:])
def test_variants_agree_on_clade_batches(gpu, variant):
    """All product variants give byte-identical C, sizes and J on the clade recipe."""
    off, ids = synth.clade1024(n=200, median=5e4)
    with jsim.Context(variant="popc", batch_rows=1 << 28) as ctx:
        ref = ctx.all_pairs(off, ids)
    with jsim.Context(variant=variant, batch_rows=1 << 28) as ctx:
        out = ctx.all_pairs(off, ids)
    for a, b in zip(out, ref):
        np.testing.assert_array_equal(a.view(np.uint8), b.view(np.uint8))


# ---- filter_min 2: the product over rows two or more samples hold ------------------

@pytest.mark.parametrize("variant", ["popc", "tc", "tc2", "f8"])
@pytest.mark.parametrize("batch_rows", [0, 1 << 14])
def test_two_or_more_filter_ancestral64(gpu, c1, c1_ref, variant, batch_rows):
    """Dropping rows only one sample holds leaves C, sizes and J unchanged."""
    with jsim.Context(variant=variant, batch_rows=batch_rows, filter_min=2) as ctx:
        assert_same(ctx.all_pairs(*c1), c1_ref)
        st2 = ctx.stats()
    with jsim.Context(variant=variant, batch_rows=batch_rows) as ctx:
        ctx.all_pairs(*c1)
        st1 = ctx.stats()
    assert st2["rows_nonzero"] < st1["rows_nonzero"]


@pytest.mark.parametrize("n,median", [(130, 2e4), (257, 5e3)])
def test_two_or_more_filter_clade(gpu, n, median):
    off, ids = synth.clade1024(n=n, median=median)
    ref = oracle.all_pairs(off, ids)
    for count_bits in (32, 64):
        with jsim.Context(filter_min=2, count_bits=count_bits) as ctx:
            assert_same(ctx.all_pairs(off, ids), ref)


def test_two_or_more_filter_edge_cases(gpu):
    segs = [[], [0], [0, 0, 0], [5, 5, 9], [9], list(range(100, 400)), list(range(100, 400)), [2**64 - 1],
            [2**64 - 1, 2**64 - 1], [7, 8, 9, 10], []]
    off, ids = collection(segs)
    ref = oracle.all_pairs(off, ids)
    for br in (0, 64, 1 << 20):
        with jsim.Context(filter_min=2, batch_rows=br) as ctx:
            assert_same(ctx.all_pairs(off, ids), ref)
    # every row held by one sample: nothing to multiply, the diagonal is |X_i|
    off, ids = collection([[1, 2, 3], [4, 5], [], [6]])
    with jsim.Context(filter_min=2) as ctx:
        assert_same(ctx.all_pairs(off, ids), oracle.all_pairs(off, ids))
        assert ctx.stats()["words"] == 0
    with pytest.raises(jsim.JsimError):
        jsim.Context(filter_min=3)


@pytest.mark.parametrize("lo,width", [(0, 1 << 20), (123 * 64, 64 * 1000)])
def test_pack_two_or_more_matches_packed_oracle(gpu, c1, lo, width):
    off, ids = c1
    sub_off = off[:9]
    sub_ids = ids[:int(off[8])]
    ref = packed.run_batch(sub_off, sub_ids, lo, width, 64, min_count=2)
    with jsim.Context(filter_min=2) as ctx:
        filt, words, R, sz = ctx.pack(sub_off, sub_ids, lo, width)
    assert R == ref["R"]
    fbits = np.unpackbits(filt.view(np.uint8), bitorder="little").astype(bool)
    np.testing.assert_array_equal(fbits, ref["f"])
    np.testing.assert_array_equal(words[:, :ref["words"].shape[1]], ref["words"])
    np.testing.assert_array_equal(sz, ref["ahat"])


@pytest.mark.parametrize("n,m,p", [(130, 1 << 20, 0.01), (64, 1 << 22, 1e-3), (200, 1 << 16, 0.3)])
@pytest.mark.parametrize("variant", ["auto", "popc", "tc", "tc2"])
def test_bernoulli_matrices(gpu, n, m, p, variant):
    """The paper's synthetic indicator matrices (every entry present with
    probability p) at three densities, with both filters; at low density the
    two-or-more filter keeps far fewer rows."""
    off, ids = synth.bernoulli(n, m, p)
    ref = oracle.all_pairs(off, ids)
    with jsim.Context(variant=variant, id_bits=max(20, (m - 1).bit_length())) as ctx:
        assert_same(ctx.all_pairs(off, ids), ref)
        w1 = ctx.stats()["words"]
    with jsim.Context(variant=variant, filter_min=2, batch_rows=1 << 14) as ctx:
        assert_same(ctx.all_pairs(off, ids), ref)
    with jsim.Context(variant=variant, filter_min=2) as ctx:
        assert_same(ctx.all_pairs(off, ids), ref)
        w2 = ctx.stats()["words"]
    assert w2 <= w1


@pytest.mark.parametrize("variant", ["auto", "popc", "tc2"])
def test_row_permutation_invariance(gpu, variant):
    """Values relabelled by a bijection of their 32-bit domain (a reordering
    of the indicator matrix's rows, Sec. III-C): the GPU path gives the
    original collection's oracle results, with either filter and batch size."""
    from test_oracle import permute_rows
    off, ids = synth.clade1024(n=130, median=2e4)
    ref = oracle.all_pairs(off, ids)
    poff, pids = permute_rows(off, ids, bits=32)
    with jsim.Context(variant=variant, id_bits=32) as ctx:
        assert_same(ctx.all_pairs(poff, pids), ref)
    with jsim.Context(variant=variant, filter_min=2, batch_rows=1 << 26) as ctx:
        assert_same(ctx.all_pairs(poff, pids), ref)


@pytest.mark.parametrize("filter_min", [1, 2])
def test_useful_work_count(gpu, c1, filter_min):
    """bitops_useful = 64 x the pairs (i <= j) of nonzero packed words per
    word column, summed over batches: against the packed step oracle's words
    for the same batches; the dense count is 64 x W x n(n+1)/2 as before."""
    off, ids = c1
    mt = 1 << 16
    F = 0
    for lo in range(0, 1 << 20, mt):
        words = packed.run_batch(off, ids, lo, mt, min_count=filter_min)["words"]
        nnz = (words != 0).sum(axis=0).astype(np.int64)
        F += int((nnz * (nnz + 1) // 2).sum())
    with jsim.Context(batch_rows=mt, filter_min=filter_min, count_useful=True) as ctx:
        ctx.all_pairs(*c1)
        st = ctx.stats()
        assert st["bitops_useful"] == 64.0 * F
        assert 0 < st["bitops_useful"] <= st["bitops_dense"]
        # a streamed call packs super-batches of several row batches: fewer,
        # longer word columns, so its count differs but is also positive
        ctx.all_pairs_streamed(*c1, staging_bytes=4 << 20)
        assert 0 < ctx.stats()["bitops_useful"] <= ctx.stats()["bitops_dense"]
    with jsim.Context(batch_rows=mt, filter_min=filter_min) as ctx:
        ctx.all_pairs(*c1)
        assert ctx.stats()["bitops_useful"] == 0.0


@pytest.mark.parametrize("filter_min", [1, 2])
def test_split_contraction_parts_sum_to_the_whole(gpu, c1, c1_ref, filter_min):
    """jsim_all_pairs_part over 1, 2, 3 and 5 parts (emulating that many
    devices one after the other), summed on the host and finished, gives the
    oracle's C and J bit for bit; a part past the last batch counts nothing."""
    with jsim.Context(batch_rows=1 << 14, filter_min=filter_min) as ctx:
        for parts in (1, 2, 3, 5):
            acc = None
            for p in range(parts):
                Cp, sp = ctx.all_pairs_part(*c1, p, parts)
                np.testing.assert_array_equal(sp, c1_ref[1])
                acc = Cp.astype(np.uint64) if acc is None else acc + Cp.astype(np.uint64)
            C, J = ctx.finish(acc.astype(np.uint32), sp)
            assert_same((C, sp, J), c1_ref)
        # more parts than batches (64 here): part 0 of 200 holds none
        Cp, _ = ctx.all_pairs_part(*c1, 0, 200)
        assert not Cp.any()


def test_split_contraction_device(gpu):
    import torch
    off, ids = synth.clade1024(n=130, median=2e4)
    ref = oracle.all_pairs(off, ids)
    d_off = torch.from_numpy(off.view(np.int64)).cuda()
    d_ids = torch.from_numpy(ids.view(np.int64)).cuda()
    with jsim.Context(id_bits=32, count_bits=64) as ctx:
        acc = None
        for p in range(4):
            Cp, sp = ctx.all_pairs_part(d_off, d_ids, p, 4)
            Ci = Cp.view(torch.int64)  # the same bits; the sums stay below 2^63
            acc = Ci.clone() if acc is None else acc + Ci
        C, J = ctx.finish(acc, sp)
        torch.cuda.synchronize()
        assert_same((to_np(C), to_np(sp), J.cpu().numpy()), ref)
    with jsim.Context() as ctx:
        with pytest.raises(jsim.JsimError):
            ctx.all_pairs_part(off, ids, 4, 4)
