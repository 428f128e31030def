"""The windowed ingest of the block-sparse variant: per window of rows, the
tiles' filter bitmaps and row classes are built in shared memory, ranks are
numbered range after range (each range rounded up to a word), and every
sample's words are gathered and stored whole.  It runs where samples have
values in most windows; C, sizes and J bit for bit against the oracle there,
with both filters, both count widths, the distance output, one to sixteen
tiles, ragged last tiles, empty and identical samples, repeated values,
windows packed by ranges of several windows (more ranges than resident
CTAs), batches of one scan granule, and bad input reported before any
output is written.  Sparse value ranges keep the per-value ingest."""
import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu


def clades(n, median, bits, seed=synth.SEED_BASE + 40):
    """The clade recipe of the default workload over [0, 2^bits)."""
    return synth.generate("clade", n=n, id_bits=bits, seed=seed, n_clades=max(1, n // 32), core=0.3, u_max=0.4,
                          median=median, sigma=synth.SIGMA_DECADE, lo=median / 10, hi=median * 10)


def check(off, ids, C, s, J, count_bits=32, distance=False):
    Co, so, Jo = oracle.all_pairs(off, ids)
    np.testing.assert_array_equal(s, so)
    np.testing.assert_array_equal(C, Co.astype(np.uint64 if count_bits == 64 else np.uint32))
    if distance:
        Jo = oracle.distance_matrix(Co, so, so)
    np.testing.assert_array_equal(J.view(np.uint64), Jo.view(np.uint64))


def run(off, ids, **kw):
    with jsim.Context(variant="sparse", **kw) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        st = ctx.stats()
    assert st["variant"] == "sparse"
    return C, s, J, st


def collection(segs):
    off = np.zeros(len(segs) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([x.size for x in segs])
    ids = np.concatenate(segs).astype(np.uint64) if segs else np.zeros(0, dtype=np.uint64)
    return off, ids


@pytest.mark.parametrize("n,median,bits", [(300, 4e3, 22), (257, 2e3, 20), (130, 8e3, 24), (64, 1e4, 20),
                                           (1000, 1.5e3, 22)])
def test_windowed_matches_oracle(gpu, n, median, bits):
    off, ids = clades(n, median, bits)
    C, s, J, st = run(off, ids, id_bits=bits)
    assert st["windows"] > 0, "the windowed ingest did not run"
    check(off, ids, C, s, J)


@pytest.mark.parametrize("filter_min,count_bits,distance", [(2, 32, False), (1, 64, False), (2, 64, True),
                                                           (1, 32, True)])
def test_windowed_filters_widths_distance(gpu, filter_min, count_bits, distance):
    off, ids = clades(400, 3e3, 22)
    C, s, J, st = run(off, ids, id_bits=22, filter_min=filter_min, count_bits=count_bits, distance=distance)
    assert st["windows"] > 0
    check(off, ids, C, s, J, count_bits, distance)


@pytest.mark.timeout(600)
@pytest.mark.parametrize("filter_min", [1, 2])
def test_windowed_ranges_of_several_windows(gpu, filter_min):
    # batches of 2^27 rows: 2048 windows, more than the pass-1 CTAs resident
    # at once, so every CTA walks a range of several windows (and there are
    # more ranges than resident CTAs)
    off, ids = clades(300, 3e4, 27)
    C, s, J, st = run(off, ids, id_bits=27, batch_rows=1 << 27, filter_min=filter_min)
    assert st["windows"] >= 2048
    check(off, ids, C, s, J)
    with jsim.Context(variant="tc2", id_bits=27, filter_min=filter_min) as ctx:
        C2, s2, J2 = ctx.all_pairs(off, ids)
    np.testing.assert_array_equal(C, C2)
    np.testing.assert_array_equal(J.view(np.uint64), J2.view(np.uint64))


def test_windowed_narrow_batches_and_device_buffers(gpu):
    import torch
    off, ids = clades(520, 2e3, 22)
    d_off = torch.from_numpy(off.view(np.int64)).cuda()
    d_ids = torch.from_numpy(ids.view(np.int64)).cuda()
    for batch_rows in (1 << 18, 1 << 20, 0):
        with jsim.Context(variant="sparse", id_bits=22, batch_rows=batch_rows) as ctx:
            C, s, J = ctx.all_pairs(d_off, d_ids)
            st = ctx.stats()
            torch.cuda.synchronize()
        assert st["windows"] > 0
        if batch_rows:
            assert st["batch_rows"] == batch_rows
        check(off, ids, C.view(torch.int32).cpu().numpy().view(np.uint32),
              s.view(torch.int64).cpu().numpy().view(np.uint64), J.cpu().numpy())


@pytest.mark.parametrize("filter_min", [1, 2])
def test_windowed_edge_cases(gpu, filter_min):
    rng = np.random.default_rng(41)
    cases = []
    # one dense sample; a few samples (one tile); every value in one window
    cases.append([np.arange(10, 200000, 3, dtype=np.uint64)])
    cases.append([np.unique(rng.integers(0, 1 << 16, 9000)).astype(np.uint64) for _ in range(7)])
    # empty samples among others, a ragged last tile
    segs = [np.unique(rng.integers(0, 1 << 20, 3000)).astype(np.uint64) for _ in range(200)]
    for k in (0, 17, 133, 199):
        segs[k] = np.zeros(0, dtype=np.uint64)
    cases.append(segs)
    # identical samples over two tiles, and one other
    base = np.unique(rng.integers(0, 1 << 20, 6000)).astype(np.uint64)
    cases.append([base.copy() for _ in range(140)] + [np.unique(rng.integers(0, 1 << 20, 500)).astype(np.uint64)])
    # repeated values inside samples (one set element each), at window edges too
    segs = []
    for k in range(150):
        v = np.unique(rng.integers(0, 1 << 20, 4000)).astype(np.uint64)
        v = np.concatenate([v, np.arange(k % 3, 1 << 20, 1 << 16, dtype=np.uint64)])
        v.sort()
        segs.append(np.repeat(v, rng.integers(1, 4, v.size)))
    cases.append(segs)
    # values up to the top of the id range
    top = [np.unique(rng.integers((1 << 22) - (1 << 17), 1 << 22, 5000)).astype(np.uint64) for _ in range(130)]
    cases.append(top)
    for segs in cases:
        off, ids = collection(segs)
        C, s, J, st = run(off, ids, id_bits=22, filter_min=filter_min)
        assert st["windows"] > 0
        check(off, ids, C, s, J)


def test_windowed_sixteen_tiles(gpu):
    off, ids = clades(2048, 500, 20)
    for filter_min in (1, 2):
        C, s, J, st = run(off, ids, id_bits=20, filter_min=filter_min)
        assert st["windows"] > 0
        check(off, ids, C, s, J)


def test_sparse_value_ranges_keep_the_per_value_ingest(gpu):
    off, ids = synth.clade1024(n=300, median=3e3)
    C, s, J, st = run(off, ids, id_bits=32)
    assert st["windows"] == 0
    check(off, ids, C, s, J)


def test_windowed_input_errors(gpu):
    off, ids = clades(300, 4e3, 22)
    i = 257
    a, b = int(off[i]), int(off[i + 1])
    bad_sorted = ids.copy()
    bad_sorted[a + 5], bad_sorted[b - 3] = bad_sorted[b - 3], bad_sorted[a + 5]
    bad_range = ids.copy()
    bad_range[(a + b) // 2:b] = np.arange(b - (a + b) // 2, dtype=np.uint64) + (1 << 23)
    n = len(off) - 1
    for bad, name in ((bad_sorted, "JSIM_ERR_UNSORTED"), (bad_range, "JSIM_ERR_ID_RANGE")):
        outs = (np.full((n, n), 7, dtype=np.uint32), np.full(n, 7, dtype=np.uint64), np.full((n, n), -1.0))
        with jsim.Context(variant="sparse", id_bits=22) as ctx:
            with pytest.raises(jsim.JsimError) as e:
                ctx.all_pairs(off, bad, out=outs)
            assert e.value.name == name
            C, s, J = ctx.all_pairs(off, ids)
            assert ctx.stats()["windows"] > 0
        assert (outs[0] == 7).all() and (outs[1] == 7).all() and (outs[2] == -1.0).all()
        check(off, ids, C, s, J)
