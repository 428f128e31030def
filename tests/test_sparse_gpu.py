"""The block-sparse variant of the all-pairs call (samples ordered by a
sketch of their similarity into tiles of 128; rows held by one tile
multiplied only within that tile's diagonal block).  C, sizes and J bit for
bit against the oracle's merges and against the dense product, on clade
collections (where the ordering pays), Bernoulli matrices (where it does not
and AUTO stays dense), both filters, both count widths, the distance output,
host and device buffers, and the edge cases: one tile, a ragged last tile,
sixteen tiles, empty and identical samples, many narrow batches."""
import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu


def check(off, ids, C, s, J, count_bits=32, distance=False):
    Co, so, Jo = oracle.all_pairs(off, ids)
    np.testing.assert_array_equal(s, so)
    np.testing.assert_array_equal(C, Co.astype(np.uint64 if count_bits == 64 else np.uint32))
    if distance:
        Jo = oracle.distance_matrix(Co, so, so)
    np.testing.assert_array_equal(J.view(np.uint64), Jo.view(np.uint64))


@pytest.mark.parametrize("n,median", [(300, 3e3), (257, 2e3), (130, 4e3)])
def test_sparse_clade_matches_oracle(gpu, n, median):
    off, ids = synth.clade1024(n=n, median=median)
    with jsim.Context(variant="sparse", id_bits=32) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        st = ctx.stats()
    assert st["variant"] == "sparse"
    assert st["bitops_done"] < st["bitops_dense"]
    check(off, ids, C, s, J)


def test_auto_picks_sparse_on_clades_and_equals_dense(gpu):
    off, ids = synth.clade1024(n=1024, median=1e4)
    with jsim.Context(id_bits=32) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        st = ctx.stats()
    assert st["variant"] == "sparse"
    assert st["bitops_done"] * 4 < st["bitops_dense"]
    with jsim.Context(id_bits=32, variant="tc2") as ctx:
        C2, s2, J2 = ctx.all_pairs(off, ids)
    np.testing.assert_array_equal(C, C2)
    np.testing.assert_array_equal(J.view(np.uint64), J2.view(np.uint64))
    check(off, ids, C, s, J)


def test_auto_stays_dense_on_bernoulli_and_sparse_is_exact_there(gpu):
    off, ids = synth.bernoulli(300, 1 << 20, 0.02)
    with jsim.Context(id_bits=20) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        assert ctx.stats()["variant"] != "sparse"
    check(off, ids, C, s, J)
    with jsim.Context(id_bits=20, variant="sparse") as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        assert ctx.stats()["variant"] == "sparse"
    check(off, ids, C, s, J)


@pytest.mark.parametrize("filter_min,count_bits,distance", [(2, 32, False), (1, 64, False), (2, 64, True),
                                                           (1, 32, True)])
def test_sparse_filters_widths_distance(gpu, filter_min, count_bits, distance):
    off, ids = synth.clade1024(n=400, median=3e3)
    with jsim.Context(variant="sparse", id_bits=32, filter_min=filter_min, count_bits=count_bits,
                      distance=distance) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        assert ctx.stats()["variant"] == "sparse"
    check(off, ids, C, s, J, count_bits, distance)


def test_sparse_device_buffers_and_narrow_batches(gpu):
    import torch
    off, ids = synth.clade1024(n=520, median=2e3)
    d_off = torch.from_numpy(off.view(np.int64)).cuda()
    d_ids = torch.from_numpy(ids.view(np.int64)).cuda()
    for batch_rows in (0, 1 << 18, 1 << 24):
        with jsim.Context(variant="sparse", id_bits=32, batch_rows=batch_rows) as ctx:
            C, s, J = ctx.all_pairs(d_off, d_ids)
            st = ctx.stats()
            torch.cuda.synchronize()
        if batch_rows:
            assert st["batch_rows"] == batch_rows
        check(off, ids, C.view(torch.int32).cpu().numpy().view(np.uint32),
              s.view(torch.int64).cpu().numpy().view(np.uint64), J.cpu().numpy())


def test_sparse_edge_cases(gpu):
    rng = np.random.default_rng(4)
    cases = []
    # one sample; a few samples (one tile); empty samples among others; identical samples
    cases.append([np.arange(10, 500, 3, dtype=np.uint64)])
    cases.append([np.unique(rng.integers(0, 5000, 300)).astype(np.uint64) for _ in range(7)])
    segs = [np.unique(rng.integers(0, 1 << 30, 2000)).astype(np.uint64) for _ in range(200)]
    for k in (0, 17, 133, 199):
        segs[k] = np.zeros(0, dtype=np.uint64)
    cases.append(segs)
    base = np.unique(rng.integers(0, 1 << 25, 4000)).astype(np.uint64)
    cases.append([base.copy() for _ in range(140)] + [np.unique(rng.integers(0, 1 << 25, 500)).astype(np.uint64)])
    for segs in cases:
        off = np.zeros(len(segs) + 1, dtype=np.uint64)
        off[1:] = np.cumsum([x.size for x in segs])
        ids = np.concatenate(segs) if segs else np.zeros(0, dtype=np.uint64)
        with jsim.Context(variant="sparse") as ctx:
            C, s, J = ctx.all_pairs(off, ids)
        check(off, ids, C, s, J)


def test_sparse_sixteen_tiles_and_its_limit(gpu):
    off, ids = synth.clade1024(n=2048, median=600)
    with jsim.Context(variant="sparse", id_bits=32) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
    check(off, ids, C, s, J)
    off2, ids2 = synth.clade1024(n=2049, median=50)
    with jsim.Context(variant="sparse", id_bits=32) as ctx:
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs(off2, ids2)
        assert e.value.name == "JSIM_ERR_UNSUPPORTED"


def test_sparse_input_errors_found_beside_the_loop(gpu):
    """On the block-sparse path the input is validated beside the sketch and
    the batch loop: a descent or a value beyond id_bits, in host or device
    input, is reported before any output is written, and the context keeps
    working."""
    import torch
    off, ids = synth.clade1024(n=300, median=3e3)
    n = len(off) - 1
    i = 257
    a, b = int(off[i]), int(off[i + 1])
    bad_sorted = ids.copy()
    bad_sorted[b - 3], bad_sorted[b - 2] = bad_sorted[b - 2], bad_sorted[b - 3]
    bad_range = ids.copy()
    bad_range[(a + b) // 2:b] = np.arange(b - (a + b) // 2, dtype=np.uint64) + (1 << 33)
    for bad, name in ((bad_sorted, "JSIM_ERR_UNSORTED"), (bad_range, "JSIM_ERR_ID_RANGE")):
        for dev in (False, True):
            with jsim.Context(variant="sparse", id_bits=32) as ctx:
                if dev:
                    d_off = torch.from_numpy(off.view(np.int64)).cuda()
                    d_ids = torch.from_numpy(bad.view(np.int64)).cuda()
                    C = torch.full((n, n), 7, dtype=torch.int32, device="cuda")
                    S = torch.full((n,), 7, dtype=torch.int64, device="cuda")
                    J = torch.full((n, n), -1.0, dtype=torch.float64, device="cuda")
                    with pytest.raises(jsim.JsimError) as e:
                        ctx.all_pairs(d_off, d_ids, out=(C.view(torch.uint32), S.view(torch.uint64), J))
                    torch.cuda.synchronize()
                    assert bool((C == 7).all()) and bool((S == 7).all()) and bool((J == -1.0).all())
                else:
                    outs = (np.full((n, n), 7, dtype=np.uint32), np.full(n, 7, dtype=np.uint64),
                            np.full((n, n), -1.0))
                    with pytest.raises(jsim.JsimError) as e:
                        ctx.all_pairs(off, bad, out=outs)
                    assert (outs[0] == 7).all() and (outs[1] == 7).all() and (outs[2] == -1.0).all()
                assert e.value.name == name
                Cg, sg, Jg = ctx.all_pairs(off, ids)
            check(off, ids, Cg, sg, Jg)
