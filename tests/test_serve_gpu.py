"""GPU parity of the serving pattern: a resident reference index, query
requests under continuous batching, against the oracle's query x reference
merge.  Counts and sizes are integers and J their correctly rounded binary64
quotient, so every comparison is exact; a request's results must be the
same alone and in a mix of concurrent requests."""
import threading

import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu

N_REF = 96
MEDIAN = 2e4


def collection(segs):
    offsets = np.zeros(len(segs) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([len(s) for s in segs])
    ids = np.concatenate([np.asarray(s, dtype=np.uint64) for s in segs]) if segs else np.zeros(0, np.uint64)
    return offsets, ids.astype(np.uint64)


def sub(off, ids, a, b):
    """Samples [a, b) of a collection as a collection of its own."""
    o = off[a:b + 1] - off[a]
    return o.astype(np.uint64), ids[int(off[a]):int(off[b])].copy()


def assert_same(res, ref):
    C, s, J = res
    Co, so, Jo = ref
    np.testing.assert_array_equal(s, so)
    np.testing.assert_array_equal(C.astype(np.uint64), Co)
    np.testing.assert_array_equal(J.view(np.uint64), Jo.view(np.uint64))


@pytest.fixture(scope="module")
def ref():
    return synth.serving_reference(n=N_REF, median=MEDIAN)


@pytest.fixture(scope="module")
def queries():
    return synth.serving_queries(0, 48, n_ref=N_REF, median=MEDIAN)


@pytest.mark.parametrize("count_bits,slots,max_samples", [(32, 2, 64), (64, 1, 64), (32, 3, 8)])
def test_requests_match_oracle(gpu, ref, queries, count_bits, slots, max_samples):
    qoff, qids = queries
    with jsim.Context(count_bits=count_bits, id_bits=32) as ctx:
        with jsim.Index(ctx, *ref, max_batch_samples=max_samples, slots=slots) as ix:
            np.testing.assert_array_equal(ix.ref_sizes(), oracle.sizes_of(*ref))
            # requests of 1..7 samples over the 48 query samples
            bounds = [0, 1, 3, 10, 11, 17, 24, 30, 37, 40, 48]
            reqs = [ix.submit(*sub(qoff, qids, a, b)) for a, b in zip(bounds, bounds[1:])]
            for (a, b), r in zip(zip(bounds, bounds[1:]), reqs):
                assert_same(r.wait(), oracle.cross(*sub(qoff, qids, a, b), *ref))
                qms, tms = r.latency()
                assert 0 <= qms <= tms
            st = ix.stats()
            assert st["requests_done"] == len(reqs) and st["samples_done"] == 48
            assert st["batches"] >= 1 and st["rows_read"] > 0


def test_alone_and_in_the_mix_are_identical(gpu, ref, queries):
    """Continuous batching: the same request alone, then among 40 requests
    submitted concurrently from 4 threads (arriving while batches run)."""
    qoff, qids = queries
    probe = sub(qoff, qids, 5, 12)
    with jsim.Context(id_bits=32) as ctx:
        with jsim.Index(ctx, *ref, max_batch_samples=16, slots=2) as ix:
            alone = ix.submit(*probe).wait()
            assert_same(alone, oracle.cross(*probe, *ref))
            rng = np.random.default_rng(7)
            jobs = []
            for k in range(40):
                a = int(rng.integers(0, 47))
                b = int(rng.integers(a + 1, min(a + 9, 48) + 1))
                jobs.append((a, b))
            jobs[17] = (5, 12)
            results = [None] * len(jobs)

            def client(t):
                mine = [(k, ix.submit(*sub(qoff, qids, *jobs[k]))) for k in range(t, len(jobs), 4)]
                for k, r in mine:
                    results[k] = r.wait()

            th = [threading.Thread(target=client, args=(t,)) for t in range(4)]
            for x in th:
                x.start()
            for x in th:
                x.join()
            mixed = results[17]
            for x, y in zip(alone, mixed):
                np.testing.assert_array_equal(np.asarray(x).view(np.uint8), np.asarray(y).view(np.uint8))
            for (a, b), res in zip(jobs, results):
                assert_same(res, oracle.cross(*sub(qoff, qids, a, b), *ref))
            assert ix.stats()["batches"] < len(jobs) + 1


def test_serve_edge_cases(gpu):
    rsegs = [[], [0], [5, 5, 9], list(range(100, 400, 3)), [2**32 - 1], list(range(1000, 1064))]
    roff, rids = collection(rsegs)
    qsegs = [[], [0, 1, 2], [9], [5, 9, 9, 100, 103, 2**32 - 1], [7, 8], list(range(90, 1100)), [2**40]]
    qoff, qids = collection(qsegs)
    with jsim.Context(id_bits=64) as ctx:
        with jsim.Index(ctx, roff, rids) as ix:
            assert_same(ix.submit(qoff, qids).wait(), oracle.cross(qoff, qids, roff, rids))
            # a request without samples
            C, s, J = ix.submit(np.zeros(1, np.uint64), np.zeros(0, np.uint64)).wait()
            assert C.shape == (0, len(rsegs))
    # a reference whose samples are all empty: every query meets nothing
    with jsim.Context() as ctx:
        eoff, eids = collection([[], []])
        with jsim.Index(ctx, eoff, eids) as ix:
            assert ix.rows == 0
            C, s, J = ix.submit(*collection([[1, 2], []])).wait()
            assert np.all(C == 0) and list(s) == [2, 0]
            assert list(J[0]) == [0.0, 0.0] and list(J[1]) == [1.0, 1.0]


def test_serve_errors(gpu, ref, queries):
    qoff, qids = queries
    with jsim.Context(id_bits=32) as ctx:
        with pytest.raises(jsim.JsimError) as e:
            jsim.Index(ctx, *ref, max_batch_samples=65)
        assert e.value.name == "JSIM_ERR_ARG"
        with pytest.raises(jsim.JsimError) as e:
            jsim.Index(ctx, *collection([[3, 1]]))
        assert e.value.name == "JSIM_ERR_UNSORTED"
        with jsim.Index(ctx, *ref, max_batch_samples=8, max_batch_values=1 << 20) as ix:
            # more samples than a batch holds
            with pytest.raises(jsim.JsimError) as e:
                ix.submit(*sub(qoff, qids, 0, 9))
            assert e.value.name == "JSIM_ERR_ARG"
            # bad requests fail alone; the good ones in the same batches do not
            good1 = ix.submit(*sub(qoff, qids, 0, 2))
            bad_sort = ix.submit(*collection([[1, 5, 3]]))
            bad_range = ix.submit(*collection([[1, 2**32]]))
            good2 = ix.submit(*sub(qoff, qids, 2, 5))
            for r, name in ((bad_sort, "JSIM_ERR_UNSORTED"), (bad_range, "JSIM_ERR_ID_RANGE")):
                with pytest.raises(jsim.JsimError) as e:
                    r.wait()
                assert e.value.name == name
            assert_same(good1.wait(), oracle.cross(*sub(qoff, qids, 0, 2), *ref))
            assert_same(good2.wait(), oracle.cross(*sub(qoff, qids, 2, 5), *ref))


def test_destroy_with_requests_in_flight(gpu, ref, queries):
    """Closing the index finishes running batches and cancels queued requests;
    every request ends either with its exact result or JSIM_ERR_CANCELLED."""
    qoff, qids = queries
    with jsim.Context(id_bits=32) as ctx:
        ix = jsim.Index(ctx, *ref, max_batch_samples=4, slots=1)
        reqs = [(a, ix.submit(*sub(qoff, qids, a, a + 4))) for a in range(0, 44, 4)]
        ix.close()
        done = 0
        for a, r in reqs:
            try:
                res = r.wait()
            except jsim.JsimError as e:
                assert e.name == "JSIM_ERR_CANCELLED"
                continue
            assert_same(res, oracle.cross(*sub(qoff, qids, a, a + 4), *ref))
            done += 1
        for _, r in reqs:
            r.free()
