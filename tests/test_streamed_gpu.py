"""GPU parity of the streamed all-pairs call (host input copied to the device
in super-batches through pinned double-buffered staging) against the oracle
and against the one-shot call.  All results are integers or correctly
rounded binary64 quotients of integers, so the tolerance is zero."""
import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu

MIB = 1 << 20


def collection(segs):
    offsets = np.zeros(len(segs) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([len(s) for s in segs])
    ids = np.concatenate([np.asarray(s, dtype=np.uint64) for s in segs]) if segs else np.zeros(0, np.uint64)
    return offsets, ids.astype(np.uint64)


def assert_same(res, ref):
    C, sizes, J = res
    Co, so, Jo = ref
    np.testing.assert_array_equal(np.asarray(sizes, dtype=np.uint64), so)
    np.testing.assert_array_equal(np.asarray(C).astype(np.uint64), Co)
    np.testing.assert_array_equal(np.asarray(J).view(np.uint64), Jo.view(np.uint64))


@pytest.fixture(scope="module")
def c1():
    return synth.ancestral64()


@pytest.fixture(scope="module")
def c1_ref(c1):
    return oracle.all_pairs(*c1)


@pytest.mark.parametrize("batch_rows,staging", [(1 << 14, MIB), (3 << 12, MIB), (1 << 16, 4 * MIB), (0, 64 * MIB)])
@pytest.mark.parametrize("variant", ["auto", "popc", "tc", "tc2"])
def test_ancestral64_streamed(gpu, c1, c1_ref, batch_rows, staging, variant):
    """Several super-batches (1 MiB staging = 131,072 values of 3.1e6), each
    several row batches with a ragged last one, give the oracle's results."""
    with jsim.Context(batch_rows=batch_rows, variant=variant) as ctx:
        assert_same(ctx.all_pairs_streamed(*c1, staging_bytes=staging), c1_ref)
        st = ctx.stats()
        if batch_rows:
            assert st["batch_rows"] == batch_rows
        # a second call on the same context reuses its pinned staging
        assert_same(ctx.all_pairs_streamed(*c1, staging_bytes=staging), c1_ref)


def test_ancestral64_streamed_device_out(gpu, c1, c1_ref):
    import torch
    with jsim.Context(batch_rows=1 << 15) as ctx:
        C, s, J = ctx.all_pairs_streamed(*c1, staging_bytes=2 * MIB, out_device=True)
        torch.cuda.synchronize()
        C = C.view(torch.int32).cpu().numpy().view(np.uint32)
        s = s.view(torch.int64).cpu().numpy().view(np.uint64)
        assert_same((C, s, J.cpu().numpy()), c1_ref)


@pytest.mark.parametrize("n,median", [(130, 3e4), (257, 1e4)])
def test_clade40_streamed_matches_oracle_and_one_shot(gpu, n, median):
    """The 4096-sample 40-bit clade recipe at sizes the oracle finishes in
    seconds, 64-bit counts, streamed through 4 MiB staging."""
    off, ids = synth.clade4096(n=n, median=median)
    ref = oracle.all_pairs(off, ids)
    with jsim.Context(count_bits=64, id_bits=40) as ctx:
        assert_same(ctx.all_pairs_streamed(off, ids, staging_bytes=4 * MIB), ref)
        st = ctx.stats()
        assert st["batches"] > 1
        assert_same(ctx.all_pairs(off, ids), ref)


def test_streamed_edge_cases(gpu):
    segs = [[], [], [0], [0, 2**64 - 1], [5, 5, 5, 7], list(range(1000, 1300)), [2**63, 2**63 + 1],
            [2**64 - 1], [2**40 + k * 977 for k in range(3000)]]
    off, ids = collection(segs)
    ref = oracle.all_pairs(off, ids)
    for batch_rows in (0, 64, 1 << 20):
        with jsim.Context(batch_rows=batch_rows) as ctx:
            assert_same(ctx.all_pairs_streamed(off, ids, staging_bytes=MIB), ref)
    with jsim.Context() as ctx:
        C, s, J = ctx.all_pairs_streamed(*collection([[], [], []]), staging_bytes=MIB)
        assert np.all(C == 0) and np.all(s == 0) and np.all(J == 1.0)
        C, s, J = ctx.all_pairs_streamed(np.zeros(1, np.uint64), np.zeros(0, np.uint64))
        assert C.shape == (0, 0)


def test_streamed_errors(gpu):
    import torch
    with jsim.Context(batch_rows=64) as ctx:
        # a descent inside one slice (seen on the device)
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*collection([[1, 2, 3], [5, 3, 9]]), staging_bytes=MIB)
        assert e.value.name == "JSIM_ERR_UNSORTED"
        # a descent between slices (seen on the host)
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*collection([[1, 2, 10**6], [100, 5 * 10**6, 200]]), staging_bytes=MIB)
        assert e.value.name == "JSIM_ERR_UNSORTED"
        # first value above the last
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*collection([[1, 2], [9, 3]]), staging_bytes=MIB)
        assert e.value.name == "JSIM_ERR_UNSORTED"
        # staging below 1 MiB
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*collection([[1, 2]]), staging_bytes=1000)
        assert e.value.name == "JSIM_ERR_ARG"
        # device input is not streamed
        off, ids = collection([[1, 2]])
        with pytest.raises(ValueError):
            ctx.all_pairs_streamed(torch.from_numpy(off.view(np.int64)).cuda(),
                                   torch.from_numpy(ids.view(np.int64)).cuda())
        # still usable after errors
        C, s, J = ctx.all_pairs_streamed(*collection([[1, 2], [2, 3]]), staging_bytes=MIB)
        assert C[0, 1] == 1 and J[0, 1] == 1 / 3
    # one row batch with more values than the staging holds
    with jsim.Context(batch_rows=1 << 20) as ctx:
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*collection([list(range(200_000))]), staging_bytes=MIB)
        assert e.value.name == "JSIM_ERR_OOM"
    with jsim.Context(id_bits=20) as ctx:
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*collection([[1, 2**20], [4]]), staging_bytes=MIB)
        assert e.value.name == "JSIM_ERR_ID_RANGE"


def test_streamed_two_or_more_filter(gpu, c1, c1_ref):
    with jsim.Context(batch_rows=1 << 14, filter_min=2) as ctx:
        assert_same(ctx.all_pairs_streamed(*c1, staging_bytes=MIB), c1_ref)


def run_to_end(ctx, c, path, staging, every=0, step=0, out_device=False):
    """Resume a checkpointed streamed call `step` super-batches at a time
    until it completes; returns the result and the number of calls."""
    calls = 0
    while True:
        calls += 1
        try:
            return ctx.all_pairs_streamed(*c, staging_bytes=staging, out_device=out_device,
                                          checkpoint={"path": path, "every": every, "max_supers": step,
                                                      "resume": True}), calls
        except jsim.JsimError as e:
            if e.name != "JSIM_ERR_INCOMPLETE":
                raise
            assert calls < 1000


@pytest.mark.parametrize("filter_min,count_bits", [(1, 32), (2, 64)])
def test_checkpoint_resume_matches_one_call(gpu, c1, c1_ref, tmp_path, filter_min, count_bits):
    """A streamed call stopped after every 3 super-batches and resumed from its
    file gives the one-call result bit for bit (and the same statistics)."""
    path = str(tmp_path / "ck.bin")
    with jsim.Context(batch_rows=1 << 14, filter_min=filter_min, count_bits=count_bits) as ctx:
        one = ctx.all_pairs_streamed(*c1, staging_bytes=MIB)
        st_one = ctx.stats()
        assert st_one["batches"] > 6
        res, calls = run_to_end(ctx, c1, path, MIB, every=2, step=3)
        assert calls > 2
        assert_same(res, c1_ref)
        assert_same(res, (one[0].astype(np.uint64), one[1], one[2]))
        st = ctx.stats()
        for k in ("rows_nonzero", "words", "batches"):
            assert st[k] == st_one[k]
        # the file keeps the last checkpoint before the end: resuming it again
        # redoes only the super-batches after it
        again = ctx.all_pairs_streamed(*c1, staging_bytes=MIB, checkpoint={"path": path, "resume": True})
        assert_same(again, c1_ref)
        assert 0 < ctx.stats()["product_launches"] < st_one["product_launches"]


def test_checkpoint_mismatch_corruption_and_errors(gpu, c1, c1_ref, tmp_path):
    path = str(tmp_path / "ck.bin")
    with jsim.Context(batch_rows=1 << 14) as ctx:
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*c1, staging_bytes=MIB, checkpoint={"path": path, "max_supers": 2})
        assert e.value.name == "JSIM_ERR_INCOMPLETE"
        good = open(path, "rb").read()
        # another staging size is another call
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*c1, staging_bytes=2 * MIB, checkpoint={"path": path, "resume": True})
        assert e.value.name == "JSIM_ERR_CHECKPOINT"
        # another collection is another call
        other = synth.ancestral64(seed=synth.SEED_BASE + 77)
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*other, staging_bytes=MIB, checkpoint={"path": path, "resume": True})
        assert e.value.name == "JSIM_ERR_CHECKPOINT"
        # a flipped byte in C fails the checksum; a truncated file is refused
        bad = bytearray(good)
        bad[len(bad) // 2] ^= 0x40
        open(path, "wb").write(bytes(bad))
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*c1, staging_bytes=MIB, checkpoint={"path": path, "resume": True})
        assert e.value.name == "JSIM_ERR_CHECKPOINT"
        open(path, "wb").write(good[:-9])
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*c1, staging_bytes=MIB, checkpoint={"path": path, "resume": True})
        assert e.value.name == "JSIM_ERR_CHECKPOINT"
        # the intact file still resumes to the right answer
        open(path, "wb").write(good)
        res, _ = run_to_end(ctx, c1, path, MIB, step=0)
        assert_same(res, c1_ref)
        # a missing file with resume starts from the beginning
        res = ctx.all_pairs_streamed(*c1, staging_bytes=MIB,
                                     checkpoint={"path": str(tmp_path / "none.bin"), "resume": True})
        assert_same(res, c1_ref)
        # stopping without a file would lose the progress
        with pytest.raises(jsim.JsimError) as e:
            ctx.all_pairs_streamed(*c1, staging_bytes=MIB, checkpoint={"path": None, "max_supers": 1})
        assert e.value.name == "JSIM_ERR_CHECKPOINT"
        # an input error is reported by the resumed call that reaches it
        bad_c = collection([[1, 2, 3], list(range(10, 300000, 3)), [5, 3, 9]])
        with pytest.raises(jsim.JsimError) as e:
            run_to_end(ctx, bad_c, str(tmp_path / "bad.bin"), MIB, step=1)
        assert e.value.name == "JSIM_ERR_UNSORTED"


def test_streamed_page_locked_input_copies_slices_directly(gpu, c1, c1_ref):
    """Page-locked input takes the direct path (one copy per sample slice, no
    host gather); results are the oracle's, with several super-batches."""
    import torch
    off, ids = c1
    pin = torch.empty(len(ids), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    pin[:] = ids
    poff = torch.empty(len(off), dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    poff[:] = off
    for batch_rows, staging in ((1 << 14, MIB), (0, 64 * MIB)):
        with jsim.Context(batch_rows=batch_rows) as ctx:
            assert_same(ctx.all_pairs_streamed(poff, pin, staging_bytes=staging), c1_ref)
    with jsim.Context(batch_rows=1 << 14, filter_min=2) as ctx:
        assert_same(ctx.all_pairs_streamed(poff, pin, staging_bytes=MIB), c1_ref)
