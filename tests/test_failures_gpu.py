"""Failure detection without a GPU fault.

* Bounded device waits: every wait inside the tensor-core products has a
  clock budget (the context's timeout_ms).  A product whose accumulator
  segments take tens of milliseconds, run with a 1 ms budget, makes the
  epilogue's first wait run out: the kernel raises its error word, drains its
  own work, frees its tensor memory and returns; the call reports
  JSIM_ERR_TIMEOUT, writes no output, and the context (and the device) keep
  working.
* Allocation failures: an allocator hook that refuses the k-th request, for
  every k a call makes, on the plain, streamed, batched and index-build
  paths: the call returns JSIM_ERR_OOM, writes no output, and every device
  block it got is returned (none live after the context is destroyed).
"""
import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu


def to_np(t):
    import torch
    m = {torch.uint64: (torch.int64, np.uint64), torch.uint32: (torch.int32, np.uint32)}
    sdt, ndt = m[t.dtype]
    return t.view(sdt).cpu().numpy().view(ndt)


@pytest.mark.timeout(600)
@pytest.mark.parametrize("variant", ["tc", "tc2"])
def test_bounded_wait_runs_out_and_the_context_stays_usable(gpu, variant):
    import torch
    n, W = 1024, 1 << 19              # 4 GiB of packed words: segments of ~16k stages, tens of ms each
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randint(-(2**62), 2**62, (n, W), dtype=torch.int64, device="cuda", generator=g)
    sentinel = 0x5A5A5A5A
    C = torch.full((n, n), sentinel, dtype=torch.int32, device="cuda").view(torch.uint32)
    with jsim.Context(timeout_ms=1) as ctx:
        with pytest.raises(jsim.JsimError) as e:
            ctx.product(X, n, W, W, C, variant=variant)
        assert e.value.name == "JSIM_ERR_TIMEOUT"
        torch.cuda.synchronize()
        assert bool((C.view(torch.int32) == sentinel).all()), "an output was written after a timed-out wait"
        # the same context, a product small enough for the 1 ms budget
        n2, W2 = 300, 200
        Xs = X[:n2, :W2].contiguous()
        got = to_np(ctx.product(Xs, n2, W2, W2, variant=variant))
    del X
    with jsim.Context() as ctx2:
        ref = to_np(ctx2.product(Xs, n2, W2, W2, variant="popc"))
    np.testing.assert_array_equal(got, ref)


class FailAt:
    """Device allocator (PyTorch's caching allocator underneath) that refuses
    its k-th request (k >= 1; 0: never) and tracks what is live."""

    def __init__(self, k=0):
        import torch
        self.torch = torch
        self.k = k
        self.calls = 0
        self.live = {}

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.calls == self.k:
            return 0
        p = self.torch.cuda.caching_allocator_alloc(nbytes, 0, stream)
        self.live[p] = nbytes
        return p

    def free(self, ptr, nbytes, stream):
        assert ptr in self.live, "freed a block it did not get"
        del self.live[ptr]
        self.torch.cuda.caching_allocator_delete(ptr)


def run_with_failures(call, check_ok, **ctx_kw):
    """call(ctx) once with no failure (counting the requests), then once per
    request k with the k-th refused: OOM and outputs untouched, or success;
    no block live after the context is gone."""
    base = FailAt(0)
    with jsim.Context(allocator=base, **ctx_kw) as ctx:
        check_ok(call(ctx))
    assert not base.live
    total = base.calls
    assert total >= 2
    seen_oom = 0
    for k in range(1, total + 1):
        a = FailAt(k)
        try:
            ctx = jsim.Context(allocator=a, **ctx_kw)
        except jsim.JsimError as e:
            assert k == 1 and e.name == "JSIM_ERR_OOM"   # the context's own error word
            assert not a.live
            seen_oom += 1
            continue
        try:
            with pytest.raises(jsim.JsimError) as e:
                call(ctx)
            assert e.value.name == "JSIM_ERR_OOM", e.value
            seen_oom += 1
        finally:
            ctx.close()
        assert not a.live, "blocks still live after an allocation failure at request %d" % k
    assert seen_oom == total


def test_allocation_failures_plain_call(gpu):
    off, ids = synth.ancestral64(n=24, anc_size=4000)
    Cr, sr, Jr = oracle.all_pairs(off, ids)
    outs = []

    def call(ctx):
        C = np.full((24, 24), 7, dtype=np.uint32)
        s = np.full(24, 7, dtype=np.uint64)
        J = np.full((24, 24), -1.0)
        outs.append((C, s, J))
        return ctx.all_pairs(off, ids, out=(C, s, J))

    def ok(res):
        C, s, J = res
        np.testing.assert_array_equal(C, Cr)
        np.testing.assert_array_equal(J.view(np.uint64), Jr.view(np.uint64))

    run_with_failures(call, ok)
    for C, s, J in outs[1:]:
        assert (C == 7).all() and (s == 7).all() and (J == -1.0).all()


def test_allocation_failures_streamed_call(gpu):
    off, ids = synth.clade1024(n=40, median=3e4)
    Cr, sr, Jr = oracle.all_pairs(off, ids)
    outs = []

    def call(ctx):
        C = np.full((40, 40), 7, dtype=np.uint32)
        s = np.full(40, 7, dtype=np.uint64)
        J = np.full((40, 40), -1.0)
        outs.append((C, s, J))
        return ctx.all_pairs_streamed(off, ids, staging_bytes=1 << 20, out=(C, s, J))

    def ok(res):
        C, s, J = res
        np.testing.assert_array_equal(C, Cr)
        np.testing.assert_array_equal(J.view(np.uint64), Jr.view(np.uint64))

    run_with_failures(call, ok, batch_rows=1 << 24)
    for C, s, J in outs[1:]:
        assert (C == 7).all() and (s == 7).all() and (J == -1.0).all()


def test_allocation_failures_batched_call(gpu):
    cols = synth.batched_collections(count=3, n_lo=5, n_hi=40, median=2e3)
    refs = [oracle.all_pairs(o, i) for o, i in cols]

    def call(ctx):
        return ctx.all_pairs_batched(cols)

    def ok(res):
        for (C, s, J), (Cr, sr, Jr) in zip(res, refs):
            np.testing.assert_array_equal(C, Cr)
            np.testing.assert_array_equal(J.view(np.uint64), Jr.view(np.uint64))

    run_with_failures(call, ok)


def test_allocation_failures_index_build(gpu):
    roff, rids = synth.serving_reference(n=70, median=2e3)
    qoff, qids = synth.serving_queries(0, 3, n_ref=70, median=2e3)
    Cr, qsr, Jr = oracle.cross(qoff, qids, roff, rids)

    def call(ctx):
        with jsim.Index(ctx, roff, rids, max_batch_samples=8, max_batch_values=1 << 16, slots=2) as ix:
            r = ix.submit(qoff, qids)
            res = r.wait()
            r.free()
            return res

    def ok(res):
        C, qs, J = res
        np.testing.assert_array_equal(C, Cr)
        np.testing.assert_array_equal(J.view(np.uint64), Jr.view(np.uint64))

    run_with_failures(call, ok)
