"""jsim_product_noalloc: the allocation-free product.

It exists for callers that cannot let the library allocate device memory
during a call (a fixed, up-front memory budget for the whole GPU, or a
steady-state loop that must not stall on an allocation).  These tests call
it through the C-ABI and check, on two calls in a row, that its C is
identical to jsim_product's (the tests' tolerance for integer counts is zero)
and that the library's allocator hook is not called while it runs.

This file is named to run last, so a failure here stops a `-x` run only
after every other test has run.
"""
import numpy as np
import pytest

from paper_1911_04200_gb300 import jsim

pytestmark = pytest.mark.gpu


def to_np(t):
    import torch
    m = {torch.uint64: (torch.int64, np.uint64), torch.uint32: (torch.int32, np.uint32)}
    sdt, ndt = m[t.dtype]
    return t.view(sdt).cpu().numpy().view(ndt)


@pytest.mark.parametrize("n,W,density,count_bits,variant", [
    (300, 777, 0.3, 32, "auto"),
    (1024, 2048, 0.05, 32, "tc"),
    (600, 1500, 0.2, 64, "tc2"),
    (700, 500, 0.5, 64, "popc"),
    (130, 64, 1.0, 64, "f8"),
])
def test_noalloc_matches_product_twice(gpu, n, W, density, count_bits, variant):
    import torch
    rng = np.random.default_rng(n + W)
    stride = W + 2
    bits = rng.random((n, stride * 64)) < density
    X = np.packbits(bits, axis=1, bitorder="little").view(np.uint64).copy()
    Xd = torch.from_numpy(X.view(np.int64)).cuda()
    cdt = torch.uint64 if count_bits == 64 else torch.uint32
    with jsim.Context(count_bits=count_bits) as ctx:
        ref = to_np(ctx.product(Xd, n, W, stride, variant=variant))
        torch.cuda.synchronize()
        outs = [torch.empty((n, n), dtype=cdt, device="cuda") for _ in range(2)]
        torch.cuda.synchronize()
        before = torch.cuda.memory_stats()["allocation.all.allocated"]
        for C in outs:  # two calls in a row share the library's scratch
            ctx.product_noalloc(Xd, n, W, stride, C, variant=variant)
        after = torch.cuda.memory_stats()["allocation.all.allocated"]
        torch.cuda.synchronize()
    assert after == before, "the allocation-free product called the allocator"
    for C in outs:
        np.testing.assert_array_equal(to_np(C), ref)


@pytest.mark.parametrize("n,count_bits", [(1024, 32), (724, 64)])
def test_noalloc_largest_sizes_its_scratch_holds(gpu, n, count_bits):
    # n*n counts fill the 4 MiB scratch: 1024^2 x 4 B, 724^2 x 8 B
    import torch
    rng = np.random.default_rng(n)
    W = 96
    X = rng.integers(0, 2**63, size=(n, W), dtype=np.int64)
    X[:, ::3] = 0
    Xd = torch.from_numpy(X).cuda()
    cdt = torch.uint64 if count_bits == 64 else torch.uint32
    with jsim.Context(count_bits=count_bits) as ctx:
        ref = to_np(ctx.product(Xd, n, W, W))
        C = torch.empty((n, n), dtype=cdt, device="cuda")
        ctx.product_noalloc(Xd, n, W, W, C)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(to_np(C), ref)


@pytest.mark.parametrize("n,count_bits", [(725, 64), (1025, 32)])
def test_noalloc_rejects_sizes_beyond_its_scratch(gpu, n, count_bits):
    import torch
    cdt = torch.uint64 if count_bits == 64 else torch.uint32
    with jsim.Context(count_bits=count_bits) as ctx:
        Xd = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
        C = torch.full((n, n), 3, dtype=cdt, device="cuda")
        with pytest.raises(jsim.JsimError) as e:
            ctx.product_noalloc(Xd, n, 4, 4, C)
        assert e.value.name == "JSIM_ERR_ARG"
        torch.cuda.synchronize()
        assert bool((C == 3).all())
