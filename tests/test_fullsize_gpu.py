"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times, on outputs the oracle can compute one by one: sampled pairs
(merge counts and binary64 J), every size, and the invariants that hold at
any size (symmetry, C_ii = |X_i|, C_ij <= min, J_ii = 1, 0 <= J <= 1).
Integers and correctly rounded quotients: tolerance zero."""
import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu


def check_sampled(off, ids, C, sizes, J, pairs=384, seed=5):
    n = len(off) - 1
    np.testing.assert_array_equal(sizes, oracle.sizes_of(off, ids))
    C = C.astype(np.uint64)
    # invariants over the whole matrix
    np.testing.assert_array_equal(C, C.T)
    np.testing.assert_array_equal(J.view(np.uint64), J.T.view(np.uint64))
    np.testing.assert_array_equal(np.diag(C), sizes)
    assert np.all(C <= np.minimum(sizes[:, None], sizes[None, :]))
    assert np.all((J >= 0.0) & (J <= 1.0))
    assert np.all(np.diag(J) == 1.0)
    # sampled pairs against the plain merge
    rng = np.random.default_rng(seed)
    pi = rng.integers(0, n, pairs).astype(np.uint64)
    pj = rng.integers(0, n, pairs).astype(np.uint64)
    Co, Jo = oracle.pairs(off, ids, pi, pj)
    np.testing.assert_array_equal(C[pi, pj], Co)
    np.testing.assert_array_equal(J[pi, pj].view(np.uint64), Jo.view(np.uint64))


@pytest.fixture(scope="module")
def clade1024():
    return synth.clade1024()


@pytest.mark.timeout(900)
def test_clade1024_full_size(gpu, clade1024):
    """The benchmark's workload (1024 samples, 1.3e9 values) with the automatic
    product (SM pairs) and with the two-or-more filter: sampled parity, and the
    two runs byte-identical."""
    off, ids = clade1024
    with jsim.Context(id_bits=32) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
        assert ctx.stats()["variant"] == "tc2"
    check_sampled(off, ids, C, s, J)
    with jsim.Context(id_bits=32, filter_min=2) as ctx:
        C2, s2, J2 = ctx.all_pairs(off, ids)
    np.testing.assert_array_equal(C2, C)
    np.testing.assert_array_equal(s2, s)
    np.testing.assert_array_equal(J2.view(np.uint64), J.view(np.uint64))


@pytest.mark.timeout(900)
def test_batched_recipe_full_size_subset(gpu):
    """The first 12 collections of the 200-collection recipe at full size
    (n ~ U{8..512}, sizes log-normal median 2e5 in [1e4, 5e6]) through one
    batched call."""
    cols = synth.batched_collections(count=12)
    with jsim.Context(id_bits=32) as ctx:
        outs = ctx.all_pairs_batched(cols)
    for (off, ids), (C, s, J) in zip(cols, outs):
        check_sampled(off, ids, C, s, J, pairs=128)
