"""The CUDA path on the paper's own synthetic inputs (Sec. V-A): m x n
indicator matrices whose every entry is present independently with
probability p.  C, sizes and J bit for bit against the oracle's pairwise
merge, for each product variant, both filters, host and device input, and
several row-batch sizes (so the batch loop, the zero-row filter and ragged
last words and tiles are all exercised at both a sparse and a dense
density)."""
import numpy as np
import pytest

import oracle
from paper_1911_04200_gb300 import jsim, synth

pytestmark = pytest.mark.gpu

CASES = {}


def case(n, m, p):
    key = (n, m, p)
    if key not in CASES:
        off, ids = synth.bernoulli(n, m, p)
        CASES[key] = (off, ids, oracle.all_pairs(off, ids))
    return CASES[key]


@pytest.mark.timeout(600)
@pytest.mark.parametrize("n,m,p", [(64, 1 << 22, 1e-3), (64, 1 << 22, 0.05), (200, 1 << 22, 1e-3),
                                   (200, 1 << 21, 0.05)])
@pytest.mark.parametrize("variant", ["auto", "popc", "tc", "tc2"])
def test_bernoulli_matches_oracle(gpu, n, m, p, variant):
    off, ids, (Cr, sr, Jr) = case(n, m, p)
    with jsim.Context(variant=variant, id_bits=22) as ctx:
        C, s, J = ctx.all_pairs(off, ids)
    np.testing.assert_array_equal(C, Cr.astype(np.uint32))
    np.testing.assert_array_equal(s, sr)
    np.testing.assert_array_equal(J.view(np.uint64), Jr.view(np.uint64))


@pytest.mark.timeout(600)
@pytest.mark.parametrize("batch_rows", [1 << 16, 1 << 19, 0])
@pytest.mark.parametrize("filter_min", [1, 2])
def test_bernoulli_batches_filters_device_input(gpu, batch_rows, filter_min):
    import torch
    off, ids, (Cr, sr, Jr) = case(200, 1 << 21, 0.05)
    with jsim.Context(batch_rows=batch_rows, filter_min=filter_min) as ctx:
        C, s, J = ctx.all_pairs(torch.from_numpy(off.view(np.int64)).cuda(),
                                torch.from_numpy(ids.view(np.int64)).cuda())
        torch.cuda.synchronize()
        C = C.view(torch.int32).cpu().numpy().view(np.uint32)
        s = s.view(torch.int64).cpu().numpy().view(np.uint64)
        J = J.cpu().numpy()
    np.testing.assert_array_equal(C, Cr.astype(np.uint32))
    np.testing.assert_array_equal(s, sr)
    np.testing.assert_array_equal(J.view(np.uint64), Jr.view(np.uint64))
