"""The work schedule of the job-table tensor-core product (the persistent
launch behind jsim_all_pairs_batched), checked on the host with the same
schedule functions the kernel runs (jsim_check_tc_schedule): every load
inside its packed matrix (also for matrices of exactly n rows and ragged last
tiles and stages), 16-byte loads aligned, every (collection, tile, stage)
unit taken by exactly one CTA, every pair i <= j in exactly one tile, no
accumulator beyond the exact-count cap, every accumulator drained as often
as committed.  No GPU: nothing here launches a kernel."""
import numpy as np
import pytest

from paper_1911_04200_gb300 import jsim


def stride_of(W):
    return max(64, -(-W // 64) * 64)


@pytest.mark.parametrize("tile_n", [256, 128])
@pytest.mark.parametrize("n", [1, 2, 127, 128, 129, 255, 256, 257, 300, 1024])
@pytest.mark.parametrize("W", [1, 2, 3, 4, 5, 7, 1023])
@pytest.mark.parametrize("grid", [1, 7, 148, 152])
def test_single_collection_exact_rows(n, W, grid, tile_n):
    """One collection whose matrix has exactly n rows (as jsim_product
    allows): the shapes of the plain path, for both tile widths."""
    rc, msg = jsim.check_tc_schedule([(n, W, stride_of(W), n)], grid, tile_n)
    assert rc == 0, msg


@pytest.mark.parametrize("tile_n", [256, 128])
def test_plain_path_shapes(tile_n):
    """The shapes of the default workload's batches (1024 samples, a few
    thousand to 3.5e5 words per batch) and odd row strides."""
    for n, W, stride in [(1024, 5000, 5120), (1024, 351826, 352256), (1000, 65536, 66560), (4096, 2700, 2752)]:
        rc, msg = jsim.check_tc_schedule([(n, W, stride, n)], 152, tile_n)
        assert rc == 0, msg


@pytest.mark.parametrize("stage_bits", [256, 512])
def test_block_sparse_tile_jobs(stage_bits):
    """The block-sparse path's per-tile products: up to 16 jobs of one
    diagonal 128 x 128 tile each (the last one ragged), deep word counts,
    rows taken from one shared matrix; the diagonal-only launch's 512-bit
    stages too (segments cut at 8192 stages)."""
    rng = np.random.default_rng(1)
    for trial in range(12):
        T = int(rng.integers(1, 17))
        jobs = []
        for t in range(T):
            W = int(rng.integers(1, 700000))
            m = 128 if t < T - 1 else int(rng.integers(1, 129))
            jobs.append((m, W, -(-W // 1024) * 1024 + 1024, m))
        for grid in (152, 37, 1):
            rc, msg = jsim.check_tc_schedule(jobs, grid, 128, stage_bits)
            assert rc == 0, msg


def test_512_bit_stages_only_for_128_wide_tiles():
    rc, _ = jsim.check_tc_schedule([(128, 100, 128, 128)], 4, 256, 512)
    assert jsim.ERRORS.get(rc) == "JSIM_ERR_ARG"
    for W in (1, 7, 8, 9, 8191 * 8, 8192 * 8 + 3, 3 * 8192 * 8):
        rc, msg = jsim.check_tc_schedule([(100, W, -(-W // 64) * 64, 128)], 3, 128, 512)
        assert rc == 0, msg


@pytest.mark.parametrize("tile_n", [256, 128])
def test_exact_count_cap_splits_segments(tile_n):
    """Tiles deeper than the 2^22 bit-row cap (16384 stages): segments are cut
    and accumulators flushed before the cap, on one CTA and on many."""
    for grid in (1, 2, 152):
        rc, msg = jsim.check_tc_schedule([(200, 70001, 70016, 200)], grid, tile_n)
        assert rc == 0, msg


def test_many_collections_like_the_batched_recipe():
    """200 collections of n ~ U{8..512} with uneven word counts, some empty,
    in one launch of 152 CTAs, and in launches of fewer CTAs than
    collections."""
    rng = np.random.default_rng(3)
    jobs = []
    for k in range(200):
        n = int(rng.integers(8, 513))
        W = int(rng.integers(0, 400)) if k % 17 else 0
        stride = stride_of(W)
        rows = -(-n // 128) * 128 if k % 2 else n
        jobs.append((n, W, stride, rows))
    jobs.append((0, 0, 64, 0))
    for grid in (152, 37, 1):
        for tile_n in (256, 128):
            rc, msg = jsim.check_tc_schedule(jobs, grid, tile_n)
            assert rc == 0, msg


def test_check_catches_a_matrix_too_small():
    """The check fails when the matrix lacks rows the schedule reads (so a
    passing check means something)."""
    rc, _ = jsim.check_tc_schedule([(300, 10, 64, 299)], 152)
    assert rc != 0
    rc, _ = jsim.check_tc_schedule([(300, 100, 64, 300)], 152)
    assert rc != 0
