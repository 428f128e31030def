"""Pins of the CPU oracles against facts fixed by the paper and by mathematics.

Nothing here compares an oracle with itself or retypes its formula: each
check uses an independent route (dense boolean A^T A by matrix product,
Python's exact integer division, Python sets, closed forms for interval
sets, the metric property of the Jaccard distance, the paper's worked k-mer
example), chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import packed

HERE = os.path.dirname(os.path.abspath(__file__))


def random_collection(rng, n, m, density, dup_prob=0.0):
    """Tiny collection as (offsets, ids, dense A[m, n])."""
    A = (rng.random((m, n)) < density)
    segs = []
    for i in range(n):
        v = np.flatnonzero(A[:, i]).astype(np.uint64)
        if dup_prob and v.size:
            rep = rng.random(v.size) < dup_prob
            v = np.sort(np.concatenate([v, v[rep]]))
        segs.append(v)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([s.size for s in segs])
    ids = np.concatenate(segs) if segs else np.zeros(0, dtype=np.uint64)
    return offsets, ids.astype(np.uint64), A


def exact_jaccard(c, si, sj):
    """Correctly rounded binary64 of c / (si + sj - c) via Python's exact int division."""
    u = int(si) + int(sj) - int(c)
    return 1.0 if u == 0 else int(c) / u


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("density", [0.0, 0.05, 0.3, 0.9, 1.0])
def test_brute_force_dense_AtA(seed, density):
    """Sec. III-A: B = A^T A and a-hat = column sums, from a dense 0/1 matrix product."""
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 13)), int(rng.integers(1, 300))
    offsets, ids, A = random_collection(rng, n, m, density)
    C, sizes, J = oracle.all_pairs(offsets, ids)
    Ai = A.astype(np.int64)
    np.testing.assert_array_equal(C.astype(np.int64), Ai.T @ Ai)
    np.testing.assert_array_equal(sizes.astype(np.int64), Ai.sum(axis=0))
    for i in range(n):
        for j in range(n):
            c = int((Ai[:, i] * Ai[:, j]).sum())
            assert J[i, j] == exact_jaccard(c, Ai[:, i].sum(), Ai[:, j].sum())


def test_exact_division_matches_fraction():
    """The quotient is the correctly rounded value of the exact rational."""
    rng = np.random.default_rng(7)
    for _ in range(2000):
        si, sj = (int(x) for x in rng.integers(0, 2**40, 2))
        c = int(rng.integers(0, min(si, sj) + 1))
        u = si + sj - c
        ref = 1.0 if u == 0 else float(Fraction(c, u))
        assert oracle.jaccard(c, si, sj) == ref


def test_python_sets():
    rng = np.random.default_rng(11)
    segs = [np.unique(rng.integers(0, 20000, int(rng.integers(0, 4000)))).astype(np.uint64) for _ in range(7)]
    segs.append(np.zeros(0, dtype=np.uint64))
    offsets = np.zeros(len(segs) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([s.size for s in segs])
    ids = np.concatenate(segs)
    C, sizes, J = oracle.all_pairs(offsets, ids)
    for i, a in enumerate(segs):
        assert sizes[i] == len(set(a.tolist()))
        for j, b in enumerate(segs):
            inter = len(set(a.tolist()) & set(b.tolist()))
            union = len(set(a.tolist()) | set(b.tolist()))
            assert C[i, j] == inter
            assert J[i, j] == (1.0 if union == 0 else inter / union)


def test_interval_sets_closed_form():
    """X_i = [a_i, b_i): |X_i ∩ X_j| = max(0, min(b) - max(a))."""
    rng = np.random.default_rng(3)
    n = 10
    a = rng.integers(0, 10**6, n)
    b = a + rng.integers(0, 10**5, n)
    segs = [np.arange(a[i], b[i], dtype=np.uint64) for i in range(n)]
    offsets = np.zeros(n + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([s.size for s in segs])
    C, sizes, J = oracle.all_pairs(offsets, np.concatenate(segs))
    for i in range(n):
        assert sizes[i] == b[i] - a[i]
        for j in range(n):
            assert C[i, j] == max(0, min(b[i], b[j]) - max(a[i], a[j]))


def test_special_cases():
    """Empty/empty J = 1 (Sec. II-A), empty/non-empty 0, disjoint 0, nested |small|, J_ii = 1."""
    segs = [np.zeros(0, np.uint64), np.zeros(0, np.uint64), np.array([1, 5, 9], np.uint64),
            np.array([2, 4, 6, 8], np.uint64), np.array([5], np.uint64), np.array([1, 5, 9, 11, 2**63], np.uint64),
            np.array([0, 2**64 - 1], np.uint64)]
    offsets = np.zeros(len(segs) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([s.size for s in segs])
    C, sizes, J = oracle.all_pairs(offsets, np.concatenate(segs))
    assert J[0, 1] == 1.0 and J[0, 0] == 1.0 and C[0, 1] == 0
    assert J[0, 2] == 0.0 and J[2, 0] == 0.0
    assert C[2, 3] == 0 and J[2, 3] == 0.0
    assert C[2, 4] == 1 and J[2, 4] == 1 / 3
    assert C[2, 5] == 3 and J[2, 5] == 3 / 5
    assert C[5, 6] == 0 and sizes[6] == 2 and C[6, 6] == 2
    assert np.all(np.diag(J) == 1.0)


def test_duplicates_are_one_element():
    rng = np.random.default_rng(5)
    o1, i1, A = random_collection(rng, 8, 400, 0.2)
    rng = np.random.default_rng(5)
    o2, i2, _ = random_collection(rng, 8, 400, 0.2, dup_prob=0.5)
    assert i2.size > i1.size
    r1, r2 = oracle.all_pairs(o1, i1), oracle.all_pairs(o2, i2)
    for x, y in zip(r1, r2):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("seed", range(3))
def test_invariants_and_metric(seed):
    """Symmetry, C_ii = |X_i|, C_ij <= min, 0 <= J <= 1, inclusion-exclusion against
    an independently merged union, and the triangle inequality of d_J = 1 - J (Sec. II-A)."""
    rng = np.random.default_rng(100 + seed)
    n = 9
    segs = [np.unique(rng.integers(0, 3000, int(rng.integers(0, 900)))).astype(np.uint64) for _ in range(n)]
    offsets = np.zeros(n + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([s.size for s in segs])
    C, sizes, J = oracle.all_pairs(offsets, np.concatenate(segs))
    assert np.array_equal(C, C.T) and np.array_equal(J, J.T)
    assert np.array_equal(np.diag(C), sizes)
    assert np.all(C <= np.minimum(sizes[:, None], sizes[None, :]))
    assert np.all((J >= 0) & (J <= 1))
    for i in range(n):
        for j in range(n):
            assert sizes[i] + sizes[j] - C[i, j] == np.union1d(segs[i], segs[j]).size
    D = 1.0 - J
    for i in range(n):
        for j in range(n):
            for k in range(n):
                assert D[i, k] <= D[i, j] + D[j, k] + 1e-12


def test_pairs_and_cross_agree_with_all_pairs():
    rng = np.random.default_rng(9)
    offsets, ids, _ = random_collection(rng, 10, 500, 0.1)
    C, sizes, J = oracle.all_pairs(offsets, ids)
    pi = np.array([0, 3, 9, 9, 4], np.uint64)
    pj = np.array([0, 7, 2, 9, 4], np.uint64)
    Cp, Jp = oracle.pairs(offsets, ids, pi, pj)
    assert np.array_equal(Cp, C[pi.astype(int), pj.astype(int)])
    assert np.array_equal(Jp, J[pi.astype(int), pj.astype(int)])
    Cx, qs, Jx = oracle.cross(offsets[:4] - offsets[0], ids[:int(offsets[3])], offsets, ids)
    assert np.array_equal(Cx, C[:3]) and np.array_equal(Jx, J[:3]) and np.array_equal(qs, sizes[:3])


def encode_kmer(s):
    v = 0
    for ch in s:
        v = v * 4 + "ACGT".index(ch)
    return v


def test_paper_kmer_example():
    """Sec. II-B: AATGTC has four 3-mers and three 4-mers."""
    with open(os.path.join(HERE, "golden", "kmer_example.json")) as f:
        g = json.load(f)
    seq = g["sequence"]
    segs = []
    for k in ("3", "4"):
        listed = g["kmers"][k]
        kk = int(k)
        mine = [seq[t:t + kk] for t in range(len(seq) - kk + 1)]
        assert mine == listed
        segs.append(np.array(sorted(encode_kmer(x) for x in listed), dtype=np.uint64))
    offsets = np.array([0, segs[0].size, segs[0].size + segs[1].size], np.uint64)
    C, sizes, J = oracle.all_pairs(offsets, np.concatenate(segs))
    assert sizes.tolist() == [g["counts"]["3"], g["counts"]["4"]]
    assert J[0, 0] == 1.0 and J[1, 1] == 1.0


# ---- the packed-method oracle (Sec. III-B) -----------------------------------

@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("b", [32, 64])
def test_packed_method_equals_definition(seed, b):
    """Eq. 7 summed over batches (Eq. 4) equals A^T A for several batch sizes."""
    rng = np.random.default_rng(200 + seed)
    n, m = 7, 3000
    offsets, ids, A = random_collection(rng, n, m, [0.001, 0.02, 0.2, 0.7][seed])
    Ai = A.astype(np.int64)
    for mt in (64, 192, 1024, 4096):
        B, ahat, J = packed.similarity_at_scale(offsets, ids, mt, m, b)
        np.testing.assert_array_equal(B.astype(np.int64), Ai.T @ Ai)
        np.testing.assert_array_equal(ahat.astype(np.int64), Ai.sum(axis=0))
        Co, so, Jo = oracle.all_pairs(offsets, ids)
        np.testing.assert_array_equal(J, Jo)


def test_filter_invariance_and_word_layout():
    """A^T A = Abar^T Abar (Sec. III-B): packing the raw rows (no filter) gives
    the same products as packing the filtered rows; b = 32 and b = 64 words
    hold the same bits (little-endian halves)."""
    rng = np.random.default_rng(17)
    offsets, ids, A = random_collection(rng, 6, 640, 0.05)
    out = packed.run_batch(offsets, ids, 0, 640, 64)
    raw = packed.bitmask_words(out["members"], 0, np.arange(640), 640, 64)
    np.testing.assert_array_equal(packed.popcount_product(raw), out["s"])
    assert out["R"] == int(A.any(axis=1).sum())
    w32 = packed.bitmask_words(out["members"], 0, out["p"], out["R"], 32)
    w64 = out["words"]
    pad = np.zeros((w64.shape[0], 2 * w64.shape[1]), dtype=np.uint32)
    pad[:, :w32.shape[1]] = w32
    np.testing.assert_array_equal(pad.view(np.uint64), w64)
    # rank p_k of every nonzero row is its position among nonzero rows
    nz = np.flatnonzero(out["f"])
    np.testing.assert_array_equal(out["p"][nz], np.arange(nz.size))


@pytest.mark.parametrize("seed", range(4))
def test_two_or_more_filter_keeps_every_off_diagonal_count(seed):
    """Rows held by a single sample (the library's filter_min 2 drops them)
    add only to that sample's diagonal entry: packing the rows held by two or
    more samples gives A^T A off the diagonal, and the column sums restore the
    diagonal.  Pinned against the dense 0/1 product, duplicates included."""
    rng = np.random.default_rng(300 + seed)
    n, m = 9, 2000
    offsets, ids, A = random_collection(rng, n, m, [0.002, 0.03, 0.3, 0.8][seed], dup_prob=0.2)
    Ai = A.astype(np.int64)
    AtA = Ai.T @ Ai
    for mt in (64, 512, 2048):
        B = np.zeros((n, n), dtype=np.int64)
        for lo in range(0, m, mt):
            width = min(mt, m - lo)
            out = packed.run_batch(offsets, ids, lo, width, 64, min_count=2)
            B += out["s"].astype(np.int64)
            counts = A[lo:lo + width].sum(axis=1)
            np.testing.assert_array_equal(out["f"], counts >= 2)
            assert out["R"] == int((counts >= 2).sum())
        off = ~np.eye(n, dtype=bool)
        np.testing.assert_array_equal(B[off], AtA[off])
        assert np.all(np.diag(B) <= np.diag(AtA))
        B[np.diag_indices(n)] = Ai.sum(axis=0)
        np.testing.assert_array_equal(B, AtA)


def test_pins_catch_planted_mistakes():
    """A union without the -C term, or an off-by-one in the merge, fails the
    brute-force pin (mistakes planted in copies of the oracle's formulas)."""
    rng = np.random.default_rng(23)
    offsets, ids, A = random_collection(rng, 6, 200, 0.3)
    Ai = A.astype(np.int64)
    ref_C = Ai.T @ Ai
    s = Ai.sum(axis=0)
    wrong_J = ref_C / np.maximum(s[:, None] + s[None, :], 1)  # dropped "- C"
    _, _, J = oracle.all_pairs(offsets, ids)
    assert not np.array_equal(wrong_J, J)
    segs = [ids[int(offsets[i]):int(offsets[i + 1])] for i in range(6)]
    off_by_one = np.array([[np.intersect1d(a[1:], b).size for b in segs] for a in segs])
    assert not np.array_equal(off_by_one, ref_C)


def test_bernoulli_recipe_statistics():
    """Statistical sanity of the synthetic Bernoulli(p) matrices (Sec. V-A):
    sizes average m p, pairwise intersections m p^2, and J about p / (2 - p);
    the draw is sorted, distinct, inside [0, m) and repeatable."""
    from paper_1911_04200_gb300 import synth
    n, m, p = 48, 1 << 16, 0.05
    off, ids = synth.bernoulli(n, m, p)
    off2, ids2 = synth.bernoulli(n, m, p)
    np.testing.assert_array_equal(off, off2)
    np.testing.assert_array_equal(ids, ids2)
    for i in range(n):
        a = ids[int(off[i]):int(off[i + 1])].astype(np.int64)
        assert np.all(np.diff(a) > 0) and a[0] >= 0 and a[-1] < m
    C, s, J = oracle.all_pairs(off, ids)
    sd_size = np.sqrt(m * p * (1 - p))
    assert abs(s.astype(np.float64).mean() - m * p) < 4 * sd_size / np.sqrt(n)
    iu = np.triu_indices(n, 1)
    c = C[iu].astype(np.float64)
    # pairs share samples, so allow a wide band: 8 standard errors of independent pairs
    assert abs(c.mean() - m * p * p) < 8 * np.sqrt(m * p * p) / np.sqrt(c.size)
    assert abs(J[iu].mean() - p / (2 - p)) < 0.002
    # the extremes: p = 1 gives every value, p = 0 none
    o1, i1 = synth.bernoulli(3, 1000, 1.0)
    np.testing.assert_array_equal(i1, np.tile(np.arange(1000, dtype=np.uint64), 3))
    o0, i0 = synth.bernoulli(3, 1000, 0.0)
    assert int(o0[-1]) == 0


def test_distance_is_one_minus_J_within_one_rounding():
    """D = 1 - J (Sec. II-A) in binary64: D lies within two roundings (half an
    ulp of J and half an ulp of D) of the exact rational (U - C) / U (checked
    with fractions), within J's rounding alone when J >= 1/2 (then 1 - J has
    no rounding), D(empty, empty) = 0,
    D(X, X) = 0, D of disjoint sets = 1, and the distance obeys the triangle
    inequality on random small sets."""
    rng = np.random.default_rng(31)
    for _ in range(400):
        sx, sy = (int(v) for v in rng.integers(0, 10**6, 2))
        b = int(rng.integers(0, min(sx, sy) + 1))
        d = oracle.distance(b, sx, sy)
        u = sx + sy - b
        if u == 0:
            assert d == 0.0
            continue
        exact = Fraction(u - b, u)
        j = oracle.jaccard(b, sx, sy)
        # two roundings at most: J's (half an ulp of J) and the subtraction's
        # (half an ulp of D)
        bound = (Fraction(float(np.spacing(j))) + Fraction(float(np.spacing(d)))) / 2
        assert abs(Fraction(d) - exact) <= bound
        if 2 * b >= u:  # J >= 1/2: 1 - J is exact, only J's rounding remains
            assert abs(Fraction(d) - exact) <= Fraction(float(np.spacing(j))) / 2
    assert oracle.distance(0, 0, 0) == 0.0
    assert oracle.distance(7, 7, 7) == 0.0
    assert oracle.distance(0, 3, 5) == 1.0
    # metric: d(a, c) <= d(a, b) + d(b, c) (up to one rounding each)
    sets = [set(rng.integers(0, 40, int(rng.integers(0, 30))).tolist()) for _ in range(12)]

    def dist(p, q):
        return oracle.distance(len(p & q), len(p), len(q))
    for p in sets:
        for q in sets:
            for r in sets:
                assert dist(p, r) <= dist(p, q) + dist(q, r) + 1e-15
    # the matrix form matches the scalar one
    C = np.array([[3, 1], [0, 2]], dtype=np.uint64)
    D = oracle.distance_matrix(C, np.array([3, 4], np.uint64), np.array([5, 2], np.uint64))
    assert D[0, 0] == oracle.distance(3, 3, 5) and D[1, 1] == oracle.distance(2, 4, 2)


def permute_rows(offsets, ids, bits=64, a=0x9E3779B97F4A7C15, b=0x632BE59BD9B4E019):
    """Relabel every value of [0, 2^bits) by x -> a*x + b mod 2^bits (a
    bijection of that domain: a is odd) and re-sort each sample."""
    mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(2**64 - 1)
    out = np.empty_like(ids)
    for i in range(len(offsets) - 1):
        s, e = int(offsets[i]), int(offsets[i + 1])
        v = (ids[s:e].astype(np.uint64) * np.uint64(a) + np.uint64(b)) & mask
        out[s:e] = np.sort(v)
    return offsets.copy(), out


def test_row_permutation_invariance():
    """Reordering the rows of the indicator matrix (Sec. III-C permutes rows
    for load balance) changes no count: the oracle gives the same C, sizes
    and J for a collection and for its values relabelled by a bijection of
    the 64-bit domain."""
    from paper_1911_04200_gb300 import synth
    off, ids = synth.clade1024(n=40, median=3e3)
    poff, pids = permute_rows(off, ids)
    assert not np.array_equal(pids, ids)
    C0, s0, J0 = oracle.all_pairs(off, ids)
    C1, s1, J1 = oracle.all_pairs(poff, pids)
    np.testing.assert_array_equal(C0, C1)
    np.testing.assert_array_equal(s0, s1)
    np.testing.assert_array_equal(J0.view(np.uint64), J1.view(np.uint64))


@pytest.mark.parametrize("seed", range(5))
def test_rows_range_sums_to_dense_AtA(seed):
    """The row-by-row count (B = sum over rows a_x a_x^T, Sec. III-A),
    restricted to value ranges and added over a partition of the values
    (Eq. 4), equals the dense A^T A by integer matrix product and the
    pairwise merge; cuts land on values that samples hold, so a range bound
    taken inclusive or exclusive the wrong way shows up, and duplicates
    inside a sample count once."""
    rng = np.random.default_rng(100 + seed)
    n, m = int(rng.integers(1, 14)), int(rng.integers(1, 600))
    density = [0.0, 0.02, 0.3, 0.8, 1.0][seed]
    offsets, ids, A = random_collection(rng, n, m, density, dup_prob=0.2)
    Ai = A.astype(np.int64)
    AtA = Ai.T @ Ai
    held = np.unique(ids).astype(np.int64)
    picks = rng.choice(held, size=min(4, held.size), replace=False) if held.size else np.zeros(0, np.int64)
    cuts = sorted(set([0, m] + [int(x) for x in picks] + [int(x) + 1 for x in picks]))
    cuts = [c for c in cuts if 0 <= c <= m]
    Cu = np.zeros((n, n), dtype=np.uint64)
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        oracle.rows_range(offsets, ids, lo, hi, Cu, pieces=int(rng.integers(1, 9)))
    np.testing.assert_array_equal(Cu.astype(np.int64), np.triu(AtA))
    C, J = oracle.finish_upper(Cu, Ai.sum(axis=0).astype(np.uint64))
    Cm, sm, Jm = oracle.all_pairs(offsets, ids)
    np.testing.assert_array_equal(C, Cm)
    np.testing.assert_array_equal(J.view(np.uint64), Jm.view(np.uint64))
    # one range alone: the rows of A inside it
    if len(cuts) > 2:
        lo, hi = cuts[1], cuts[2]
        part = oracle.rows_range(offsets, ids, lo, hi)
        Ar = Ai[lo:hi]
        np.testing.assert_array_equal(part.astype(np.int64), np.triu(Ar.T @ Ar))


def test_rows_range_interval_closed_form_and_empty_ranges():
    """Interval sets [a_i, b_i): the count restricted to [lo, hi) is the
    length of [max(a_i, a_j, lo), min(b_i, b_j, hi)), zero when negative; a
    range nobody holds adds nothing."""
    rng = np.random.default_rng(31)
    n = 9
    a = rng.integers(0, 5000, n)
    b = a + rng.integers(0, 4000, n)
    segs = [np.arange(a[i], b[i], dtype=np.uint64) for i in range(n)]
    off = np.zeros(n + 1, dtype=np.uint64)
    off[1:] = np.cumsum([s.size for s in segs])
    ids = np.concatenate(segs)
    for lo, hi in [(0, 10000), (1234, 5678), (7000, 9100), (20000, 30000)]:
        Cu = oracle.rows_range(off, ids, lo, hi, pieces=7)
        for i in range(n):
            for j in range(i, n):
                want = max(0, min(b[i], b[j], hi) - max(a[i], a[j], lo))
                assert int(Cu[i, j]) == want
                if j > i:
                    assert int(Cu[j, i]) == 0


def test_generated_ranges_tile_the_collection():
    """The generator's restriction to disjoint value ranges gives exactly the
    pieces of the whole collection, for the clade, ancestral and Bernoulli
    recipes (so an out-of-memory collection can be visited range by range)."""
    from paper_1911_04200_gb300 import synth
    cases = [
        ("clade", dict(n=40, id_bits=40, seed=77, n_clades=4, core=0.3, u_max=0.4, median=3e3,
                       sigma=synth.SIGMA_DECADE, lo=300, hi=3e4), [0, 1 << 20, 5 << 36, 1 << 39, 1 << 40]),
        ("ancestral", dict(n=16, id_bits=20, seed=5, n_anc=4, anc_size=3000, u_max=0.6),
         [0, 77777, 500000, 1 << 20]),
        ("bernoulli", dict(n=20, id_bits=16, seed=9, m=1 << 16, p=0.05), [0, 1, 30000, 1 << 16]),
    ]
    for kind, kw, cuts in cases:
        off, ids = synth.generate(kind, **kw)
        parts = [synth.generate_range(kind, lo, hi, **kw) for lo, hi in zip(cuts[:-1], cuts[1:])]
        for i in range(len(off) - 1):
            whole = ids[int(off[i]):int(off[i + 1])]
            pieces = [pi[int(po[i]):int(po[i + 1])] for po, pi in parts]
            for (lo, hi), piece in zip(zip(cuts[:-1], cuts[1:]), pieces):
                assert piece.size == 0 or (int(piece[0]) >= lo and int(piece[-1]) < hi)
            np.testing.assert_array_equal(whole, np.concatenate(pieces))
