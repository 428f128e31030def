"""The paper's batched bitmask method, step by step, in numpy: TEST INFRASTRUCTURE ONLY.

Written from Sec. III-B of arXiv 1911.04200 in the paper's order and notation.
Rows of the indicator matrix A (Sec. III-A) are the value domain, columns are
samples: a_ki = 1 iff value k is in sample i.  Values are 0-based here (the
paper's 1..m shifted by one), and a value is any unsigned 64-bit integer.

For each row batch l (Eq. 3), the rows [l*mt, (l+1)*mt) with mt = m~:

  f^(l)_k = 1 iff some sample holds value l*mt + k            (Eq. 5)
  p^(l)   = exclusive prefix sum of f^(l)                     (text before Eq. 6)
  abar^(l)_{p_k, i} = a^(l)_{k, i}                            (Eq. 6)
  ahat^(l): b consecutive rows of abar^(l) -> one b-bit word,
            row r goes to word r // b, bit r % b (LSB first)  (text before Eq. 7)
  s^(l)_ij = sum_w popcount(ahat^(l)_wi AND ahat^(l)_wj)      (Eq. 7)
  ahat_i^(l) = sum_k a^(l)_ki                                  (Eq. 4)

and B = sum_l s^(l), ahat = sum_l ahat^(l) (Eq. 4), then the union
c_ij = ahat_i + ahat_j - b_ij and s_ij = b_ij / c_ij (Sec. III-A, Eq. 2).

The bit order inside a word (LSB = lowest rank) and the zero padding of the
last word are this library's reading; neither can change any count.  Packed
words are stored sample-major: ``words[i, w]`` is word w of sample i.
"""
from __future__ import annotations

import numpy as np


def batch_members(offsets, ids, lo: int, hi: int):
    """Per-sample values that fall in the row batch [lo, hi) (Eq. 3)."""
    offsets = np.asarray(offsets, dtype=np.uint64)
    ids = np.asarray(ids, dtype=np.uint64)
    out = []
    for i in range(offsets.size - 1):
        seg = ids[int(offsets[i]):int(offsets[i + 1])]
        sel = seg[(seg >= np.uint64(lo)) & (seg < np.uint64(hi))] if hi > lo else seg[:0]
        out.append(sel)
    return out


def filter_vector(members, lo: int, mt: int, min_count: int = 1):
    """f^(l) as a boolean array of length mt (Eq. 5): rows held by at least
    min_count samples.  min_count 1 is the paper's filter; min_count 2 keeps
    the rows two or more samples hold (the library's filter_min 2 option: a
    row held by sample i alone adds 1 to b_ii and nothing else)."""
    cnt = np.zeros(mt, dtype=np.int64)
    for seg in members:
        if seg.size:
            np.add.at(cnt, (np.unique(seg) - np.uint64(lo)).astype(np.int64), 1)
    return cnt >= min_count


def prefix_sum(f):
    """p^(l)_k = number of nonzero rows before row k (exclusive prefix sum)."""
    c = np.cumsum(f, dtype=np.int64)
    return c - f.astype(np.int64)


def bitmask_words(members, lo: int, p, R: int, b: int = 64, f=None):
    """ahat^(l): sample-major words[n, ceil(R/b)] of b bits (uint32 or uint64);
    with f, only the values whose row f keeps."""
    assert b in (32, 64)
    dt = np.uint64 if b == 64 else np.uint32
    W = (R + b - 1) // b
    words = np.zeros((len(members), W), dtype=dt)
    for i, seg in enumerate(members):
        if f is not None and seg.size:
            seg = seg[f[(seg - np.uint64(lo)).astype(np.int64)]]
        if seg.size == 0:
            continue
        r = p[(seg - np.uint64(lo)).astype(np.int64)]
        w = r // b
        bit = (np.ones(r.size, dtype=dt) << (r % b).astype(dt))
        np.bitwise_or.at(words[i], w, bit)
    return words


_POP8 = np.array([bin(v).count("1") for v in range(256)], dtype=np.uint8)


def popcount(x):
    """Number of set bits of every element of an unsigned integer array."""
    x = np.ascontiguousarray(x)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(x)
    return _POP8[x.view(np.uint8)].reshape(x.shape + (x.itemsize,)).sum(axis=-1)


def popcount_product(words):
    """s^(l)_ij = sum_w popcount(ahat_wi AND ahat_wj) for all pairs (Eq. 7)."""
    n = words.shape[0]
    s = np.zeros((n, n), dtype=np.uint64)
    for i in range(n):
        s[i, :] = popcount(words[i][None, :] & words).sum(axis=1, dtype=np.uint64)
    return s


def column_sums(members):
    """ahat^(l)_i = number of distinct values of sample i in the batch (Eq. 4)."""
    return np.array([np.unique(seg).size for seg in members], dtype=np.uint64)


def run_batch(offsets, ids, lo: int, mt: int, b: int = 64, min_count: int = 1):
    """All intermediate values of one batch, as a dict."""
    members = batch_members(offsets, ids, lo, lo + mt)
    f = filter_vector(members, lo, mt, min_count)
    p = prefix_sum(f)
    R = int(f.sum())
    words = bitmask_words(members, lo, p, R, b, f if min_count > 1 else None)
    return {"members": members, "f": f, "p": p, "R": R, "words": words,
            "s": popcount_product(words), "ahat": column_sums(members)}


def jaccard_matrix(B, ahat):
    """c_ij = ahat_i + ahat_j - b_ij, s_ij = b_ij / c_ij (binary64), 1 when c_ij = 0."""
    B = np.asarray(B, dtype=np.uint64)
    a = np.asarray(ahat, dtype=np.uint64)
    U = a[:, None] + a[None, :] - B
    J = np.ones(B.shape, dtype=np.float64)
    nz = U != 0
    J[nz] = B[nz].astype(np.float64) / U[nz].astype(np.float64)
    return J


def similarity_at_scale(offsets, ids, mt: int, m: int, b: int = 64):
    """Listing 1 end to end: batches of mt rows over [0, m), accumulated (Eq. 4).

    The last batch may be partial: r = ceil(m / mt) batches.
    """
    offsets = np.asarray(offsets, dtype=np.uint64)
    n = offsets.size - 1
    B = np.zeros((n, n), dtype=np.uint64)
    ahat = np.zeros(n, dtype=np.uint64)
    r = (m + mt - 1) // mt
    for l in range(r):
        lo = l * mt
        width = min(mt, m - lo)
        out = run_batch(offsets, ids, lo, width, b)
        B += out["s"]
        ahat += out["ahat"]
    return B, ahat, jaccard_matrix(B, ahat)
