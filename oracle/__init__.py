"""CPU oracle for exact all-pairs Jaccard similarity: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and it imports nothing from the product
path.  The two share no code: the only common inputs are the seeded synthetic
sets, which come from a generator module that holds none of the method's
arithmetic.

Two oracles live here, both written from arXiv 1911.04200:

* ``oracle.c`` (loaded through ``ctypes`` below) is the plain definition:
  distinct-value counts, pairwise intersections by a two-pointer merge of
  sorted lists, union by inclusion-exclusion and the binary64 quotient
  (Sec. II-A, Sec. III-A, Eq. 2), and the Jaccard distance as the binary64
  subtraction 1.0 - J (Sec. II-A).
* ``oracle_rows_range`` in the same file counts the intersections by the
  other plain reading of B = A^T A (Sec. III-A): the sum over values x of
  the outer product of x's 0/1 row, restricted to a value range.  Counts
  over disjoint ranges add up (Eq. 4), so collections larger than memory
  are counted range by range (``rows_range`` below).
* ``packed.py`` follows the paper's batched method step by step in numpy:
  row batches (Eq. 3), the zero-row filter (Eq. 5), its prefix sum and the
  compacted rows (Eq. 6), b-bit bitmask words and the AND+popcount product
  (Eq. 7), accumulated over batches (Eq. 4).  It gives the intermediate
  values (filter bitmap, ranks, packed words) that the kernels' step-level
  parity tests compare against.

Both are pinned by ``tests/test_oracle.py`` against brute force on tiny
inputs, closed forms, invariants and the paper's worked k-mer example.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".tmp.%d" % os.getpid()
    # -ffp-contract=off: the one division must not be fused with anything.
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
           "-fPIC", "-shared", src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_distinct.restype = ctypes.c_uint64
            lib.oracle_distinct.argtypes = [_u64p, ctypes.c_uint64]
            lib.oracle_intersect.restype = ctypes.c_uint64
            lib.oracle_intersect.argtypes = [_u64p, ctypes.c_uint64, _u64p, ctypes.c_uint64]
            lib.oracle_jaccard.restype = ctypes.c_double
            lib.oracle_jaccard.argtypes = [ctypes.c_uint64] * 3
            lib.oracle_distance.restype = ctypes.c_double
            lib.oracle_distance.argtypes = [ctypes.c_uint64] * 3
            lib.oracle_jaccard_matrix.restype = None
            lib.oracle_jaccard_matrix.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p, _u64p, _f64p]
            lib.oracle_rows_range.restype = ctypes.c_int
            lib.oracle_rows_range.argtypes = [ctypes.c_uint64, _u64p, _u64p, ctypes.c_uint64, ctypes.c_uint64,
                                              ctypes.c_uint64, _u64p, ctypes.c_int]
            lib.oracle_distance_matrix.restype = None
            lib.oracle_distance_matrix.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p, _u64p, _f64p]
            lib.oracle_all_pairs.restype = None
            lib.oracle_all_pairs.argtypes = [ctypes.c_uint64, _u64p, _u64p, _u64p, _u64p, _f64p, ctypes.c_int]
            lib.oracle_pairs.restype = None
            lib.oracle_pairs.argtypes = [ctypes.c_uint64, _u64p, _u64p, ctypes.c_uint64, _u64p, _u64p,
                                         _u64p, _f64p, ctypes.c_int]
            lib.oracle_cross.restype = None
            lib.oracle_cross.argtypes = [ctypes.c_uint64, _u64p, _u64p, ctypes.c_uint64, _u64p, _u64p,
                                         _u64p, _u64p, _f64p, ctypes.c_int]
            _lib = lib
    return _lib


def _p64(a):
    return a.ctypes.data_as(_u64p)


def _pf(a):
    return a.ctypes.data_as(_f64p)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def distinct(a) -> int:
    """|X| of one sorted value list."""
    a = _u64(a)
    return int(_load().oracle_distinct(_p64(a), a.size))


def intersect(a, b) -> int:
    """|X ∩ Y| of two sorted value lists (two-pointer merge)."""
    a, b = _u64(a), _u64(b)
    return int(_load().oracle_intersect(_p64(a), a.size, _p64(b), b.size))


def jaccard(inter: int, size_x: int, size_y: int) -> float:
    """b / (|X|+|Y|-b) in binary64, 1.0 for two empty sets."""
    return float(_load().oracle_jaccard(inter, size_x, size_y))


def distance(inter: int, size_x: int, size_y: int) -> float:
    """Jaccard distance 1 - J (Sec. II-A) as the binary64 subtraction 1.0 - J,
    0.0 for two empty sets."""
    return float(_load().oracle_distance(inter, size_x, size_y))


def distance_matrix(C, srow, scol):
    """Distances of a count matrix C (rows x cols) with the row and column
    samples' sizes."""
    C, srow, scol = _u64(C), _u64(srow), _u64(scol)
    nr, nc = C.shape
    D = np.zeros((nr, nc), dtype=np.float64)
    if nr and nc:
        _load().oracle_distance_matrix(nr, nc, _p64(C), _p64(srow), _p64(scol), _pf(D))
    return D


def all_pairs(offsets, ids, threads: int | None = None):
    """All pairs of one collection -> (C uint64 n*n, sizes uint64 n, J float64 n*n)."""
    offsets, ids = _u64(offsets), _u64(ids)
    n = offsets.size - 1
    C = np.zeros((n, n), dtype=np.uint64)
    sizes = np.zeros(n, dtype=np.uint64)
    J = np.zeros((n, n), dtype=np.float64)
    if ids.size == 0:
        ids = np.zeros(1, dtype=np.uint64)
    _load().oracle_all_pairs(n, _p64(offsets), _p64(ids), _p64(C), _p64(sizes), _pf(J),
                             threads or default_threads())
    return C, sizes, J


def pairs(offsets, ids, pi, pj, threads: int | None = None):
    """Sampled pairs (pi[t], pj[t]) -> (C uint64[t], J float64[t])."""
    offsets, ids = _u64(offsets), _u64(ids)
    pi, pj = _u64(pi), _u64(pj)
    C = np.zeros(pi.size, dtype=np.uint64)
    J = np.zeros(pi.size, dtype=np.float64)
    if ids.size == 0:
        ids = np.zeros(1, dtype=np.uint64)
    _load().oracle_pairs(offsets.size - 1, _p64(offsets), _p64(ids), pi.size, _p64(pi), _p64(pj),
                         _p64(C), _pf(J), threads or default_threads())
    return C, J


def sizes_of(offsets, ids):
    """|X_i| of every sample of a collection."""
    offsets, ids = _u64(offsets), _u64(ids)
    return np.array([distinct(ids[offsets[i]:offsets[i + 1]]) for i in range(offsets.size - 1)],
                    dtype=np.uint64)


def cross(qoffsets, qids, roffsets, rids, threads: int | None = None):
    """Queries against a reference collection -> (C nq*nr, qsizes nq, J nq*nr)."""
    qoffsets, qids = _u64(qoffsets), _u64(qids)
    roffsets, rids = _u64(roffsets), _u64(rids)
    nq, nr = qoffsets.size - 1, roffsets.size - 1
    C = np.zeros((nq, nr), dtype=np.uint64)
    qs = np.zeros(nq, dtype=np.uint64)
    J = np.zeros((nq, nr), dtype=np.float64)
    if qids.size == 0:
        qids = np.zeros(1, dtype=np.uint64)
    if rids.size == 0:
        rids = np.zeros(1, dtype=np.uint64)
    _load().oracle_cross(nq, _p64(qoffsets), _p64(qids), nr, _p64(roffsets), _p64(rids),
                         _p64(C), _p64(qs), _pf(J), threads or default_threads())
    return C, qs, J


def jaccard_matrix(C, srow, scol):
    """J of a count matrix C (rows x cols) with the row and column samples'
    sizes, each entry by ``jaccard``."""
    C, srow, scol = _u64(C), _u64(srow), _u64(scol)
    nr, nc = C.shape
    J = np.zeros((nr, nc), dtype=np.float64)
    if nr and nc:
        _load().oracle_jaccard_matrix(nr, nc, _p64(C), _p64(srow), _p64(scol), _pf(J))
    return J


def rows_range(offsets, ids, lo: int, hi: int, C=None, pieces: int | None = None,
               threads: int | None = None):
    """Add to the upper triangle (i <= j) of C (uint64 n*n, created when None)
    the number of values of [lo, hi) that samples i and j both hold, counted
    row by row of the indicator matrix; returns C.  Calls over disjoint
    ranges add up to the whole counts (the diagonal to the sizes)."""
    offsets, ids = _u64(offsets), _u64(ids)
    n = offsets.size - 1
    if C is None:
        C = np.zeros((n, n), dtype=np.uint64)
    assert C.dtype == np.uint64 and C.shape == (n, n) and C.flags.c_contiguous
    if ids.size == 0:
        ids = np.zeros(1, dtype=np.uint64)
    t = threads or default_threads()
    if pieces is None:
        pieces = max(1, min(hi - lo, 64 * t))
    rc = _load().oracle_rows_range(n, _p64(offsets), _p64(ids), lo, hi, pieces, _p64(C), t)
    if rc != 0:
        raise MemoryError("oracle_rows_range: allocation failed")
    return C


def finish_upper(Cu, sizes):
    """Mirror an upper-triangle count matrix and form J: (C n*n, J n*n)."""
    Cu = _u64(Cu)
    C = np.triu(Cu) + np.triu(Cu, 1).T
    return C, jaccard_matrix(C, sizes, sizes)
