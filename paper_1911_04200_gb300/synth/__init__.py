"""Seeded synthetic sample collections for the all-pairs Jaccard workloads.

This module only draws sets of values; it holds none of the similarity
method's arithmetic and imports nothing else from this package.  The CUDA
path's tests and benchmark and the CPU oracle's tests all take their inputs
from here, so both sides see identical collections.

A collection is ``(offsets, ids)``: ``offsets`` is uint64[n+1], sample i is
``ids[offsets[i]:offsets[i+1]]``, sorted ascending with no repeats.

The recipes (``ANCESTRAL``, ``CLADE`` and ``BERNOULLI``) are documented in
``synth.c``.  The
named workloads stand in for the paper's k-mer datasets (Kingsford RNASeq and
BIGSI, Sec. V-A), which are not available here; they reproduce the stated
shapes (sample counts, set-size distributions, value domains, clade
structure), not those datasets.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libjsim_synth.so")
_lock = threading.Lock()
_lib = None

SEED_BASE = 1911042000


class _Params(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("id_bits", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("n", ctypes.c_uint64), ("sample_base", ctypes.c_uint64),
                ("n_anc", ctypes.c_uint64), ("anc_size", ctypes.c_uint64),
                ("n_clades", ctypes.c_uint64), ("core", ctypes.c_double), ("u_max", ctypes.c_double),
                ("median", ctypes.c_double), ("sigma", ctypes.c_double),
                ("lo", ctypes.c_double), ("hi", ctypes.c_double),
                ("m", ctypes.c_uint64), ("p", ctypes.c_double)]


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "synth.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".tmp.%d" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    src, "-o", tmp], check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.synth_lengths.argtypes = [ctypes.POINTER(_Params), u64p]
            lib.synth_lengths.restype = None
            lib.synth_fill.argtypes = [ctypes.POINTER(_Params), u64p, u64p, u64p]
            lib.synth_fill.restype = None
            lib.synth_fill_range.argtypes = [ctypes.POINTER(_Params), u64p, ctypes.c_uint64, ctypes.c_uint64,
                                             u64p, u64p, u64p]
            lib.synth_fill_range.restype = None
            lib.synth_compact.argtypes = [ctypes.c_uint64, u64p, u64p, u64p, u64p]
            lib.synth_compact.restype = ctypes.c_uint64
            lib.synth_range_distinct.argtypes = [ctypes.c_uint64, u64p, ctypes.c_int, ctypes.c_uint64, u64p]
            lib.synth_range_distinct.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _params(kind: str, *, n: int, id_bits: int, seed: int, sample_base: int = 0,
            n_anc: int = 8, anc_size: int = 50_000, u_max: float = 0.6,
            n_clades: int = 32, core: float = 0.3, median: float = 1e6,
            sigma: float | None = None, lo: float | None = None, hi: float | None = None,
            m: int = 0, p: float = 0.0):
    prob = p
    p = _Params()
    p.kind = {"ancestral": 0, "clade": 1, "bernoulli": 2}[kind]
    p.m = m
    p.p = prob
    p.id_bits = id_bits
    p.seed = seed
    p.n = n
    p.sample_base = sample_base
    p.n_anc = n_anc
    p.anc_size = anc_size
    p.n_clades = max(1, n_clades)
    p.core = core
    p.u_max = u_max
    p.median = median
    p.sigma = sigma if sigma is not None else math.log(10.0) / 3.0
    p.lo = lo if lo is not None else median / 10.0
    p.hi = hi if hi is not None else median * 10.0
    return p


def generate(kind: str, *, alloc=None, **kw):
    """Draw one collection.  ``alloc(count) -> uint64 ndarray`` may supply the
    value buffer (for example pinned host memory); it must hold ``count``
    entries and the result is a prefix view of it."""
    p = _params(kind, **kw)
    n = p.n
    lib = _load()
    lens = np.zeros(n, dtype=np.uint64)
    if n:
        lib.synth_lengths(ctypes.byref(p), _ptr(lens))
    slot = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(lens, out=slot[1:])
    total = int(slot[-1])
    ids = alloc(max(total, 1)) if alloc is not None else np.empty(max(total, 1), dtype=np.uint64)
    distinct = np.zeros(n, dtype=np.uint64)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    if n:
        lib.synth_fill(ctypes.byref(p), _ptr(slot), _ptr(ids), _ptr(distinct))
        lib.synth_compact(n, _ptr(slot), _ptr(distinct), _ptr(ids), _ptr(offsets))
    return offsets, ids[:int(offsets[-1])]


def generate_range(kind: str, value_lo: int, value_hi: int, **kw):
    """The collection ``generate(kind, **kw)`` draws, restricted to the values
    of [value_lo, value_hi): every sample keeps its values inside the range (possibly
    none).  The restrictions to disjoint ranges that cover the value domain
    are exactly the pieces of the whole collection, so a collection too large
    for memory can be visited range by range."""
    p = _params(kind, **kw)
    n = p.n
    lib = _load()
    lens = np.zeros(n, dtype=np.uint64)
    counts = np.zeros(n, dtype=np.uint64)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    if n == 0:
        return offsets, np.zeros(0, dtype=np.uint64)
    lib.synth_lengths(ctypes.byref(p), _ptr(lens))
    null = ctypes.POINTER(ctypes.c_uint64)()
    lib.synth_fill_range(ctypes.byref(p), _ptr(lens), value_lo, value_hi, _ptr(counts), null, null)
    np.cumsum(counts, out=offsets[1:])
    ids = np.empty(max(int(offsets[-1]), 1), dtype=np.uint64)
    lib.synth_fill_range(ctypes.byref(p), _ptr(lens), value_lo, value_hi, _ptr(counts), _ptr(offsets), _ptr(ids))
    return offsets, ids[:int(offsets[-1])]


# ---------------------------------------------------------------------------
# The five workloads, and scaled-down variants of the same recipes for tests.
# ---------------------------------------------------------------------------

SIGMA_DECADE = math.log(10.0) / 3.0          # range median/10 .. 10*median at +-3 sigma
SIGMA_C3 = math.log(5e6 / 1e4) / 6.0         # range 1e4 .. 5e6 at +-3 sigma


def ancestral64(seed: int = SEED_BASE + 1, n: int = 64, anc_size: int = 50_000, alloc=None):
    """n=64 samples over [0, 2^20): 8 ancestors of 50k uniform values, each
    sample one ancestor with 0-60 % of its values replaced (plain all-pairs,
    the small case)."""
    return generate("ancestral", n=n, id_bits=20, seed=seed, n_anc=8, anc_size=anc_size,
                    u_max=0.6, alloc=alloc)


def clade1024(seed: int = SEED_BASE + 2, n: int = 1024, median: float = 1e6, alloc=None):
    """n=1024 samples over [0, 2^32): log-normal sizes (median 1e6, range
    1e5-1e7), 32 clades, 30 % shared core, 0-40 % substitution."""
    return generate("clade", n=n, id_bits=32, seed=seed, n_clades=32, core=0.3, u_max=0.4,
                    median=median, sigma=SIGMA_DECADE, lo=median / 10, hi=median * 10, alloc=alloc)


def batched_collection(k: int, seed: int = SEED_BASE + 3, n_lo: int = 8, n_hi: int = 512,
                       median: float = 2e5, lo: float = 1e4, hi: float = 5e6, alloc=None):
    """Collection k of the batched recipe: n ~ U{n_lo..n_hi} samples (a
    per-collection splitmix64 draw), sizes log-normal (median 2e5, range
    1e4-5e6, both scaled with the median), values in [0, 2^32), ceil(n/32)
    clades."""
    h = (seed * 0x9E3779B97F4A7C15 + k * 0xBF58476D1CE4E5B9) & (2**64 - 1)
    h ^= h >> 31
    n = n_lo + (h % (n_hi - n_lo + 1))
    scale = median / 2e5
    return generate("clade", n=n, id_bits=32, seed=seed * 1000 + k, n_clades=(n + 31) // 32,
                    core=0.3, u_max=0.4, median=median, sigma=SIGMA_C3,
                    lo=lo * scale, hi=hi * scale, alloc=alloc)


def batched_collections(seed: int = SEED_BASE + 3, count: int = 200, n_lo: int = 8, n_hi: int = 512,
                        median: float = 2e5, lo: float = 1e4, hi: float = 5e6, first: int = 0):
    """Collections first .. first+count-1 of the batched recipe (200
    independent collections with n ~ U{n_lo..n_hi} samples, sizes log-normal
    (median 2e5, range 1e4-5e6), values in [0, 2^32), ceil(n/32) clades
    each)."""
    return [batched_collection(k, seed=seed, n_lo=n_lo, n_hi=n_hi, median=median, lo=lo, hi=hi)
            for k in range(first, first + count)]


def _clade4096_kw(seed, n, median):
    return dict(n=n, id_bits=40, seed=seed, n_clades=64, core=0.3, u_max=0.4,
                median=median, sigma=SIGMA_DECADE, lo=median / 10, hi=median * 10)


def clade4096(seed: int = SEED_BASE + 4, n: int = 4096, median: float = 2e6, alloc=None):
    """n=4096 samples over [0, 2^40): sizes log-normal (median 2e6, range
    2e5-2e7), 64 clades; about 1e10 values in total."""
    return generate("clade", alloc=alloc, **_clade4096_kw(seed, n, median))


def clade4096_range(value_lo: int, value_hi: int, seed: int = SEED_BASE + 4, n: int = 4096,
                    median: float = 2e6):
    """``clade4096`` restricted to the values of [value_lo, value_hi)."""
    return generate_range("clade", value_lo, value_hi, **_clade4096_kw(seed, n, median))


def serving_reference(seed: int = SEED_BASE + 5, n: int = 2048, median: float = 1e6, alloc=None):
    """Reference of 2048 samples over [0, 2^32), median 1e6 (1e5-1e7), 64 clades."""
    return generate("clade", n=n, id_bits=32, seed=seed, n_clades=64, core=0.3, u_max=0.4,
                    median=median, sigma=SIGMA_DECADE, lo=median / 10, hi=median * 10, alloc=alloc)


def serving_queries(first: int, count: int, seed: int = SEED_BASE + 5, n_ref: int = 2048,
                    median: float = 1e6):
    """`count` new query samples from the reference's clades (sample indices
    n_ref + first ...), sizes log-normal median 1e6 (1e5-1e7)."""
    return generate("clade", n=count, id_bits=32, seed=seed, sample_base=n_ref + first, n_clades=64,
                    core=0.3, u_max=0.4, median=median, sigma=SIGMA_DECADE,
                    lo=median / 10, hi=median * 10)


def bernoulli(n: int, m: int, p: float, seed: int = SEED_BASE + 6, alloc=None):
    """n samples over [0, m): every value is in every sample independently
    with probability p (the paper's synthetic indicator matrices, Sec. V-A:
    density p)."""
    bits = max(1, int(m - 1).bit_length())
    return generate("bernoulli", n=n, id_bits=bits, seed=seed, m=m, p=p, alloc=alloc)


def bernoulli10k(seed: int = SEED_BASE + 6, alloc=None):
    """The paper's synthetic strong-scaling matrix: m = 32M (2^25) rows,
    n = 10,000 samples, density p = 0.01 (about 3.4e9 values)."""
    return bernoulli(10_000, 1 << 25, 0.01, seed=seed, alloc=alloc)


def range_distinct(ids, range_bits: int, nranges: int):
    """Distinct values of a whole collection per aligned range of 2^range_bits
    values (a workload statistic: with batches of that size, batch r has
    counts[r] nonzero rows and ceil(counts[r] / 64) packed words per sample)."""
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    counts = np.zeros(nranges, dtype=np.uint64)
    rc = _load().synth_range_distinct(ids.size, _ptr(ids), range_bits, nranges, _ptr(counts))
    if rc != 0:
        raise ValueError("range_distinct failed (%d)" % rc)
    return counts
