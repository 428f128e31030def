"""Write tests/golden/full_size_sha256.json: SHA-256 digests of the oracle's
results (C, sizes as uint64, J as binary64 bit patterns, all row-major
little-endian) for the workloads at their full sizes, together with a digest
of the generated input.  Calls only the oracle and the seeded input
generator; run it once on any machine (the generator draws identical sets on
x86-64 and AArch64):

    python tests/golden/make_full_size_hashes.py [workload ...]

Workloads and the oracle route each takes:

* ancestral64 (64 samples, 3.1e6 values) and clade1024 (1024 samples,
  1.3e9 values; 12 minutes of 8 host cores): the pairwise merge
  (oracle.all_pairs).  C as uint32.
* batched200: all 200 collections of the batched recipe (n ~ U{8..512},
  sizes log-normal median 2e5 in [1e4, 5e6], 1.8e10 values in all), one at a
  time, counted by rows of the indicator matrix (oracle.rows_range over the
  whole value range).  C as uint32; digests over the collections in order,
  plus a short digest per collection for diagnosis.
* stream4096 (4096 samples, 1.1e10 values in [0, 2^40), 88 GB: more than
  this machine's memory): drawn and counted range by range (PASSES equal
  ranges of the value domain; oracle.rows_range per range, added up, Eq. 4),
  sizes added per range.  C as uint64 (the workload's count width).  The
  input digest runs over the ranges in order: each range's offsets, then its
  values.
* serve2048_q256: the first 256 query samples of the serving recipe against
  the whole 2048-sample reference, by the pairwise merge (oracle.cross).  C
  as uint32 (256 x 2048).

``check-rows`` recomputes clade1024 by rows (oracle.rows_range) and compares
it with the stored merge digests: the two oracle routes must agree.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1911_04200_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "full_size_sha256.json")
PASSES = 4                     # value ranges of the out-of-memory workload
N_BATCHED = 200
N_QUERY = 256


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes()).hexdigest()


def input_digest(off, ids, h=None):
    h = h or hashlib.sha256()
    h.update(np.ascontiguousarray(off, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(ids, dtype="<u8").tobytes())
    return h


FP_STRIDE = 4093


def fingerprint(off, ids, h=None):
    """A cheap identity of a collection (or of its restriction to a value
    range): the offsets, then every FP_STRIDE-th value of every sample.
    The GPU tests check it instead of hashing every value; the full digests
    of the results already fail on any other input."""
    h = h or hashlib.sha256()
    off = np.asarray(off, dtype=np.uint64)
    h.update(np.ascontiguousarray(off, dtype="<u8").tobytes())
    for i in range(len(off) - 1):
        h.update(np.ascontiguousarray(ids[int(off[i]):int(off[i + 1])][::FP_STRIDE], dtype="<u8").tobytes())
    return h


def whole(name):
    off, ids = getattr(synth, name)()
    t0 = time.time()
    C, s, J = oracle.all_pairs(off, ids)
    secs = time.time() - t0
    return {"n": int(len(off) - 1), "values": int(off[-1]), "input_sha256": input_digest(off, ids).hexdigest(),
            "C_u32_sha256": digest(C.astype(np.uint32)), "sizes_u64_sha256": digest(s.astype(np.uint64)),
            "J_f64_sha256": digest(J.view(np.uint64)), "oracle_seconds": round(secs, 1),
            "oracle_threads": oracle.default_threads(), "oracle": "all_pairs (pairwise merge)"}


def by_rows(off, ids, lo, hi):
    Cu = oracle.rows_range(off, ids, lo, hi)
    s = oracle.sizes_of(off, ids)
    C, J = oracle.finish_upper(Cu, s)
    return C, s, J


def batched200():
    t0 = time.time()
    hin, hC, hs, hJ, hfp = (hashlib.sha256() for _ in range(5))
    per, values, samples = [], 0, 0
    for k in range(N_BATCHED):
        off, ids = synth.batched_collection(k)
        C, s, J = by_rows(off, ids, 0, 1 << 32)
        input_digest(off, ids, hin)
        fingerprint(off, ids, hfp)
        c32 = np.ascontiguousarray(C.astype("<u4"))
        hC.update(c32.tobytes())
        hs.update(np.ascontiguousarray(s, dtype="<u8").tobytes())
        hJ.update(np.ascontiguousarray(J.view(np.uint64), dtype="<u8").tobytes())
        one = hashlib.sha256()
        one.update(c32.tobytes())
        one.update(np.ascontiguousarray(s, dtype="<u8").tobytes())
        one.update(np.ascontiguousarray(J.view(np.uint64), dtype="<u8").tobytes())
        per.append(one.hexdigest()[:16])
        values += int(off[-1])
        samples += len(off) - 1
        print("  batched200 collection %d: n=%d values=%d (%.0f s)" % (k, len(off) - 1, int(off[-1]),
                                                                    time.time() - t0), flush=True)
    return {"collections": N_BATCHED, "samples": samples, "values": values,
            "input_sha256": hin.hexdigest(), "input_fingerprint_sha256": hfp.hexdigest(),
            "C_u32_sha256": hC.hexdigest(), "sizes_u64_sha256": hs.hexdigest(),
            "J_f64_sha256": hJ.hexdigest(), "per_collection_sha256_16": per,
            "oracle_seconds": round(time.time() - t0, 1), "oracle_threads": oracle.default_threads(),
            "oracle": "rows_range over [0, 2^32) per collection",
            "digest_layout": "sha256 over the collections in order of: C (uint32 n*n), sizes (uint64), J bits; "
                             "input: offsets then values per collection; per-collection: sha256(C|sizes|J)[:16]"}


def stream4096():
    t0 = time.time()
    n = 4096
    top = 1 << 40
    Cu = np.zeros((n, n), dtype=np.uint64)
    sizes = np.zeros(n, dtype=np.uint64)
    hin = hashlib.sha256()
    hfp = hashlib.sha256()
    values = 0
    cuts = [top * p // PASSES for p in range(PASSES + 1)]
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        off, ids = synth.clade4096_range(lo, hi)
        input_digest(off, ids, hin)
        fingerprint(off, ids, hfp)
        oracle.rows_range(off, ids, lo, hi, Cu)
        sizes += oracle.sizes_of(off, ids)
        values += int(off[-1])
        print("  stream4096 range [%d, %d): %d values (%.0f s)" % (lo, hi, int(off[-1]), time.time() - t0),
              flush=True)
        del off, ids
    C, J = oracle.finish_upper(Cu, sizes)
    return {"n": n, "values": values, "ranges": cuts, "input_sha256": hin.hexdigest(),
            "input_fingerprint_sha256": hfp.hexdigest(),
            "C_u64_sha256": digest(C.astype(np.uint64)), "sizes_u64_sha256": digest(sizes),
            "J_f64_sha256": digest(J.view(np.uint64)), "oracle_seconds": round(time.time() - t0, 1),
            "oracle_threads": oracle.default_threads(),
            "oracle": "rows_range per value range, added up",
            "digest_layout": "input: for each range in order, its offsets (n+1) then its values; fingerprint: "
                             "for each range in order, its offsets then every 4093rd value of every sample's "
                             "piece"}


def serve2048_q256():
    t0 = time.time()
    roff, rids = synth.serving_reference()
    qoff, qids = synth.serving_queries(0, N_QUERY)
    C, qs, J = oracle.cross(qoff, qids, roff, rids)
    rs = oracle.sizes_of(roff, rids)
    return {"n_ref": int(len(roff) - 1), "queries": N_QUERY, "ref_values": int(roff[-1]),
            "query_values": int(qoff[-1]),
            "ref_input_sha256": input_digest(roff, rids).hexdigest(),
            "query_input_sha256": input_digest(qoff, qids).hexdigest(),
            "ref_fingerprint_sha256": fingerprint(roff, rids).hexdigest(),
            "query_fingerprint_sha256": fingerprint(qoff, qids).hexdigest(),
            "C_u32_sha256": digest(C.astype(np.uint32)), "qsizes_u64_sha256": digest(qs.astype(np.uint64)),
            "ref_sizes_u64_sha256": digest(rs), "J_f64_sha256": digest(J.view(np.uint64)),
            "oracle_seconds": round(time.time() - t0, 1), "oracle_threads": oracle.default_threads(),
            "oracle": "cross (pairwise merge of every query sample with every reference sample)"}


def add_fingerprint(name):
    """Add the cheap input fingerprint to an entry computed before it existed
    (regenerates the input only; no result changes)."""
    data = json.load(open(OUT))
    e = data[name]
    h = hashlib.sha256()
    if name == "batched200":
        for k in range(e["collections"]):
            off, ids = synth.batched_collection(k)
            fingerprint(off, ids, h)
        e["input_fingerprint_sha256"] = h.hexdigest()
    elif name == "serve2048_q256":
        roff, rids = synth.serving_reference()
        qoff, qids = synth.serving_queries(0, N_QUERY)
        e["ref_fingerprint_sha256"] = fingerprint(roff, rids).hexdigest()
        e["query_fingerprint_sha256"] = fingerprint(qoff, qids).hexdigest()
    cur = json.load(open(OUT))
    cur[name] = e
    with open(OUT + ".tmp", "w") as f:
        json.dump(cur, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(OUT + ".tmp", OUT)
    print("fingerprint", name, {k: v for k, v in e.items() if "fingerprint" in k})


def check_rows():
    g = json.load(open(OUT))["clade1024"]
    off, ids = synth.clade1024()
    t0 = time.time()
    C, s, J = by_rows(off, ids, 0, 1 << 32)
    ok = (digest(C.astype(np.uint32)) == g["C_u32_sha256"] and digest(s) == g["sizes_u64_sha256"]
          and digest(J.view(np.uint64)) == g["J_f64_sha256"])
    print("check-rows clade1024: rows oracle %s the merge oracle's digests (%.0f s)"
          % ("matches" if ok else "DOES NOT MATCH", time.time() - t0))
    return ok


def main():
    names = sys.argv[1:] or ["ancestral64", "clade1024"]
    if names == ["check-rows"]:
        sys.exit(0 if check_rows() else 1)
    if names[0] == "fingerprint":
        for name in names[1:]:
            add_fingerprint(name)
        return
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data["_how"] = ("digests of the oracle's results on the seeded workloads at full size; C, sizes (uint64) and "
                    "the bit patterns of J (binary64), row-major little-endian; written by "
                    "tests/golden/make_full_size_hashes.py, which calls only the oracle")
    for name in names:
        if name in ("ancestral64", "clade1024"):
            data[name] = whole(name)
        else:
            data[name] = {"batched200": batched200, "stream4096": stream4096,
                          "serve2048_q256": serve2048_q256}[name]()
        print(name, {k: v for k, v in data[name].items() if k != "per_collection_sha256_16"}, flush=True)
        # re-read before writing: several workloads may run as separate processes
        cur = json.load(open(OUT)) if os.path.exists(OUT) else {}
        cur.update({"_how": data["_how"], name: data[name]})
        with open(OUT + ".tmp", "w") as f:
            json.dump(cur, f, indent=1, sort_keys=True)
            f.write("\n")
        os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    main()
