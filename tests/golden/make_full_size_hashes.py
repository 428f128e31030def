"""Write tests/golden/full_size_sha256.json: SHA-256 digests of the oracle's
results (C as uint32, sizes as uint64, J as binary64 bit patterns, all
row-major little-endian) for workloads at their full size, together with a
digest of the generated input.  Calls only the oracle and the seeded input
generator; run it once on any machine (the generator draws identical sets on
x86-64 and AArch64):

    python tests/golden/make_full_size_hashes.py [workload ...]

Workloads: ancestral64 (64 samples, 3.1e6 values: seconds) and clade1024
(1024 samples, 1.3e9 values: minutes of all host cores, 11 GB of memory).
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


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes()).hexdigest()


def input_digest(off, ids):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(off, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(ids, dtype="<u8").tobytes())
    return h.hexdigest()


def run(name):
    off, ids = getattr(synth, name)()
    t0 = time.time()
    C, s, J = oracle.all_pairs(off, ids)
    secs = time.time() - t0
    return {"n": int(len(off) - 1), "values": int(off[-1]), "input_sha256": input_digest(off, ids),
            "C_u32_sha256": digest(C.astype(np.uint32)), "sizes_u64_sha256": digest(s.astype(np.uint64)),
            "J_f64_sha256": digest(J.view(np.uint64)), "oracle_seconds": round(secs, 1),
            "oracle_threads": oracle.default_threads()}


def main():
    names = sys.argv[1:] or ["ancestral64", "clade1024"]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data["_how"] = ("oracle.all_pairs on the seeded workload at full size; digests of C (uint32), sizes "
                    "(uint64) and the bit patterns of J (binary64), row-major little-endian; written by "
                    "tests/golden/make_full_size_hashes.py")
    for name in names:
        data[name] = run(name)
        print(name, data[name], flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main()
