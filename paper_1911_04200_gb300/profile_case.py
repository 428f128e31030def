"""Small, self-contained runs for profiler captures (ncu).

Default: one collection of random packed words already in device memory, a
few calls of jsim_product with a chosen variant (a few hundred MB).
--serve: a serving index of the 2048-sample reference recipe at a reduced
median set size, and a few requests submitted one at a time (one device
batch each, nothing overlapping), so every query kernel runs alone."""
import argparse
import sys
import os

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def serve(a):
    import time
    import numpy as np
    from paper_1911_04200_gb300 import jsim, synth
    roff, rids = synth.serving_reference(median=a.median)
    qoff, qids = synth.serving_queries(0, 64, median=a.median)
    ctx = jsim.Context(id_bits=32)
    ix = jsim.Index(ctx, roff, rids, max_batch_samples=64, max_batch_values=int(qoff[-1]), slots=1)
    for k in range(a.calls):
        t0 = time.perf_counter()
        ix.submit(qoff, qids).wait()
        dt = time.perf_counter() - t0
    st = ix.stats()
    b = max(1, st["batches"])
    print("serve: index rows=%d (%.2f GB), %d batches of 64 samples, %.0f rows read/batch, query kernel %.3f ms/batch "
          "-> %.1f GB/s of index rows; last request %.1f ms" % (
              ix.rows, ix.rows * 2048 / 8 / 1e9, st["batches"], st["rows_read"] / b, st["ms_product"] / b,
              st["index_bytes_read"] / (st["ms_product"] * 1e-3) / 1e9, dt * 1e3))
    ix.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--serve", action="store_true")
    ap.add_argument("--median", type=float, default=2e4)
    ap.add_argument("--variant", default="f8")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--words", type=int, default=32768)
    ap.add_argument("--density", type=float, default=0.25)
    ap.add_argument("--calls", type=int, default=3)
    ap.add_argument("--pad", type=int, default=0, help="words of padding after every row (row stride)")
    a = ap.parse_args()
    if a.serve:
        return serve(a)
    import torch
    from paper_1911_04200_gb300 import jsim
    g = torch.Generator(device="cuda").manual_seed(7)
    # random 64-bit words with the requested bit density
    bits = torch.rand((a.n, a.words * 64), device="cuda", generator=g) < a.density if a.n * a.words <= (1 << 23) \
        else None
    if bits is not None:
        w = torch.zeros((a.n, a.words), dtype=torch.int64, device="cuda")
        for k in range(64):
            w |= bits[:, k::64].to(torch.int64) << k
    else:
        w = torch.randint(-2**63, 2**63 - 1, (a.n, a.words), dtype=torch.int64, device="cuda", generator=g)
    del bits
    stride = a.words + a.pad
    if a.pad:
        wp = torch.zeros((a.n, stride), dtype=torch.int64, device="cuda")
        wp[:, :a.words] = w
        w = wp
    ctx = jsim.Context(variant=a.variant, count_bits=32, profile=True)
    C = torch.empty((a.n, a.n), dtype=torch.uint32, device="cuda")
    for _ in range(a.calls):
        ctx.product(w, a.n, a.words, stride, C=C, variant=a.variant)
        st = ctx.stats()
    torch.cuda.synchronize()
    t = st["ms_product"]
    print("variant=%s n=%d words=%d stride=%d product %.3f ms -> %.1f Tbit-ops/s" % (
        a.variant, a.n, a.words, stride, t, st["bitops_dense"] / (t * 1e-3) / 1e12))


if __name__ == "__main__":
    main()
