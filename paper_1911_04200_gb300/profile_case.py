"""Small, self-contained product runs for profiler captures (ncu): one
collection of random packed words already in device memory, a few calls of
jsim_product with a chosen variant.  Sizes stay small (a few hundred MB)."""
import argparse
import sys
import os

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--variant", default="f8")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--words", type=int, default=32768)
    ap.add_argument("--density", type=float, default=0.25)
    ap.add_argument("--calls", type=int, default=3)
    a = ap.parse_args()
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
    ctx = jsim.Context(variant=a.variant, count_bits=32, profile=True)
    C = torch.empty((a.n, a.n), dtype=torch.uint32, device="cuda")
    for _ in range(a.calls):
        ctx.product(w, a.n, a.words, a.words, C=C, variant=a.variant)
        st = ctx.stats()
    torch.cuda.synchronize()
    t = st["ms_product"]
    print("variant=%s n=%d words=%d product %.3f ms -> %.1f Tbit-ops/s" % (
        a.variant, a.n, a.words, t, st["bitops_dense"] / (t * 1e-3) / 1e12))


if __name__ == "__main__":
    main()
