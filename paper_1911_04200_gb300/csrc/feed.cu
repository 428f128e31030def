// Device side of the piece-by-piece copy of page-locked host input (the
// feed of the plain all-pairs call).  The GPU reads the host's values
// through their device-mapped address, over the NVLink-C2C link: per piece,
// one CTA finds where every sample's values reach the piece's upper boundary
// (a binary search in host memory), and a small grid copies every sample's
// slice to the same place in device memory.  A few dozen CTAs keep the link
// busy (about 211 GB/s on GB300, the rate of one large DMA copy), where a
// DMA copy per slice is bound by the cost of issuing it (about 6 us per copy
// of 1 MiB).
#include "ingest_dev.cuh"

namespace jsim {

namespace {

constexpr int kCutThreads = 256;
constexpr int kGatherThreads = 256;

// Sample i's piece is [c0[i], c1[i]): c1[i] is the first position in
// [c0[i], off[i + 1]) whose value is >= bound (every position to the end for
// the last piece); pre: exclusive prefix of the slice lengths, pre[n] their
// total.  One CTA.
__global__ void __launch_bounds__(kCutThreads)
k_feed_cuts(const u64* __restrict__ hv, const u64* __restrict__ off, u64 n, const u64* __restrict__ c0,
            u64* __restrict__ c1, u64 bound, int last, u64* __restrict__ pre)
{
    __shared__ u64 sm[kCutThreads / 32];
    u64 carry = 0;
    for (u64 base = 0; base < n; base += kCutThreads) {
        const u64 i = base + threadIdx.x;
        u64 len = 0;
        if (i < n) {
            const u64 a = c0[i], e = off[i + 1];
            const u64 q = last ? e : lower_bound_u64(hv, a, e, bound);
            c1[i] = q;
            len = q - a;
        }
        u64 ex;
        const u64 tot = block_exclusive_scan<kCutThreads>(len, ex, sm);
        if (i < n) pre[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) pre[n] = carry;
}

// The piece's values in slice order (sample 0's slice, then sample 1's, ...)
// are cut into gridDim.x equal ranges; CTA b copies range b, 16 bytes per
// lane where the host and device addresses share their offset within 16
// bytes (else 8).  Loads and stores are marked streaming (evict first): the
// batch loop running beside the copy keeps its class structures and the
// product its shared panels in L2, which a gigabyte piece passing through
// would otherwise evict.
// At most 32 registers a thread (8 CTAs an SM), so a copy CTA takes no more
// of an SM than one ingest CTA, and one fits beside a tensor-core product CTA.
__global__ void __launch_bounds__(kGatherThreads, 8)
k_feed_gather(const u64* __restrict__ hv, u64* __restrict__ dv, const u64* __restrict__ c0,
              const u64* __restrict__ pre, u64 n)
{
    const u64 total = pre[n];
    const u64 r0 = total * blockIdx.x / gridDim.x, r1 = total * (blockIdx.x + 1) / gridDim.x;
    if (r0 >= r1) return;
    const bool vec = ((((uintptr_t)hv ^ (uintptr_t)dv) & 15) == 0) && (((uintptr_t)hv & 7) == 0);
    const unsigned t = threadIdx.x, nt = blockDim.x;
    u64 i = chunk_sample(pre, n, r0);  // the last sample whose slice starts at or before r0
    u64 p = r0;
    while (p < r1 && i < n) {
        const u64 e_rel = pre[i + 1] < r1 ? pre[i + 1] : r1;
        if (e_rel > p) {
            u64 a = c0[i] + (p - pre[i]), e = c0[i] + (e_rel - pre[i]);
            if (vec) {
                if ((((uintptr_t)(hv + a)) & 15) != 0) {
                    if (t == 0) __stcs(dv + a, __ldcs(hv + a));
                    ++a;
                }
                if (a < e && ((e - a) & 1)) {
                    if (t == 0) __stcs(dv + e - 1, __ldcs(hv + e - 1));
                    --e;
                }
                const uint4* s4 = reinterpret_cast<const uint4*>(hv + a);
                uint4* d4 = reinterpret_cast<uint4*>(dv + a);
                const u64 m = a < e ? (e - a) / 2 : 0;
                u64 k = t;
                for (; k + nt < m; k += 2 * (u64)nt) {
                    const uint4 x = __ldcs(s4 + k), y = __ldcs(s4 + k + nt);
                    __stcs(d4 + k, x);
                    __stcs(d4 + k + nt, y);
                }
                if (k < m) __stcs(d4 + k, __ldcs(s4 + k));
            } else {
                for (u64 k = a + t; k < e; k += nt) __stcs(dv + k, __ldcs(hv + k));
            }
            p = e_rel;
        }
        ++i;
    }
}

}  // namespace

cudaError_t launch_feed_piece(const u64* hv, u64* dv, const u64* off, u64 n, const u64* c0, u64* c1, u64 bound,
                              bool last, u64* pre, int grid, cudaStream_t st)
{
    k_feed_cuts<<<1, kCutThreads, 0, st>>>(hv, off, n, c0, c1, bound, last ? 1 : 0, pre);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_feed_gather<<<grid, kGatherThreads, 0, st>>>(hv, dv, c0, pre, n);
    return cudaGetLastError();
}

}  // namespace jsim
