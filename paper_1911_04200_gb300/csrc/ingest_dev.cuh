// Device helpers shared by the ingest and query kernels (internal).
#pragma once
#include "common.cuh"

namespace jsim {

namespace {

constexpr int kPlanThreads = 1024;
constexpr int kIngestThreads = 256;
constexpr int kScanThreads = 256;

__device__ __forceinline__ u64 lower_bound_u64(const u64* a, u64 lo, u64 hi, u64 v)
{
    while (lo < hi) {
        u64 mid = lo + ((hi - lo) >> 1);
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Block-wide exclusive scan of one u64 per thread; returns the block total.
template <int NT>
__device__ __forceinline__ u64 block_exclusive_scan(u64 v, u64& excl, u64* smem /* NT/32 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64 x = v;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u64 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        u64 w = lane < NT / 32 ? smem[lane] : 0;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            u64 y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) smem[lane] = w;
    }
    __syncthreads();
    u64 warp_base = warp ? smem[warp - 1] : 0;
    u64 total = smem[NT / 32 - 1];
    excl = warp_base + x - v;
    __syncthreads();
    return total;
}

// The next chunk of a plan for the calling CTA: a ticket from the plan's
// counter `which` (zeroed by the plan), so the chunks go, in order, to
// whichever CTAs are resident - a launch that shares the GPU with another
// kernel is not held up by CTAs that start late with a fixed share of work.
__device__ __forceinline__ u64 next_chunk(const Plan& plan, int which)
{
    return atomicAdd((unsigned long long*)(plan.totals + which), 1ull);
}

// Chunk c -> sample index (largest i with cofs[i] <= c, among samples with chunks).
__device__ __forceinline__ u64 chunk_sample(const u64* cofs, u64 n, u64 c)
{
    u64 lo = 0, hi = n;  // find last i in [0,n) with cofs[i] <= c
    while (lo < hi) {
        u64 mid = lo + ((hi - lo + 1) >> 1);
        if (cofs[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One chunk of a plan: ticket c (c >= the plan's chunk count: none left),
// sample i, its values [p0, p1) and the sample's first batch value b.
struct ChunkDesc {
    u64 c, i, p0, p1, b;
};

// Take the next ticket of counter `which` and describe its chunk (one thread).
// The ticket kernels keep two descriptors in shared memory: thread 0 takes
// the next chunk's ticket and finds its sample while the CTA works on the
// current chunk, so the ticket's round trip and the search do not stall it.
__device__ __forceinline__ void fetch_chunk(const Plan& plan, u64 n, u64 nch, int which, ChunkDesc& d)
{
    const u64 c = next_chunk(plan, which);
    d.c = c;
    if (c < nch) {
        const u64 i = chunk_sample(plan.cofs, n, c);
        const u64 b = plan.beg[i], p0 = b + (c - plan.cofs[i]) * kChunk;
        d.i = i;
        d.b = b;
        d.p0 = p0;
        d.p1 = min(p0 + kChunk, b + plan.len[i]);
    }
}

// Inclusive OR over the lanes that share key q, accumulated toward the
// segment's first lane (q is non-decreasing across lanes).  Returns true on
// the lane that must publish the segment's value.
template <typename T>
__device__ __forceinline__ bool segmented_or(u64 q, T& v)
{
    const int lane = threadIdx.x & 31;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T w = __shfl_down_sync(0xffffffffu, v, o);
        u64 qq = __shfl_down_sync(0xffffffffu, q, o);
        if (lane + o < 32 && qq == q) v |= w;
    }
    u64 qprev = __shfl_up_sync(0xffffffffu, q, 1);
    return lane == 0 || qprev != q;
}

}  // namespace

}  // namespace jsim
