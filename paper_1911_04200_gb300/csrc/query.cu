// Query kernels of the serving pattern: query samples against a resident
// reference index.
//
// The index holds the reference as one batch of the method (Sec. III-B):
// its filter f over [lo, lo + width) (Eq. 5), the rank directory of f
// (Eq. 6), and the rows of Abar_ref (Eq. 6): row r, the r-th kept row, is an
// n_ref-bit vector of the reference samples that hold it, stored as
// ns64 = ceil(n_ref / 64) words (rank-major).  A query value x meets a
// reference sample only if f has row x, and then exactly the samples of row
// rank(x); values absent from f count in |Q| only.  So for a query sample s
//   C[s][j] = sum over x in Q_s with f(x) of Abar_ref[rank(x)][j]
// (Eq. 7 with the query's 0/1 column), read as one row of ns64 words per
// query value.
//
//   k_pack_rows  (build) sets bit j of row rank(x) for every value x of
//                reference sample j;
//   k_qrows      a warp per chunk of one query sample's values: lanes rank
//                32 values at a time, then every lane adds its words of the
//                ranked rows into bit-sliced counters held in registers
//                (plane k = bit k of 64 column counts); at the end of the
//                chunk the counts go into C with atomic adds;
//   k_qepi       J = C / (|Q_s| + |S_j| - C) in binary64 (Sec. II-A).
#include <algorithm>
#include "ingest_dev.cuh"

namespace jsim {

namespace {

constexpr int kQThreads = 256;
constexpr int kQWarps = kQThreads / 32;
constexpr int kPlanes = 13;   // counts of one chunk (<= kChunk = 4096 values) fit 13 bits
static_assert((1ull << (kPlanes - 1)) >= kChunk, "bit planes hold a chunk's counts");
// Build-time tuning: rows in flight per lane (JSIM_QBATCH).
#ifndef JSIM_QBATCH
#define JSIM_QBATCH 8
#endif
constexpr int kQBatch = JSIM_QBATCH;

// rank of x in the reference filter, if f has row x
__device__ __forceinline__ bool ref_rank(u64 x, u64 lo, u64 width, const u64* __restrict__ bm,
                                         const u32* __restrict__ dir, const u64* __restrict__ boff, u64& r)
{
    const u64 d = x - lo;
    if (d >= width) return false;
    const u64 w = d >> 6;
    const u64 word = bm[w];
    const u64 bit = 1ull << (d & 63);
    if (!(word & bit)) return false;
    r = boff[w / kScanBlockWords] + (u64)dir[w] + (u64)__popcll(word & (bit - 1ull));
    return true;
}

__global__ void __launch_bounds__(kIngestThreads)
k_pack_rows(const u64* __restrict__ ids, u64 n, Plan plan, u64 lo, u64 width, const u64* __restrict__ bm,
            const u32* __restrict__ dir, const u64* __restrict__ boff, u64* Xt, u64 ns64)
{
    __shared__ u64 s_i, s_p0, s_p1;
    const u64 nch = plan.totals[1];
    for (u64 c = blockIdx.x; c < nch; c += gridDim.x) {
        if (threadIdx.x == 0) {
            const u64 i = chunk_sample(plan.cofs, n, c);
            const u64 p0 = plan.beg[i] + (c - plan.cofs[i]) * kChunk;
            s_i = i;
            s_p0 = p0;
            s_p1 = min(p0 + kChunk, plan.beg[i] + plan.len[i]);
        }
        __syncthreads();
        const u64 i = s_i, p0 = s_p0, p1 = s_p1;
        for (u64 pos = p0 + threadIdx.x; pos < p1; pos += kIngestThreads) {
            u64 r;
            if (ref_rank(ids[pos], lo, width, bm, dir, boff, r))
                atomicOr(Xt + r * ns64 + (i >> 6), 1ull << (i & 63));
        }
        __syncthreads();
    }
}

// add the bits of v into the bit-sliced counters p (carry ripple)
__device__ __forceinline__ void bs_add(u64 (&p)[kPlanes], u64 v)
{
    #pragma unroll
    for (int k = 0; k < kPlanes; ++k) {
        if (!v) break;
        const u64 t = p[k] & v;
        p[k] ^= v;
        v = t;
    }
}

template <int KW>
__global__ void __launch_bounds__(kQThreads)
k_qrows(const u64* __restrict__ ids, u64 S, Plan plan, u64 lo, u64 width, const u64* __restrict__ bm,
        const u32* __restrict__ dir, const u64* __restrict__ boff, const u64* __restrict__ Xt, u64 ns64, u64 n_ref,
        u32* Cacc, u64* rows_read, u32 nsub)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // work item: part `part` (of nsub) of plan chunk c, so that small
    // batches still spread over every SM
    const u64 items = plan.totals[1] * nsub;
    const u64 sub = kChunk / nsub;
    for (u64 it = (u64)blockIdx.x * kQWarps + warp; it < items; it += (u64)gridDim.x * kQWarps) {
        const u64 c = it / nsub, part = it - c * nsub;
        const u64 s = chunk_sample(plan.cofs, S, c);
        const u64 sb = plan.beg[s], se = sb + plan.len[s];
        const u64 p0 = sb + (c - plan.cofs[s]) * kChunk + part * sub;
        if (p0 >= se) continue;
        const u64 p1 = min(p0 + sub, se);
        u64 pl[KW][kPlanes];
        #pragma unroll
        for (int k = 0; k < KW; ++k)
            #pragma unroll
            for (int q = 0; q < kPlanes; ++q) pl[k][q] = 0ull;
        u32 found = 0;
        for (u64 base = p0; base < p1; base += 32) {
            const u64 pos = base + lane;
            u64 r = 0;
            bool ok = false;
            if (pos < p1) {
                const u64 x = ids[pos];
                // a repeated value of the sample is one element of the set
                ok = !(pos > sb && ids[pos - 1] == x) && ref_rank(x, lo, width, bm, dir, boff, r);
            }
            unsigned vm = __ballot_sync(0xffffffffu, ok);
            found += (u32)__popc(vm);
            while (vm) {
                u64 rr[kQBatch];
                int cnt = 0;
                #pragma unroll
                for (int g = 0; g < kQBatch; ++g) {
                    const int src = vm ? __ffs((int)vm) - 1 : 0;
                    rr[g] = __shfl_sync(0xffffffffu, r, src);
                    if (vm) { vm &= vm - 1; ++cnt; }
                }
                u64 v[kQBatch][KW];
                #pragma unroll
                for (int g = 0; g < kQBatch; ++g)
                    #pragma unroll
                    for (int k = 0; k < KW; ++k) {
                        const u64 w = (u64)lane + 32ull * k;
                        v[g][k] = (g < cnt && w < ns64) ? __ldg(Xt + rr[g] * ns64 + w) : 0ull;
                    }
                #pragma unroll
                for (int g = 0; g < kQBatch; ++g)
                    #pragma unroll
                    for (int k = 0; k < KW; ++k) bs_add(pl[k], v[g][k]);
            }
        }
        // counts of this chunk into C
        #pragma unroll
        for (int k = 0; k < KW; ++k) {
            const u64 w = (u64)lane + 32ull * k;
            if (w >= ns64) continue;
            u64 any = 0ull;
            #pragma unroll
            for (int q = 0; q < kPlanes; ++q) any |= pl[k][q];
            while (any) {
                const int b = __ffsll((long long)any) - 1;
                any &= any - 1;
                u32 cntb = 0;
                #pragma unroll
                for (int q = 0; q < kPlanes; ++q) cntb |= (u32)((pl[k][q] >> b) & 1ull) << q;
                const u64 col = w * 64 + (u64)b;
                if (col < n_ref) atomicAdd(Cacc + s * n_ref + col, cntb);
            }
        }
        if (lane == 0 && found) atomicAdd(rows_read, (u64)found);
    }
}

template <typename CT>
__global__ void k_qepi(const u32* __restrict__ Cacc, u64 S, u64 n_ref, const u64* __restrict__ sq,
                       const u64* __restrict__ sr, CT* Cout, double* J)
{
    const u64 total = S * n_ref;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (u64)gridDim.x * blockDim.x) {
        const u64 s = e / n_ref, j = e - s * n_ref;
        const u64 c = Cacc[e];
        const u64 u = sq[s] + sr[j] - c;
        if (Cout) Cout[e] = (CT)c;
        if (J) J[e] = u ? __ddiv_rn(__ull2double_rn(c), __ull2double_rn(u)) : 1.0;
    }
}

inline unsigned grid_chunks(u64 max_chunks, int sms)
{
    u64 g = (u64)sms * 8;
    if (max_chunks < g) g = max_chunks;
    return (unsigned)(g ? g : 1);
}

inline unsigned grid_flat(u64 total, int sms, int threads)
{
    u64 g = (total + threads - 1) / threads;
    const u64 cap = (u64)sms * 8;
    if (g > cap) g = cap;
    return (unsigned)(g ? g : 1);
}

}  // namespace

cudaError_t launch_pack_rows(const u64* ids, u64 n, Plan plan, u64 max_chunks, const QueryIndex& ix, u64* Xt,
                             int sms, cudaStream_t st)
{
    k_pack_rows<<<grid_chunks(max_chunks, sms), kIngestThreads, 0, st>>>(ids, n, plan, ix.lo, ix.width, ix.bm, ix.dir,
                                                                         ix.boff, Xt, ix.ns64);
    return cudaGetLastError();
}

cudaError_t launch_qrows(const u64* ids, u64 S, Plan plan, u64 max_chunks, const QueryIndex& ix, u32* Cacc,
                         u64* rows_read, int sms, cudaStream_t st)
{
    if (ix.R == 0) return cudaSuccess;
    // split chunks into up to 8 parts while the batch gives fewer than about
    // 32 warps per SM
    u32 nsub = 1;
    while (nsub < 8 && max_chunks * nsub < (u64)sms * 32) nsub <<= 1;
    const u64 items = max_chunks * nsub;
    const u64 blocks = std::max<u64>(1, std::min<u64>((items + kQWarps - 1) / kQWarps, (u64)sms * 8));
    if (ix.ns64 <= 32)
        k_qrows<1><<<(unsigned)blocks, kQThreads, 0, st>>>(ids, S, plan, ix.lo, ix.width, ix.bm, ix.dir, ix.boff,
                                                           ix.index, ix.ns64, ix.n_ref, Cacc, rows_read, nsub);
    else if (ix.ns64 <= 64)
        k_qrows<2><<<(unsigned)blocks, kQThreads, 0, st>>>(ids, S, plan, ix.lo, ix.width, ix.bm, ix.dir, ix.boff,
                                                           ix.index, ix.ns64, ix.n_ref, Cacc, rows_read, nsub);
    else if (ix.ns64 <= 128)
        k_qrows<4><<<(unsigned)blocks, kQThreads, 0, st>>>(ids, S, plan, ix.lo, ix.width, ix.bm, ix.dir, ix.boff,
                                                           ix.index, ix.ns64, ix.n_ref, Cacc, rows_read, nsub);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_qepi(const u32* Cacc, u64 S, u64 n_ref, const u64* sq, const u64* sr, int count_bits, void* Cout,
                        double* J, int sms, cudaStream_t st)
{
    const unsigned g = grid_flat(S * n_ref, sms, 256);
    if (count_bits == 64)
        k_qepi<u64><<<g, 256, 0, st>>>(Cacc, S, n_ref, sq, sr, (u64*)Cout, J);
    else
        k_qepi<u32><<<g, 256, 0, st>>>(Cacc, S, n_ref, sq, sr, (u32*)Cout, J);
    return cudaGetLastError();
}

}  // namespace jsim
