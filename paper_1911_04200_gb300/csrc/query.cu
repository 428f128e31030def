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
//   k_rank_words (build) the query-side filter: per filter word one 16-byte
//                entry (word, rank of its first bit), so a rank is one load;
//   k_qrows      one wave of resident warps, warp w taking the w-th equal
//                range of the batch's values: rounds of 128 values are
//                ranked (coalesced values, one entry load each) into a list
//                in shared memory, then every lane streams its words of the
//                listed rows, two batches of 8 rows in flight, into
//                bit-sliced counters in registers (plane k = bit k of 64
//                column counts) through a carry-save adder tree; at the end
//                of a sample (or 4096 values) the counts go into C with
//                atomic adds;
//   k_qepi       J = C / (|Q_s| + |S_j| - C) in binary64 (Sec. II-A), or
//                the distance 1.0 - J.
#include <algorithm>
#include <atomic>
#include "ingest_dev.cuh"

namespace jsim {

namespace {

// Build-time tuning: threads per query block (JSIM_QTHREADS), values ranked
// per warp round (JSIM_QROUND), rows in flight per lane (JSIM_QBATCH, per
// batch of two), blocks per SM the one-word kernel is held to (JSIM_QMINB).
#ifndef JSIM_QTHREADS
#define JSIM_QTHREADS 128
#endif
#ifndef JSIM_QROUND
#define JSIM_QROUND 128
#endif
#ifndef JSIM_QMINB
#define JSIM_QMINB 6
#endif
constexpr int kQThreads = JSIM_QTHREADS;
constexpr int kQWarps = kQThreads / 32;
constexpr int kPlanes = 13;   // counts of one chunk (<= kChunk = 4096 values) fit 13 bits
static_assert((1ull << (kPlanes - 1)) >= kChunk, "bit planes hold a chunk's counts");
#ifndef JSIM_QBATCH
#define JSIM_QBATCH 8
#endif
constexpr int kQBatch = JSIM_QBATCH;
constexpr int kQRound = JSIM_QROUND;
static_assert(kQRound % 32 == 0 && kQRound <= kChunk, "a round is whole warp groups");

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

// add v * 2^k0 into the bit-sliced counters p (carry ripple from plane k0)
template <int K0 = 0>
__device__ __forceinline__ void bs_add(u64 (&p)[kPlanes], u64 v)
{
    #pragma unroll
    for (int k = K0; k < kPlanes; ++k) {
        if (!v) break;
        const u64 t = p[k] & v;
        p[k] ^= v;
        v = t;
    }
}

// carry-save adder: a + b + c = l + 2 h per bit (a becomes l)
__device__ __forceinline__ u64 csa(u64& a, u64 b, u64 c)
{
    const u64 u = a ^ b;
    const u64 h = (a & b) | (u & c);
    a = u ^ c;
    return h;
}

// add D words (D = 2, 4 or 8) into the counters: a carry-save tree on the
// low planes, one carry ripple from plane log2(D) for the whole batch
template <int D>
__device__ __forceinline__ void bs_add_batch(u64 (&p)[kPlanes], const u64 (&v)[D])
{
    static_assert(D == 2 || D == 4 || D == 8, "batch of 2, 4 or 8 words");
    if constexpr (D == 2) {
        bs_add<1>(p, csa(p[0], v[0], v[1]));
    } else if constexpr (D == 4) {
        const u64 t1 = csa(p[0], v[0], v[1]);
        const u64 t2 = csa(p[0], v[2], v[3]);
        bs_add<2>(p, csa(p[1], t1, t2));
    } else {
        u64 t1 = csa(p[0], v[0], v[1]);
        u64 t2 = csa(p[0], v[2], v[3]);
        const u64 f1 = csa(p[1], t1, t2);
        t1 = csa(p[0], v[4], v[5]);
        t2 = csa(p[0], v[6], v[7]);
        const u64 f2 = csa(p[1], t1, t2);
        bs_add<3>(p, csa(p[2], f1, f2));
    }
}

// fr[w] = (word w of f, rank of its first bit): one 16-byte entry per filter
// word, so that a query value's rank is one load
__global__ void k_rank_words(const u64* __restrict__ bm, const u32* __restrict__ dir, const u64* __restrict__ boff,
                             u64 nw, ulonglong2* __restrict__ fr)
{
    for (u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (u64)gridDim.x * blockDim.x)
        fr[w] = make_ulonglong2(bm[w], boff[w / kScanBlockWords] + (u64)dir[w]);
}

// rows of one load batch in flight per lane, two batches at a time
template <int KW>
struct QRowBatch {
    static constexpr int D = kQBatch / KW > 1 ? kQBatch / KW : 2;
    static_assert(D == 2 || D == 4 || D == 8, "row batches of 2, 4 or 8");
};

template <int KW>
__global__ void __launch_bounds__(kQThreads, KW == 1 ? JSIM_QMINB : 1)
k_qrows(const u64* __restrict__ ids, u64 S, Plan plan, u64 lo, u64 width, const ulonglong2* __restrict__ fr,
        const u64* __restrict__ Xt, u64 ns64, u64 n_ref, u32* Cacc, u64* rows_read)
{
    constexpr int D = QRowBatch<KW>::D;
    __shared__ u64 rk_s[kQWarps][kQRound];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64* rk = rk_s[warp];
    const unsigned lt = (1u << lane) - 1u;
    // The batch's samples lie back to back from beg[0]; warp w of W takes
    // the w-th of W equal ranges of their T values, in segments that stay
    // inside one sample and hold at most kChunk values (so that a count fits
    // the planes).
    const u64 T = plan.totals[0];
    if (S == 0 || T == 0) return;
    const u64 W = (u64)gridDim.x * kQWarps, wid = (u64)blockIdx.x * kQWarps + warp;
    const u64 P0 = plan.beg[0];
    u64 pos = P0 + T * wid / W;
    const u64 end = P0 + T * (wid + 1) / W;
    u64 s = 0;
    {   // last sample that starts at or before pos
        u64 a = 0, b = S - 1;
        while (a < b) {
            const u64 m = a + ((b - a + 1) >> 1);
            if (plan.beg[m] <= pos) a = m; else b = m - 1;
        }
        s = a;
    }
    while (pos < end) {
        while (s + 1 < S && pos >= plan.beg[s] + plan.len[s]) ++s;  // empty or finished samples
        if (pos >= plan.beg[s] + plan.len[s]) break;
        const u64 sb = plan.beg[s];
        const u64 p1 = min(min(end, sb + plan.len[s]), pos + kChunk);
        const u64 p0 = pos;
        pos = p1;
        u64 pl[KW][kPlanes];
        #pragma unroll
        for (int k = 0; k < KW; ++k)
            #pragma unroll
            for (int q = 0; q < kPlanes; ++q) pl[k][q] = 0ull;
        u32 found = 0;
        for (u64 base = p0; base < p1; base += kQRound) {
            // rank phase: kQRound values, kQRound / 32 per lane (coalesced),
            // every rank one 16-byte load; the found ranks go to rk in order
            u64 x[kQRound / 32];
            bool live[kQRound / 32];
            #pragma unroll
            for (int g = 0; g < kQRound / 32; ++g) {
                const u64 q = base + (u64)(g * 32 + lane);
                live[g] = false;
                x[g] = 0;
                if (q < p1) {
                    x[g] = ids[q];
                    // a repeated value of the sample is one element of the set
                    live[g] = !(q > sb && ids[q - 1] == x[g]) && (x[g] - lo) < width;
                }
            }
            ulonglong2 e[kQRound / 32];
            #pragma unroll
            for (int g = 0; g < kQRound / 32; ++g)
                e[g] = live[g] ? __ldg(fr + ((x[g] - lo) >> 6)) : make_ulonglong2(0ull, 0ull);
            int cnt = 0;
            #pragma unroll
            for (int g = 0; g < kQRound / 32; ++g) {
                const u64 bit = 1ull << ((x[g] - lo) & 63);
                const bool ok = (e[g].x & bit) != 0;
                const unsigned m = __ballot_sync(0xffffffffu, ok);
                if (ok) rk[cnt + __popc(m & lt)] = e[g].y + (u64)__popcll(e[g].x & (bit - 1ull));
                cnt += __popc(m);
            }
            __syncwarp();
            found += (u32)cnt;
            // row phase: every lane adds its words of the cnt rows; batch b+1
            // is loaded while batch b is added
            u64 va[D][KW], vb[D][KW];
            auto load = [&](u64 (&v)[D][KW], int i) {
                #pragma unroll
                for (int g = 0; g < D; ++g) {
                    const bool in = i + g < cnt;
                    const u64* row = Xt + (in ? rk[i + g] : 0ull) * ns64;
                    #pragma unroll
                    for (int k = 0; k < KW; ++k) {
                        const u64 w = (u64)lane + 32ull * k;
                        v[g][k] = (in && w < ns64) ? __ldg(row + w) : 0ull;
                    }
                }
            };
            auto add = [&](u64 (&v)[D][KW]) {
                #pragma unroll
                for (int k = 0; k < KW; ++k) {
                    u64 col[D];
                    #pragma unroll
                    for (int g = 0; g < D; ++g) col[g] = v[g][k];
                    bs_add_batch<D>(pl[k], col);
                }
            };
            load(va, 0);
            for (int i = 0; i < cnt; i += 2 * D) {
                load(vb, i + D);
                add(va);
                load(va, i + 2 * D);
                add(vb);
            }
            __syncwarp();  // rk is rewritten by the next round
        }
        // counts of this segment into C
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
                       const u64* __restrict__ sr, CT* Cout, double* J, int distance)
{
    const u64 total = S * n_ref;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (u64)gridDim.x * blockDim.x) {
        const u64 s = e / n_ref, j = e - s * n_ref;
        const u64 c = Cacc[e];
        const u64 u = sq[s] + sr[j] - c;
        if (Cout) Cout[e] = (CT)c;
        if (J) {
            const double s = u ? __ddiv_rn(__ull2double_rn(c), __ull2double_rn(u)) : 1.0;
            J[e] = distance ? __dsub_rn(1.0, s) : s;
        }
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

cudaError_t launch_rank_words(const QueryIndex& ix, ulonglong2* fr, int sms, cudaStream_t st)
{
    const u64 nw = ix.width / 64;
    if (nw == 0) return cudaSuccess;
    k_rank_words<<<grid_flat(nw, sms, 256), 256, 0, st>>>(ix.bm, ix.dir, ix.boff, nw, fr);
    return cudaGetLastError();
}

template <int KW>
cudaError_t launch_qrows_kw(const u64* ids, u64 S, Plan plan, u64 values, const QueryIndex& ix, u32* Cacc,
                            u64* rows_read, int sms, cudaStream_t st)
{
    // one wave of resident blocks, fewer when the batch gives a warp less
    // than two rounds of values
    int dev = 0;
    cudaGetDevice(&dev);
    static std::atomic<int> per_sm_by_dev[kMaxDevices];
    int per_sm = dev < kMaxDevices ? per_sm_by_dev[dev].load(std::memory_order_relaxed) : 0;
    if (!per_sm) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qrows<KW>, kQThreads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        if (dev < kMaxDevices) per_sm_by_dev[dev].store(per_sm, std::memory_order_relaxed);
    }
    const u64 want = (values + 2 * kQRound * kQWarps - 1) / (2 * kQRound * kQWarps);
    const u64 blocks = std::max<u64>(1, std::min<u64>(want, (u64)sms * per_sm));
    k_qrows<KW><<<(unsigned)blocks, kQThreads, 0, st>>>(ids, S, plan, ix.lo, ix.width, ix.fr, ix.index, ix.ns64,
                                                        ix.n_ref, Cacc, rows_read);
    return cudaGetLastError();
}

cudaError_t launch_qrows(const u64* ids, u64 S, Plan plan, u64 values, const QueryIndex& ix, u32* Cacc,
                         u64* rows_read, int sms, cudaStream_t st)
{
    if (ix.R == 0 || S == 0 || values == 0) return cudaSuccess;
    if (ix.ns64 <= 32) return launch_qrows_kw<1>(ids, S, plan, values, ix, Cacc, rows_read, sms, st);
    if (ix.ns64 <= 64) return launch_qrows_kw<2>(ids, S, plan, values, ix, Cacc, rows_read, sms, st);
    if (ix.ns64 <= 128) return launch_qrows_kw<4>(ids, S, plan, values, ix, Cacc, rows_read, sms, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_qepi(const u32* Cacc, u64 S, u64 n_ref, const u64* sq, const u64* sr, int count_bits, void* Cout,
                        double* J, int sms, cudaStream_t st, int distance)
{
    const unsigned g = grid_flat(S * n_ref, sms, 256);
    if (count_bits == 64)
        k_qepi<u64><<<g, 256, 0, st>>>(Cacc, S, n_ref, sq, sr, (u64*)Cout, J, distance);
    else
        k_qepi<u32><<<g, 256, 0, st>>>(Cacc, S, n_ref, sq, sr, (u32*)Cout, J, distance);
    return cudaGetLastError();
}

}  // namespace jsim
