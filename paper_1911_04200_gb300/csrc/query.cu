// Query kernels of the serving pattern: query samples against a resident
// reference index.
//
// The index holds the reference as one batch of the method (Sec. III-B):
// its filter f over [lo, lo + width) (Eq. 5), the rank directory of f
// (Eq. 6) and the packed words, word-major (row w = word w of every
// reference sample, so one query word reads one contiguous row).  A query
// value x can meet a reference sample only if f has row x; its rank r there
// names index word r/64, bit r%64.  Values absent from f count in |Q| only.
//
// For a batch of S query samples:
//   k_qtouch  marks the index words any query value falls in (bitmap over W);
//   rank scan of that bitmap numbers the U touched words;
//   k_qpack   builds Qc[u][s], the query's mask on touched word u;
//   k_qemit   lists the index word of every touched word;
//   k_qprod   C[s][j] = sum_u popcount(Qc[u][s] & index[w_u][j]) (Eq. 7
//             restricted to the words a query touches), reading each touched
//             index row once for the whole batch;
//   k_qepi    J = C / (|Q_s| + |S_j| - C) in binary64 (Sec. II-A).
#include <algorithm>
#include "ingest_dev.cuh"

namespace jsim {

namespace {

// Build-time tuning of the query product: index rows per tile and query
// samples per CTA (measured on GB300, 64-sample batches: 8 rows and 32
// samples - 2.32 ms per batch of 223,613 touched words - beat 4 or 16 rows
// and 8, 16 or 64 samples by 2 to 50 %).
#ifndef JSIM_QTILE
#define JSIM_QTILE 8
#endif
// query samples per CTA (the batch's samples are split over grid.z)
#ifndef JSIM_QGROUP
#define JSIM_QGROUP 32
#endif
constexpr int kQThreads = 256;
constexpr int kQCols = 2 * kQThreads;  // reference columns per CTA (two per thread)
constexpr int kQTile = JSIM_QTILE;     // index rows in flight per thread
constexpr int kQGroup = JSIM_QGROUP;   // query samples per CTA
static_assert(kQGroup >= 1 && kQGroup <= 64, "at most 64 samples per batch");

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
k_qtouch(const u64* __restrict__ ids, u64 S, Plan plan, u64 lo, u64 width, const u64* __restrict__ bm,
         const u32* __restrict__ dir, const u64* __restrict__ boff, u32* touched)
{
    __shared__ u64 s_p0, s_p1;
    const u64 nch = plan.totals[1];
    for (u64 c = blockIdx.x; c < nch; c += gridDim.x) {
        if (threadIdx.x == 0) {
            const u64 i = chunk_sample(plan.cofs, S, c);
            const u64 p0 = plan.beg[i] + (c - plan.cofs[i]) * kChunk;
            s_p0 = p0;
            s_p1 = min(p0 + kChunk, plan.beg[i] + plan.len[i]);
        }
        __syncthreads();
        const u64 p0 = s_p0, p1 = s_p1;
        for (u64 base = p0 + (threadIdx.x & ~31u); base < p1; base += kIngestThreads) {
            const u64 pos = base + (threadIdx.x & 31);
            u64 q = ~0ull, r;
            u32 bit = 0;
            if (pos < p1 && ref_rank(ids[pos], lo, width, bm, dir, boff, r)) {
                const u64 w = r >> 6;
                q = w >> 5;
                bit = 1u << (w & 31);
            }
            const bool lead = segmented_or<u32>(q, bit);
            if (lead && bit) atomicOr(touched + q, bit);
        }
        __syncthreads();
    }
}

__global__ void k_zero_dyn(u64* X, const u64* __restrict__ count, u64 per, u64 cap)
{
    const u64 total = min(*count, cap) * per;
    for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (u64)gridDim.x * blockDim.x)
        X[t] = 0ull;
}

__global__ void __launch_bounds__(kIngestThreads)
k_qpack(const u64* __restrict__ ids, u64 S, Plan plan, u64 lo, u64 width, const u64* __restrict__ bm,
        const u32* __restrict__ dir, const u64* __restrict__ boff, const u64* __restrict__ touched,
        const u32* __restrict__ dir_t, const u64* __restrict__ boff_t, u64* Qc)
{
    __shared__ u64 s_i, s_p0, s_p1;
    const u64 nch = plan.totals[1];
    for (u64 c = blockIdx.x; c < nch; c += gridDim.x) {
        if (threadIdx.x == 0) {
            const u64 i = chunk_sample(plan.cofs, S, c);
            const u64 p0 = plan.beg[i] + (c - plan.cofs[i]) * kChunk;
            s_i = i;
            s_p0 = p0;
            s_p1 = min(p0 + kChunk, plan.beg[i] + plan.len[i]);
        }
        __syncthreads();
        const u64 s = s_i, p0 = s_p0, p1 = s_p1;
        for (u64 base = p0 + (threadIdx.x & ~31u); base < p1; base += kIngestThreads) {
            const u64 pos = base + (threadIdx.x & 31);
            u64 key = ~0ull, bit = 0, r;
            if (pos < p1 && ref_rank(ids[pos], lo, width, bm, dir, boff, r)) {
                const u64 w = r >> 6, tw = w >> 6;
                const u64 u = boff_t[tw / kScanBlockWords] + (u64)dir_t[tw] +
                              (u64)__popcll(touched[tw] & ((1ull << (w & 63)) - 1ull));
                key = u * S + s;
                bit = 1ull << (r & 63);
            }
            const bool lead = segmented_or<u64>(key, bit);
            if (lead && bit) atomicOr(Qc + key, bit);
        }
        __syncthreads();
    }
}

__global__ void k_qemit(const u64* __restrict__ touched, u64 nwt, const u32* __restrict__ dir_t,
                        const u64* __restrict__ boff_t, u64* wlist)
{
    for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < nwt; t += (u64)gridDim.x * blockDim.x) {
        u64 x = touched[t];
        u64 u = boff_t[t / kScanBlockWords] + (u64)dir_t[t];
        while (x) {
            wlist[u++] = t * 64 + (u64)(__ffsll((long long)x) - 1);
            x &= x - 1;
        }
    }
}

// One CTA: reference columns [blockIdx.x * 512, +512), touched words
// [U * y / Y, U * (y + 1) / Y) and query samples [kQGroup z, +kQGroup).
// Splitting the samples over CTAs keeps the counters small, so several CTAs
// share an SM and hide the load latency; the CTAs of the sample groups read
// the same index rows at about the same time, from L2.  Counts per (query
// sample, column) live in shared memory; each thread owns two columns, so
// no two threads share a counter.  Per tile of kQTile touched words the CTA compacts each word's
// nonzero query masks into a list of (mask, sample) entries (a warp per
// word: ballot + prefix popcount), issues all index-row loads, then adds
// popcounts two entries at a time (a word's entries have distinct samples,
// so the two counter updates are independent).
__global__ void __launch_bounds__(kQThreads)
k_qprod(const u64* __restrict__ index, u64 ns, u64 n_ref, const u64* __restrict__ wlist,
        const u64* __restrict__ Udev, const u64* __restrict__ Qc, int S, u32* Cacc)
{
    extern __shared__ __align__(16) u64 q_smem[];
    uint2* cnt = (uint2*)q_smem;                   // [kQGroup][kQThreads] pairs of counters
    u64* eq = q_smem + (size_t)kQGroup * kQThreads;  // [kQTile][kQGroup] nonzero masks
    u32* es = (u32*)(eq + kQTile * kQGroup);       // [kQTile][kQGroup] their samples (within the group)
    u64* wl = (u64*)(es + kQTile * kQGroup);       // [kQTile]
    int* ne = (int*)(wl + kQTile);                 // [kQTile] entries per word
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int z0 = (int)blockIdx.z * kQGroup, G = min(kQGroup, S - z0);
    const u64 col = (u64)blockIdx.x * kQCols + 2 * (u64)t;
    const u64 U = *Udev;
    const u64 u0 = U * blockIdx.y / gridDim.y, u1 = U * (blockIdx.y + 1) / gridDim.y;
    const u32 lt = (1u << lane) - 1u;
    for (int e = t; e < G * kQThreads; e += kQThreads) cnt[e] = make_uint2(0u, 0u);
    for (u64 base = u0; base < u1; base += kQTile) {
        const int nt = (int)min((u64)kQTile, u1 - base);
        if (t < nt) wl[t] = wlist[base + t];
        for (int j = warp; j < nt; j += kQThreads / 32) {
            const u64* row = Qc + (base + j) * (u64)S + z0;
            const u64 a = lane < G ? row[lane] : 0ull;
            const u64 b = lane + 32 < G ? row[lane + 32] : 0ull;
            const u32 ba = __ballot_sync(0xffffffffu, a != 0ull), bb = __ballot_sync(0xffffffffu, b != 0ull);
            const int na = __popc(ba);
            if (a) {
                const int k = __popc(ba & lt);
                eq[j * kQGroup + k] = a;
                es[j * kQGroup + k] = (u32)lane;
            }
            if (b) {
                const int k = na + __popc(bb & lt);
                eq[j * kQGroup + k] = b;
                es[j * kQGroup + k] = (u32)lane + 32u;
            }
            if (lane == 0) ne[j] = na + __popc(bb);
        }
        __syncthreads();
        ulonglong2 r[kQTile];
        #pragma unroll
        for (int j = 0; j < kQTile; ++j)
            if (j < nt) r[j] = __ldg((const ulonglong2*)(index + wl[j] * ns + col));
        #pragma unroll
        for (int j = 0; j < kQTile; ++j) {
            if (j < nt) {
                const int m = ne[j];
                const u64* q = eq + j * kQGroup;
                const u32* sj = es + j * kQGroup;
                int k = 0;
                for (; k + 1 < m; k += 2) {
                    const u64 q0 = q[k], q1 = q[k + 1];
                    const u32 s0 = sj[k] * kQThreads + t, s1 = sj[k + 1] * kQThreads + t;
                    uint2 c0 = cnt[s0], c1 = cnt[s1];
                    c0.x += (u32)(__popcll(q0 & r[j].x));
                    c0.y += (u32)(__popcll(q0 & r[j].y));
                    c1.x += (u32)(__popcll(q1 & r[j].x));
                    c1.y += (u32)(__popcll(q1 & r[j].y));
                    cnt[s0] = c0;
                    cnt[s1] = c1;
                }
                if (k < m) {
                    const u32 s0 = sj[k] * kQThreads + t;
                    uint2 c0 = cnt[s0];
                    c0.x += (u32)(__popcll(q[k] & r[j].x));
                    c0.y += (u32)(__popcll(q[k] & r[j].y));
                    cnt[s0] = c0;
                }
            }
        }
        __syncthreads();
    }
    if (u0 >= u1) return;
    for (int s = 0; s < G; ++s) {
        const uint2 c = cnt[s * kQThreads + t];
        const u64 o = (u64)(z0 + s) * n_ref + col;
        if (c.x && col < n_ref) atomicAdd(Cacc + o, c.x);
        if (c.y && col + 1 < n_ref) atomicAdd(Cacc + o + 1, c.y);
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

cudaError_t launch_qtouch(const u64* ids, u64 S, Plan plan, u64 max_chunks, const QueryIndex& ix, u32* touched,
                          int sms, cudaStream_t st)
{
    k_qtouch<<<grid_chunks(max_chunks, sms), kIngestThreads, 0, st>>>(ids, S, plan, ix.lo, ix.width, ix.bm, ix.dir,
                                                                      ix.boff, touched);
    return cudaGetLastError();
}

cudaError_t launch_qpack(const u64* ids, u64 S, Plan plan, u64 max_chunks, const QueryIndex& ix,
                         const u64* touched, const u32* dir_t, const u64* boff_t, const u64* Udev, u64 Umax,
                         u64* Qc, int sms, cudaStream_t st)
{
    k_zero_dyn<<<grid_flat(Umax * S, sms, 256), 256, 0, st>>>(Qc, Udev, S, Umax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_qpack<<<grid_chunks(max_chunks, sms), kIngestThreads, 0, st>>>(ids, S, plan, ix.lo, ix.width, ix.bm, ix.dir,
                                                                     ix.boff, touched, dir_t, boff_t, Qc);
    return cudaGetLastError();
}

cudaError_t launch_qemit(const u64* touched, u64 nwt, const u32* dir_t, const u64* boff_t, u64* wlist, int sms,
                         cudaStream_t st)
{
    if (nwt == 0) return cudaSuccess;
    k_qemit<<<grid_flat(nwt, sms, 256), 256, 0, st>>>(touched, nwt, dir_t, boff_t, wlist);
    return cudaGetLastError();
}

size_t qprod_smem()
{
    return (size_t)kQGroup * kQThreads * sizeof(uint2) + (size_t)kQTile * kQGroup * (sizeof(u64) + sizeof(u32)) +
           kQTile * (sizeof(u64) + sizeof(int));
}

cudaError_t launch_qprod(const QueryIndex& ix, const u64* wlist, const u64* Udev, u64 Umax, const u64* Qc, int S,
                         u32* Cacc, int sms, cudaStream_t st)
{
    if (S < 1 || S > 64) return cudaErrorInvalidValue;
    if (ix.W == 0 || Umax == 0) return cudaSuccess;
    const size_t smem = qprod_smem();
    cudaError_t e = cudaFuncSetAttribute(k_qprod, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qprod, kQThreads, smem);
    if (e != cudaSuccess) return e;
    const u64 gx = ix.ns / kQCols, gz = ((u64)S + kQGroup - 1) / kQGroup;
    u64 gy = ((u64)sms * (u64)std::max(per_sm, 1) + gx * gz - 1) / (gx * gz);
    const u64 tiles = (Umax + kQTile - 1) / kQTile;
    if (gy > tiles) gy = tiles;
    if (gy > 65535) gy = 65535;
    if (gy == 0) gy = 1;
    k_qprod<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), kQThreads, smem, st>>>(ix.index, ix.ns, ix.n_ref,
                                                                                    wlist, Udev, Qc, S, Cacc);
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
