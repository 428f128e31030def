// Windowed construction of the block-sparse path's row classes and class
// matrices: the filter f^(l) of every tile of samples (Eq. 5), the class
// ranks (Eq. 6) and the bitmask compression (Sec. III-B), built range by
// range in shared memory.
//
// A row batch [lo, lo + m) is cut into windows of 2^wl rows and the windows
// into ranges of up to wpc consecutive windows.  A sample's values are
// sorted, so a sample's values in a range are one segment, walked by one
// warp; its start is found by binary search once per group of ranges.
//
// Pass 1 (k_win_tiles, one CTA per group of kTileRanges ranges and tile):
// the tile's filter bitmap of each range is set in shared memory and stored.
// k_win_classify (one CTA per window) classifies the rows - class 0: held by
// two or more tiles; class 1 + t: by tile t alone (with the two-or-more
// filter, by two or more of its samples) - and writes every class word's
// rank within its window and every class's rows per window; k_win_agg sums
// the counts per range.
//
// Ranks: a class's rows are numbered in row order, range after range, and
// each range's count is rounded up to a multiple of 64 - the rows in between
// are zero rows of the packed matrix, which add nothing to C (Eq. 4) - so
// that every packed word belongs to one range.
//
// Pass 2 (k_win_pack, one CTA per range and tile): the tile's samples are
// packed into the class-0 matrix XM and the tile's matrix XS.  A value's
// class and rank come from the range's class words and their window ranks
// in shared memory; a sample's bits are gathered in shared memory, kStage
// words at a time, and stored as whole words with plain stores.  Every word
// of the batch's part of XM and XS is written exactly once, zero words
// included, so nothing is zeroed beforehand and no global atomics are
// needed.
#include "ingest_dev.cuh"

namespace jsim {

namespace {

constexpr int kWin1Threads = 256;
constexpr int kSlots1 = 4;        // samples a warp walks at once in pass 1
constexpr int kClassThreads = 256;
constexpr int kClassWords = 4;    // words of a window per classify thread (2^16 rows = 256 x 4 words)
constexpr u64 kTileRanges = 4;    // consecutive ranges a pass-1 CTA walks
constexpr int kWin2Threads = 512;
constexpr int kWin2Warps = kWin2Threads / 32;
constexpr int kDepth2 = 4;        // 32-value chunks of a sample a warp loads at once in pass 2
constexpr int kStage = 64;        // words gathered at a time per sample and class
constexpr u64 kWinTile = 128;     // samples per tile

// Bring the 32 values from p on (up to e) toward L2 ahead of their loads.
__device__ __forceinline__ void prefetch_values(const u64* ids, u64 p, u64 e)
{
    if (p < e) asm volatile("prefetch.global.L2 [%0];" ::"l"(ids + p));
    if (p + 16 < e) asm volatile("prefetch.global.L2 [%0];" ::"l"(ids + p + 16));
}

// Pass 1: CTA (range group rq, tile t) = blockIdx.x (rq * T + t) walks
// tile t's samples through ranges kTileRanges rq .. kTileRanges rq +
// kTileRanges - 1 in turn: per range it sets the rows that the tile's
// samples hold (Eq. 5 over the tile; TWICE: also the rows two or more of
// them hold) in shared memory and stores the bitmaps to B (and B2),
// tile-major.  Only the group's first range needs its cursors found by
// search; the next range starts where the walk stopped.  Shared memory: the
// bitmaps, then the tile's cursors and ends.  A warp walks kSlots1 samples
// at once, 32 consecutive values of each per step, and takes the next
// sample when one leaves the range.  Five CTAs an SM with one filter bitmap
// (47 registers, no spills); the two-or-more filter keeps four.
template <bool TWICE>
__global__ void __launch_bounds__(kWin1Threads, TWICE ? 4 : 5)
k_win_tiles(const u64* __restrict__ ids, Plan plan, WinGeom g, u64* __restrict__ B, u64* __restrict__ B2,
            u64* __restrict__ curs)
{
    extern __shared__ __align__(16) unsigned char win_smem[];
    const u64 rq = blockIdx.x / g.T, t = blockIdx.x % g.T;
    u32* bm = reinterpret_cast<u32*>(win_smem);
    u32* bm2 = bm + (g.wpc << (g.wl - 5));
    u64* cur = reinterpret_cast<u64*>(bm + (TWICE ? 2 : 1) * (g.wpc << (g.wl - 5)));
    u64* cend = cur + kWinTile;
    __shared__ u32 s_next;
    const int tid = threadIdx.x, lane = tid & 31;
    const u64 k0 = t * kWinTile, m = min(kWinTile, g.n - k0);
    const u64 r_end = min(rq * kTileRanges + kTileRanges, g.G);

    for (u64 r = rq * kTileRanges; r < r_end; ++r) {
        const u64 w0 = r * g.wpc, w1 = min(w0 + g.wpc, g.nwin);
        const u64 rows_r = (w1 - w0) << g.wl, RW64 = rows_r >> 6;
        const u64 rlo = g.lo + (w0 << g.wl);
        {
            uint4* z = reinterpret_cast<uint4*>(bm);
            const u64 nz = (TWICE ? 2 : 1) * (g.wpc << (g.wl - 5)) / 4;
            for (u64 i = tid; i < nz; i += kWin1Threads) z[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        if (tid == 0) s_next = 0;
        for (u64 kk = tid; kk < m; kk += kWin1Threads) {
            u64 c;
            if (r == rq * kTileRanges) {
                const u64 b = plan.beg[k0 + kk], e = b + plan.len[k0 + kk];
                c = w0 == 0 ? b : lower_bound_u64(ids, b, e, rlo);
                cur[kk] = c;
                cend[kk] = e;
            } else {
                c = cur[kk];
            }
            curs[r * g.n + k0 + kk] = c;
        }
        __syncthreads();
        for (u64 kk = tid; kk < m; kk += kWin1Threads) prefetch_values(ids, cur[kk], cend[kk]);

        // samples go to warps as they free a slot (sizes vary by two decades)
        u64 ks[kSlots1], ps[kSlots1], es[kSlots1], prev[kSlots1];
        bool act[kSlots1], hp[kSlots1];
        auto take = [&](int s) {
            u32 e = 0;
            if (lane == 0) {
                e = atomicAdd(&s_next, 1u);
                if (e < m) e = g.lpt[k0 + e];  // largest samples first
            }
            e = __shfl_sync(0xffffffffu, e, 0);
            act[s] = e < m;
            ks[s] = e;
            ps[s] = act[s] ? cur[e] : 0;
            es[s] = act[s] ? cend[e] : 0;
            hp[s] = false;  // the value before a range's first one is below it (sorted input)
            prev[s] = 0;
        };
        #pragma unroll
        for (int s = 0; s < kSlots1; ++s) take(s);
        for (;;) {
            bool any = false;
            #pragma unroll
            for (int s = 0; s < kSlots1; ++s) any = any || act[s];
            if (!any) break;
            u64 x[kSlots1];
            #pragma unroll
            for (int s = 0; s < kSlots1; ++s) {
                const u64 pos = ps[s] + (u64)lane;
                x[s] = (act[s] && pos < es[s]) ? ids[pos] : 0ull;
            }
            #pragma unroll
            for (int s = 0; s < kSlots1; ++s) {
                if (!act[s]) continue;
                const u64 pos = ps[s] + (u64)lane, v = x[s], d = v - rlo;
                // the values from the first one at or past the range's end stay for
                // the next range (a value below it only comes from unsorted input,
                // and is passed over)
                const bool stop = pos >= es[s] || (v >= rlo && d >= rows_r);
                const unsigned bal = __ballot_sync(0xffffffffu, stop);
                const int run = bal ? __ffs((int)bal) - 1 : 32;
                if (TWICE) {
                    const u64 pv = __shfl_up_sync(0xffffffffu, v, 1);
                    const u64 lastv = __shfl_sync(0xffffffffu, v, 31);
                    const bool dup = lane ? pv == v : (hp[s] && prev[s] == v);
                    if (lane < run && v >= rlo && !dup) {
                        const u32 bit = 1u << (d & 31);
                        const u32 old = atomicOr(bm + (d >> 5), bit);
                        if (old & bit) atomicOr(bm2 + (d >> 5), bit);
                    }
                    hp[s] = true;
                    prev[s] = lastv;
                } else if (lane < run && v >= rlo) {
                    atomicOr(bm + (d >> 5), 1u << (d & 31));
                }
                ps[s] += (u64)run;
                if (run < 32) {
                    if (lane == 0) {
                        cur[ks[s]] = ps[s];  // the next range of the group starts here
                        // the last range's ends close pass 2's segments (every other
                        // group's CTA finds its own first cursors)
                        if (r + 1 == g.G) curs[(r + 1) * g.n + k0 + ks[s]] = ps[s];
                    }
                    take(s);
                }
            }
        }
        __syncthreads();
        const u64* b64 = reinterpret_cast<const u64*>(bm);
        u64* out = B + t * g.nw + (w0 << (g.wl - 6));
        for (u64 j = tid; j < RW64; j += kWin1Threads) out[j] = b64[j];
        if (TWICE) {
            const u64* c64 = reinterpret_cast<const u64*>(bm2);
            u64* out2 = B2 + t * g.nw + (w0 << (g.wl - 6));
            for (u64 j = tid; j < RW64; j += kWin1Threads) out2[j] = c64[j];
        }
        __syncthreads();  // the bitmaps are cleared and the cursors read for the next range
    }
}

// Classes of window w's rows = blockIdx.x from the tiles' bitmaps: class 0
// = rows of two or more tiles, class 1 + t = rows of tile t alone (with the
// two-or-more filter: rows tile t holds twice or more and no other tile
// holds); the class words, every word's rank within the window (the class's
// rows below it, 16 bits: a window has at most 2^16 rows), and the window's
// rows per class.  Thread i takes the window's words [kClassWords i,
// kClassWords (i + 1)); the words are formed twice (for the counts, then for
// the ranks), the second time from tile words still in L1.
__global__ void __launch_bounds__(kClassThreads, 4)
k_win_classify(const u64* __restrict__ B, const u64* __restrict__ B2, WinGeom g, u64* __restrict__ cls,
               unsigned short* __restrict__ pre, u32* __restrict__ cnt)
{
    __shared__ u64 s_scan[kClassThreads / 32];
    const int tid = threadIdx.x;
    const u64 w = blockIdx.x, W64 = 1ull << (g.wl - 6);
    const u64 j0 = w * W64 + (u64)tid * kClassWords;
    const bool mine = (u64)tid * kClassWords < W64;
    u64 twos[kClassWords];
    #pragma unroll
    for (int i = 0; i < kClassWords; ++i) {
        u64 ones = 0, tw = 0;
        if (mine)
            for (u64 q = 0; q < g.T; ++q) {
                const u64 v = B[q * g.nw + j0 + i];
                tw |= ones & v;
                ones |= v;
            }
        twos[i] = tw;
    }
    auto word = [&](u64 q, int i) -> u64 {  // class q's word i of this thread
        if (q == 0) return twos[i];
        const u64 v = B2 ? B2[(q - 1) * g.nw + j0 + i] : B[(q - 1) * g.nw + j0 + i];
        return v & ~twos[i];
    };
    // counts of this thread's words, three classes to a scan (fields of 21 bits)
    for (u64 q0 = 0; q0 <= g.T; q0 += 3) {
        u64 packed = 0;
        for (u64 f = 0; f < 3 && q0 + f <= g.T; ++f) {
            u64 sum = 0;
            if (mine)
                #pragma unroll
                for (int i = 0; i < kClassWords; ++i) {
                    const u64 v = word(q0 + f, i);
                    cls[(q0 + f) * g.nw + j0 + i] = v;
                    sum += (u64)__popcll(v);
                }
            packed |= sum << (21 * f);
        }
        u64 ex;
        const u64 tot = block_exclusive_scan<kClassThreads>(packed, ex, s_scan);
        for (u64 f = 0; f < 3 && q0 + f <= g.T; ++f) {
            const u64 q = q0 + f;
            u32 run = (u32)((ex >> (21 * f)) & 0x1fffffull);
            if (mine)
                #pragma unroll
                for (int i = 0; i < kClassWords; ++i) {
                    pre[q * g.nw + j0 + i] = (unsigned short)run;
                    run += (u32)__popcll(cls[q * g.nw + j0 + i]);
                }
            if (tid == 0) cnt[q * g.nwin + w] = (u32)((tot >> (21 * f)) & 0x1fffffull);
        }
    }
}

// Every range's rows per class, rounded up to 64 (one thread per class and
// range), and the rows of all classes into plan.totals.
__global__ void k_win_agg(const u32* __restrict__ cnt, WinGeom g, Plan plan, u64* __restrict__ agg)
{
    const u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x;
    if (i >= (g.T + 1) * g.G) return;
    const u64 c = i / g.G, r = i - c * g.G;
    const u64 w0 = r * g.wpc, w1 = min(w0 + g.wpc, g.nwin);
    u64 s = 0;
    for (u64 w = w0; w < w1; ++w) s += cnt[c * g.nwin + w];
    agg[i] = (s + 63) / 64 * 64;
    if (s) atomicAdd((unsigned long long*)(plan.totals + kPlanRowsTotal), (unsigned long long)s);
}

// Pass 2 state of one class of a range: the rows' first word of the range
// in the matrix (row kk of the tile at base + kk * stride) and the range's
// words per row (a multiple-of-64 rank count / 64).
struct RangeClass {
    u64* base;
    u64 stride;
    u32 qn;
};

// Store the staged words [blk, blk + kStage) of the range and clear them.
__device__ __forceinline__ void rc_flush(const RangeClass& c, u64* row, u32 blk, u64* st, int lane)
{
    __syncwarp();
    #pragma unroll
    for (int i = 0; i < kStage / 32; ++i) {
        const u32 q = blk + (u32)(32 * i + lane);
        if (q < c.qn) row[q] = st[32 * i + lane];
        st[32 * i + lane] = 0ull;
    }
    __syncwarp();
}

// Put bit `bit` of word q (lanes with has) into the staged words from blk
// on; the staged block moves forward as the sample's ranks pass it, and the
// words it passes over are stored as zeros.  Ranks grow along a sample's
// sorted values, so the lowest pending lane holds the lowest pending word;
// a word outside the range (only from unsorted input) is dropped.
__device__ __forceinline__ void rc_place(const RangeClass& c, u64* row, u32& blk, u64* st, bool has, u32 q, u64 bit,
                                         int lane)
{
    for (;;) {
        const bool fit = has && q >= blk && q < blk + kStage && q < c.qn;
        if (fit) atomicOr((unsigned long long*)(st + (q - blk)), (unsigned long long)bit);
        has = has && !fit && q >= blk && q < c.qn;
        const unsigned pend = __ballot_sync(0xffffffffu, has);
        if (!pend) return;
        const u32 qmin = __shfl_sync(0xffffffffu, q, __ffs((int)pend) - 1);
        rc_flush(c, row, blk, st, lane);
        const u32 tgt = blk + (qmin - blk) / kStage * kStage;
        for (u32 z = blk + kStage + (u32)lane; z < tgt; z += 32) row[z] = 0ull;
        blk = tgt;
    }
}

// Pass 2: CTA (range r, tile t) = blockIdx.x (r * T + t) packs the tile's
// samples over the whole range.  Shared memory: the range's class-0 and
// class-(1 + t) words, their ranks within each window, and the staged words
// of every warp's sample.  A warp packs one sample at a time,
// kDepth2 x 32 consecutive values per step; a sample's ranks run on from
// window to window, and the range holds whole words, so every word is
// stored once, by its sample's warp.
__global__ void __launch_bounds__(kWin2Threads, 2)
k_win_pack(const u64* __restrict__ ids, WinGeom g, const u64* __restrict__ cls,
           const unsigned short* __restrict__ pre, const u32* __restrict__ cnt, const u64* __restrict__ boff,
           const u64* __restrict__ curs, const u64* __restrict__ kbase, u64* XM, u64 stride_m, u64* XS, u64 stride_s)
{
    extern __shared__ __align__(16) unsigned char win_smem[];
    const u32 W64 = (u32)(1u << (g.wl - 6));
    const u64 r = blockIdx.x / g.T, t = blockIdx.x % g.T;
    const u64 w0 = r * g.wpc, w1 = min(w0 + g.wpc, g.nwin);
    const u32 nwr = (u32)(w1 - w0), RW = nwr * W64;  // the range's windows and words per class
    u64* sW = reinterpret_cast<u64*>(win_smem);                                 // [2][RW]
    u64* stage = sW + 2 * (u64)g.wpc * W64;                                     // [warps][2][kStage]
    unsigned short* sP = reinterpret_cast<unsigned short*>(stage + kWin2Warps * 2 * kStage);  // [2][RW]
    __shared__ u32 s_wb[2][kMaxWinPerRange];
    __shared__ u64 s_rb[2];
    __shared__ u32 s_qn[2];
    __shared__ u32 s_next;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u64 k0 = t * kWinTile, m = min(kWinTile, g.n - k0);
    const u64 cl1 = 1 + t;

    for (int i = tid; i < kWin2Warps * 2 * kStage; i += kWin2Threads) stage[i] = 0ull;
    for (u32 j = tid; j < RW; j += kWin2Threads) {
        sW[j] = cls[w0 * W64 + j];
        sW[RW + j] = cls[cl1 * g.nw + w0 * W64 + j];
        sP[j] = pre[w0 * W64 + j];
        sP[RW + j] = pre[cl1 * g.nw + w0 * W64 + j];
    }
    if (tid == 0) s_next = 0;
    if (tid < 2) {
        const u64 c = tid ? cl1 : 0;
        u32 s = 0;
        for (u32 wi = 0; wi < nwr; ++wi) {
            s_wb[tid][wi] = s;
            s += cnt[c * g.nwin + w0 + wi];
        }
        s_rb[tid] = (boff[c * g.G + r] - boff[c * g.G]) / 64;  // ranges start on whole words
        s_qn[tid] = (s + 63) / 64;
    }
    __syncthreads();

    RangeClass cl[2];
    cl[0].base = XM ? XM + k0 * stride_m + kbase[0] + s_rb[0] : nullptr;
    cl[0].stride = stride_m;
    cl[0].qn = XM ? s_qn[0] : 0;
    cl[1].base = XS ? XS + k0 * stride_s + kbase[cl1] + s_rb[1] : nullptr;
    cl[1].stride = stride_s;
    cl[1].qn = XS ? s_qn[1] : 0;
    u64* st_w = stage + warp * 2 * kStage;
    const u64 rlo = g.lo + (w0 << g.wl), rows_r = (u64)nwr << g.wl;

    // the tile's samples, one per warp at a time (they go to warps as the
    // warps finish one): its segment of the range, up to 4 x 32 values per step
    const int wsh = g.wl - 6;  // words of a window = 1 << wsh
    for (;;) {
        u32 e32 = 0;
        if (lane == 0) {
            e32 = atomicAdd(&s_next, 1u);
            if (e32 < m) e32 = g.lpt[k0 + e32];  // largest samples first
        }
        const u64 e = __shfl_sync(0xffffffffu, e32, 0);
        if (e >= m) break;
        const u64 a = curs[r * g.n + k0 + e], b = max(a, curs[(r + 1) * g.n + k0 + e]);
        u64* row0 = cl[0].base ? cl[0].base + e * cl[0].stride : nullptr;
        u64* row1 = cl[1].base ? cl[1].base + e * cl[1].stride : nullptr;
        u32 blk0 = 0, blk1 = 0;
        for (u64 p = a; p < b; p += kDepth2 * 32) {
            u64 x[kDepth2];
            #pragma unroll
            for (int i = 0; i < kDepth2; ++i) {
                const u64 pos = p + (u64)(32 * i + lane);
                x[i] = pos < b ? ids[pos] : 0ull;
            }
            #pragma unroll
            for (int i = 0; i < kDepth2; ++i) {
                if (p + (u64)(32 * i) >= b) break;
                // class and rank of this lane's value: class 0 if its row is
                // held by two or more tiles, else the tile's class if kept there
                const u64 d64 = x[i] - rlo;
                const bool in = p + (u64)(32 * i + lane) < b && d64 < rows_r;
                const u32 d = in ? (u32)d64 : 0u, j = d >> 6, sh = d & 63u;
                const u64 c0w = sW[j], c1w = sW[RW + j];
                const bool h0 = in && ((c0w >> sh) & 1ull), h1 = in && !h0 && ((c1w >> sh) & 1ull);
                const u32 cc = h1 ? 1u : 0u;
                const u32 rk = s_wb[0][cc * kMaxWinPerRange + (j >> wsh)] + (u32)sP[cc * RW + j] +
                               (u32)__popcll((h1 ? c1w : c0w) & ((1ull << sh) - 1ull));
                const bool has = h0 || h1;
                const u32 q = rk >> 6;
                const u64 bit = 1ull << (rk & 63u);
                const u32 bk = h1 ? blk1 : blk0, qn = h1 ? cl[1].qn : cl[0].qn;
                const bool fit = has && q >= bk && q < bk + kStage && q < qn;
                if (!__any_sync(0xffffffffu, has && !fit)) {
                    if (fit) atomicOr((unsigned long long*)(st_w + cc * kStage + (q - bk)), (unsigned long long)bit);
                } else {
                    rc_place(cl[0], row0, blk0, st_w, h0, q, bit, lane);
                    rc_place(cl[1], row1, blk1, st_w + kStage, h1, q, bit, lane);
                }
            }
        }
        rc_flush(cl[0], row0, blk0, st_w, lane);
        for (u32 z = blk0 + kStage + (u32)lane; z < cl[0].qn; z += 32) row0[z] = 0ull;
        rc_flush(cl[1], row1, blk1, st_w + kStage, lane);
        for (u32 z = blk1 + kStage + (u32)lane; z < cl[1].qn; z += 32) row1[z] = 0ull;
    }
}

}  // namespace

size_t win_tiles_smem(const WinGeom& g, bool twice)
{
    return (size_t)(twice ? 2 : 1) * ((size_t)g.wpc << (g.wl - 3)) + 2 * kWinTile * 8;
}

size_t win_pack_smem(const WinGeom& g)
{
    const size_t RW = (size_t)g.wpc << (g.wl - 6);
    return 2 * RW * 8 + (size_t)kWin2Warps * 2 * kStage * 8 + 2 * RW * 2;
}

cudaError_t launch_win_classes(const u64* ids, Plan plan, const WinGeom& g, bool twice, u64* B, u64* B2, u64* cls,
                               unsigned short* pre, u32* cnt, u64* agg, u64* curs, cudaStream_t st)
{
    if (g.G == 0) return cudaSuccess;
    const size_t smem = win_tiles_smem(g, twice);
    const unsigned grid = (unsigned)((g.G + kTileRanges - 1) / kTileRanges * g.T);
    cudaError_t e;
    if (twice) {
        e = cudaFuncSetAttribute(k_win_tiles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_win_tiles<true><<<grid, kWin1Threads, smem, st>>>(ids, plan, g, B, B2, curs);
    } else {
        e = cudaFuncSetAttribute(k_win_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_win_tiles<false><<<grid, kWin1Threads, smem, st>>>(ids, plan, g, B, nullptr, curs);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_win_classify<<<(unsigned)g.nwin, kClassThreads, 0, st>>>(B, twice ? B2 : nullptr, g, cls, pre, cnt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_win_agg<<<(unsigned)(((g.T + 1) * g.G + 255) / 256), 256, 0, st>>>(cnt, g, plan, agg);
    return cudaGetLastError();
}

cudaError_t launch_win_pack(const u64* ids, const WinGeom& g, const u64* cls, const unsigned short* pre,
                            const u32* cnt, const u64* boff, const u64* curs, const u64* kbase, u64* XM, u64 stride_m,
                            u64* XS, u64 stride_s, cudaStream_t st)
{
    if (g.G == 0 || g.T == 0 || (!XM && !XS)) return cudaSuccess;
    const size_t smem = win_pack_smem(g);
    cudaError_t e = cudaFuncSetAttribute(k_win_pack, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_win_pack<<<(unsigned)(g.G * g.T), kWin2Threads, smem, st>>>(ids, g, cls, pre, cnt, boff, curs, kbase, XM,
                                                                  stride_m, XS, stride_s);
    return cudaGetLastError();
}

}  // namespace jsim
