// Ingest kernels: per-batch plan, input validation, the zero-row filter
// f^(l) (Eq. 5), its prefix sum p^(l) as a rank directory (Eq. 6), and the
// bitmask compression of the surviving rows into 64-bit words (Sec. III-B).
#include "ingest_dev.cuh"

namespace jsim {

namespace {

// One CTA: per-sample [beg, beg+len) of values in [lo, hi) and chunk prefix.
// With perm, entry i of the plan is sample perm[i] (the ingest kernels then
// walk the samples in that order).  With ends, sample i is searched in
// [offsets[i], ends[i]) only.
__global__ void __launch_bounds__(kPlanThreads)
k_plan(const u64* __restrict__ offsets, const u64* __restrict__ ids, u64 n, u64 lo, u64 hi,
       int full, Plan plan, const u32* __restrict__ perm, const u64* __restrict__ ends)
{
    __shared__ u64 sm[kPlanThreads / 32];
    __shared__ u64 s_next;
    __shared__ int s_has_next;
    if (threadIdx.x == 0) { s_next = ~0ull; s_has_next = 0; }
    __syncthreads();
    u64 carry = 0, total_len = 0;
    for (u64 base = 0; base < n; base += kPlanThreads) {
        u64 i = base + threadIdx.x;
        u64 b = 0, l = 0, nch = 0;
        if (i < n) {
            const u64 si = perm ? (u64)perm[i] : i;
            u64 s = offsets[si], e = ends ? ends[si] : offsets[si + 1];
            if (!full) {
                const u64 se = e;
                u64 bb = lower_bound_u64(ids, s, e, lo);
                u64 ee = hi == 0 ? e : lower_bound_u64(ids, bb, e, hi);  // hi==0: unbounded
                s = bb; e = ee;
                if (ee < se) {  // first value of this sample after the batch
                    atomicMin(&s_next, ids[ee]);
                    s_has_next = 1;
                }
            }
            b = s; l = e - s; nch = (l + kChunk - 1) / kChunk;
            plan.beg[i] = b;
            plan.len[i] = l;
        }
        u64 ex;
        u64 tot = block_exclusive_scan<kPlanThreads>(nch, ex, sm);
        if (i < n) plan.cofs[i] = carry + ex;
        carry += tot;
        u64 ex2;
        total_len += block_exclusive_scan<kPlanThreads>(l, ex2, sm);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        plan.cofs[n] = carry;
        plan.totals[0] = total_len;
        plan.totals[1] = carry;
        plan.totals[2] = s_next;
        plan.totals[3] = (u64)s_has_next;
        for (u64 k = 4; k < kPlanTotals; ++k) plan.totals[k] = 0;  // chunk tickets
    }
}

constexpr int kValidateDepth = 4;  // values a thread loads per step

__global__ void __launch_bounds__(kIngestThreads)
k_validate(const u64* __restrict__ offsets, const u64* __restrict__ ids, u64 n, Plan plan,
           int id_bits, u64* sizes, u32* err, u64* maxid, u64* minid, u64 err_stride)
{
    __shared__ ChunkDesc s_d[2];
    __shared__ u32 s_cnt[kIngestThreads / 32];
    const u64 nch = plan.totals[1];
    if (threadIdx.x == 0) fetch_chunk(plan, n, nch, kTicketValidate, s_d[0]);
    __syncthreads();
    for (int db = 0;; db ^= 1) {
        const ChunkDesc d = s_d[db];
        if (d.c >= nch) break;
        if (threadIdx.x == 0) fetch_chunk(plan, n, nch, kTicketValidate, s_d[db ^ 1]);
        const u64 i = d.i, p0 = d.p0, p1 = d.p1;
        const u64 sb = offsets[i], se = offsets[i + 1];
        u32 cnt = 0, flags = 0;
        // kValidateDepth coalesced loads a thread in flight per step; a
        // value's predecessor comes from the lane before it (lane 0 loads
        // its own, ahead, with the values)
        const int lane = threadIdx.x & 31;
        for (u64 base = p0; base < p1; base += kValidateDepth * kIngestThreads) {
            u64 x[kValidateDepth], pv[kValidateDepth];
            #pragma unroll
            for (int k = 0; k < kValidateDepth; ++k) {
                const u64 pos = base + (u64)(k * kIngestThreads) + threadIdx.x;
                x[k] = pos < p1 ? ids[pos] : 0ull;
                pv[k] = (lane == 0 && pos < p1 && pos > sb) ? ids[pos - 1] : 0ull;
            }
            #pragma unroll
            for (int k = 0; k < kValidateDepth; ++k) {
                const u64 pos = base + (u64)(k * kIngestThreads) + threadIdx.x;
                const u64 up = __shfl_up_sync(0xffffffffu, x[k], 1);
                if (pos >= p1) continue;
                const u64 v = x[k];
                if (pos > sb) {
                    const u64 prev = lane ? up : pv[k];
                    if (v < prev) flags |= kFlagUnsorted;
                    cnt += (v != prev);
                } else {
                    cnt += 1;
                    atomicMin(minid, v);
                }
                if (id_bits < 64 && (v >> id_bits) != 0) flags |= kFlagIdRange;
                if (pos + 1 == se) atomicMax(maxid, v);
            }
        }
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            flags |= __shfl_xor_sync(0xffffffffu, flags, o);
        }
        if ((threadIdx.x & 31) == 0) {
            s_cnt[threadIdx.x >> 5] = cnt;
            if (flags) atomicOr(err + i * err_stride, flags);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            u32 t = 0;
            for (int w = 0; w < kIngestThreads / 32; ++w) t += s_cnt[w];
            atomicAdd(sizes + i, (u64)t);
        }
        __syncthreads();
    }
}

// f^(l): set bit (x - lo) for every value x of the batch (Eq. 5).  With
// `twice`, also set it there for rows held by two or more samples: the
// atomic OR returns the bits other samples had already set.  A sample's
// repeated value is skipped for `twice` (a set holds it once).
__global__ void __launch_bounds__(kIngestThreads)
k_filter(const u64* __restrict__ ids, u64 n, Plan plan, u64 lo, u64 width, u32* bitmap_all, u32* twice_all,
         const u32* __restrict__ tile_of, u64 tile_words)
{
    __shared__ ChunkDesc s_d[2];
    const u64 nch = plan.totals[1];
    if (threadIdx.x == 0) fetch_chunk(plan, n, nch, kTicketFilter, s_d[0]);
    __syncthreads();
    for (int db = 0;; db ^= 1) {
        const ChunkDesc d = s_d[db];
        if (d.c >= nch) break;
        if (threadIdx.x == 0) fetch_chunk(plan, n, nch, kTicketFilter, s_d[db ^ 1]);
        const u64 p0 = d.p0, p1 = d.p1, bb = d.b;
        // the sample's own bitmap (one per sample tile when tile_of is given)
        const u64 toff = tile_of ? (u64)tile_of[d.i] * tile_words : 0ull;
        u32* bitmap = bitmap_all + toff;
        u32* twice = twice_all ? twice_all + toff : nullptr;
        // every warp walks whole 32-position groups so shuffles see full warps
        for (u64 base = p0 + (threadIdx.x & ~31u); base < p1; base += kIngestThreads) {
            u64 pos = base + (threadIdx.x & 31);
            u64 q = ~0ull;
            u32 bit = 0;
            if (pos < p1) {
                const u64 x = __ldcs(ids + pos);  // read once: evict first
                u64 d = x - lo;
                if (d < width && !(twice && pos > bb && ids[pos - 1] == x)) { q = d >> 5; bit = 1u << (d & 31); }
            }
            bool lead = segmented_or<u32>(q, bit);
            if (lead && bit) {
                const u32 old = atomicOr(bitmap + q, bit);
                if (twice && (old & bit)) atomicOr(twice + q, old & bit);
            }
        }
        __syncthreads();
    }
}

// Directory pass 1: per 4096-word block, block-relative exclusive popcounts.
// Rounds of 512 consecutive words, two per thread, so every load and store
// of a warp is one contiguous 256-byte (load) or 128-byte (store) run.
__global__ void __launch_bounds__(kScanThreads)
k_scan_blocks(const u64* __restrict__ bitmap, u64 nwords, u32* __restrict__ dir, u64* __restrict__ bsum)
{
    constexpr int kRound = 2 * kScanThreads;
    static_assert(kScanBlockWords % kRound == 0, "whole rounds per block");
    __shared__ u32 wsum[kScanThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const bool vec = ((uintptr_t)bitmap & 15u) == 0 && ((uintptr_t)dir & 7u) == 0;
    const u64 b0 = (u64)blockIdx.x * kScanBlockWords;
    u32 run = 0;
    for (int it = 0; it < (int)(kScanBlockWords / kRound); ++it) {
        const u64 w = b0 + (u64)it * kRound + 2 * (u64)t;
        u64 a = 0, b = 0;
        if (vec && w + 1 < nwords) {
            const ulonglong2 v = __ldg((const ulonglong2*)(bitmap + w));
            a = v.x;
            b = v.y;
        } else {
            if (w < nwords) a = bitmap[w];
            if (w + 1 < nwords) b = bitmap[w + 1];
        }
        const u32 pa = (u32)__popcll(a), pc = pa + (u32)__popcll(b);
        u32 x = pc;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        u32 woff = 0, tot = 0;
        #pragma unroll
        for (int k = 0; k < kScanThreads / 32; ++k) {
            const u32 v = wsum[k];
            if (k < warp) woff += v;
            tot += v;
        }
        const u32 ex = run + woff + x - pc;
        if (vec && w + 1 < nwords) {
            *(uint2*)(dir + w) = make_uint2(ex, ex + pa);
        } else {
            if (w < nwords) dir[w] = ex;
            if (w + 1 < nwords) dir[w + 1] = ex + pa;
        }
        run += tot;
        __syncthreads();  // wsum is rewritten next round
    }
    if (t == 0) bsum[blockIdx.x] = run;
}

// Directory pass 2 (one CTA): exclusive prefix of block sums; R = total.
__global__ void __launch_bounds__(1024)
k_scan_top(const u64* __restrict__ bsum, u64 nb, u64* __restrict__ boff, u64* R, u64* ktotal, u64* kbase)
{
    __shared__ u64 sm[32];
    u64 carry = 0;
    for (u64 base = 0; base < nb; base += 1024) {
        u64 b = base + threadIdx.x;
        u64 v = b < nb ? bsum[b] : 0, ex;
        u64 tot = block_exclusive_scan<1024>(v, ex, sm);
        if (b < nb) boff[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        *R = carry;
        // batches appended along the word axis: this batch's words start at
        // the running total, which then grows by ceil(R / 64)
        if (ktotal) {
            *kbase = *ktotal;
            *ktotal += (carry + 63) / 64;
        }
    }
}

__global__ void k_zero_rows(u64* X, u64 rows, u64 stride, u64 words)
{
    const u64 per_row = words;
    const u64 total = rows * per_row;
    for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (u64)gridDim.x * blockDim.x) {
        u64 r = t / per_row, w = t - r * per_row;
        X[r * stride + w] = 0ull;
    }
}

// Bitmask compression: value x of sample i -> rank r = p^(l)_{x-lo}; word
// r/64, bit r%64 of row i (Eq. 6 and the b-bit masks before Eq. 7).
__global__ void __launch_bounds__(kIngestThreads)
k_pack(const u64* __restrict__ ids, u64 n, Plan plan, u64 lo, u64 width,
       const u64* __restrict__ bitmap, const u32* __restrict__ dir, const u64* __restrict__ boff,
       u64* X, u64 stride, u64* batch_sizes, const u64* kbase, u64 wstride)
{
    __shared__ u64 s_i, s_p0, s_p1, s_b, s_c;
    __shared__ u32 s_cnt[kIngestThreads / 32];
    const u64 nch = plan.totals[1];
    for (;;) {
        if (threadIdx.x == 0) {
            const u64 c = next_chunk(plan, kTicketPack);
            s_c = c;
            if (c < nch) {
                u64 i = chunk_sample(plan.cofs, n, c);
                u64 p0 = plan.beg[i] + (c - plan.cofs[i]) * kChunk;
                s_i = i; s_p0 = p0; s_b = plan.beg[i];
                s_p1 = min(p0 + kChunk, plan.beg[i] + plan.len[i]);
            }
        }
        __syncthreads();
        if (s_c >= nch) break;
        const u64 i = s_i, p0 = s_p0, p1 = s_p1, bb = s_b;
        u64* row = X + i * stride + (kbase ? *kbase : 0ull) * wstride;
        u32 cnt = 0;
        for (u64 base = p0 + (threadIdx.x & ~31u); base < p1; base += kIngestThreads) {
            u64 pos = base + (threadIdx.x & 31);
            u64 q = ~0ull, bit = 0;
            if (pos < p1) {
                u64 x = ids[pos];
                u64 d = x - lo;
                if (d < width) {
                    const u64 w = d >> 6, word = bitmap[w];
                    // rows the bitmap leaves out (held by one sample, when it
                    // is the two-or-more filter) are not packed
                    if ((word >> (d & 63)) & 1ull) {
                        u64 r = boff[w / kScanBlockWords] + (u64)dir[w] +
                                (u64)__popcll(word & ((1ull << (d & 63)) - 1ull));
                        q = r >> 6;
                        bit = 1ull << (r & 63);
                    }
                }
                if (batch_sizes) cnt += (pos == bb) || (ids[pos - 1] != x);
            }
            bool lead = segmented_or<u64>(q, bit);
            if (lead && bit) atomicOr(row + q * wstride, bit);
        }
        if (batch_sizes) {
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
            __syncthreads();
            if (threadIdx.x == 0) {
                u32 t = 0;
                for (int w = 0; w < kIngestThreads / 32; ++w) t += s_cnt[w];
                atomicAdd(batch_sizes + i, (u64)t);
            }
        }
        __syncthreads();
    }
}

// Packing with plain stores instead of atomic read-modify-writes: every
// nonzero word of a batch's rows is written once, complete, into the zeroed
// packed matrix.  Rank r' (the number of kept rows below a value) is
// non-decreasing along a sample's sorted values, and so is its word q = r'/64
// (a value whose row is not kept still has an insertion word).  A sample's
// values in a chunk are cut into warp segments of kPackSeg values; segment k
// owns the words (q of the last value before it, q of its last value]: it
// writes their completed masks, finishing its last word by reading ahead
// into the next segment's values while their word is the same.
constexpr int kPackSeg = 512;
static_assert(kChunk % kPackSeg == 0 && kPackSeg * (kIngestThreads / 32) == kChunk,
              "a chunk is one segment per warp");

// A value outside [lo, lo + width) (only an unsorted input can put one in a
// slice) gets the sentinel word 2^63 - 1, which is never written.
__device__ __forceinline__ long long insertion_word(u64 x, u64 lo, u64 width, const u64* __restrict__ bitmap,
                                                    const u32* __restrict__ dir, const u64* __restrict__ boff,
                                                    u64& bit)
{
    const u64 d = x - lo;
    if (d >= width) {
        bit = 0ull;
        return 0x7fffffffffffffffll;
    }
    const u64 w = d >> 6, word = bitmap[w];
    const u64 below = word & ((1ull << (d & 63)) - 1ull);
    const u64 r = boff[w / kScanBlockWords] + (u64)dir[w] + (u64)__popcll(below);
    bit = ((word >> (d & 63)) & 1ull) ? (1ull << (r & 63)) : 0ull;
    return (long long)(r >> 6);
}

__global__ void __launch_bounds__(kIngestThreads)
k_pack_full(const u64* __restrict__ ids, u64 n, Plan plan, u64 lo, u64 width, const u64* __restrict__ bitmap,
            const u32* __restrict__ dir, const u64* __restrict__ boff, u64* X, u64 stride,
            const u64* kbase, const u64* __restrict__ Rdev)
{
    __shared__ u64 s_i, s_p0, s_p1, s_b, s_e, s_c;
    const u64 nch = plan.totals[1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long Wl = (long long)((*Rdev + 63) / 64);
    const long long kBig = 0x7fffffffffffffffll;
    for (;;) {
        if (threadIdx.x == 0) {
            const u64 c = next_chunk(plan, kTicketPack);
            s_c = c;
            if (c < nch) {
                const u64 i = chunk_sample(plan.cofs, n, c);
                const u64 p0 = plan.beg[i] + (c - plan.cofs[i]) * kChunk;
                s_i = i; s_p0 = p0; s_b = plan.beg[i];
                s_e = plan.beg[i] + plan.len[i];
                s_p1 = min(p0 + kChunk, s_e);
            }
        }
        __syncthreads();
        if (s_c >= nch) break;
        const u64 i = s_i, bb = s_b, be = s_e;
        const u64 sbeg = s_p0 + (u64)warp * kPackSeg, send = min(sbeg + kPackSeg, s_p1);
        __syncthreads();  // the shared chunk fields are read; the next chunk may overwrite them
        if (sbeg >= send) continue;
        u64* row = X + i * stride + (kbase ? *kbase : 0ull);
        u64 tmp;
        const long long seg_prev = sbeg > bb ? insertion_word(ids[sbeg - 1], lo, width, bitmap, dir, boff, tmp) : -1ll;
        long long open_key = seg_prev;
        u64 open_mask = 0ull;
        for (u64 base = sbeg; base < send; base += 32) {
            const u64 pos = base + lane;
            long long key = kBig;
            u64 bit = 0ull;
            if (pos < send) key = insertion_word(ids[pos], lo, width, bitmap, dir, boff, bit);
            const bool lead = segmented_or<u64>((u64)key, bit);
            const bool real = lead && key != kBig;
            const unsigned leads = __ballot_sync(0xffffffffu, real);
            const int last_lead = 31 - __clz((int)leads);  // leads != 0: lane 0 holds a value
            long long nkey = open_key;
            u64 nmask = open_mask;
            if (real) {
                u64 mask = bit;
                if (lane == 0) {
                    if (key == open_key) {
                        mask |= open_mask;  // the open word continues
                    } else if (open_key > seg_prev && open_key < Wl && open_mask) {
                        row[open_key] = open_mask;  // the open word is complete
                    }
                }
                if (lane != last_lead) {
                    if (key > seg_prev && key < Wl && mask) row[key] = mask;
                } else {
                    nkey = key;
                    nmask = mask;
                }
            }
            open_key = __shfl_sync(0xffffffffu, nkey, last_lead);
            open_mask = __shfl_sync(0xffffffffu, nmask, last_lead);
        }
        if (open_key > seg_prev) {
            // finish the last word with the next segment's values of the same word
            for (u64 base = send; base < be; base += 32) {
                const u64 pos = base + lane;
                long long key = kBig;
                u64 bit = 0ull;
                if (pos < be) key = insertion_word(ids[pos], lo, width, bitmap, dir, boff, bit);
                u64 m = key == open_key ? bit : 0ull;
                #pragma unroll
                for (int o = 16; o > 0; o >>= 1) m |= __shfl_xor_sync(0xffffffffu, m, o);
                open_mask |= m;
                if (__any_sync(0xffffffffu, key != open_key)) break;
            }
            if (lane == 0 && open_key < Wl && open_mask) row[open_key] = open_mask;
        }
    }
}

// The class-major layout of the block-sparse product: the rows of a batch
// are split into classes, each with its own bitmap (class c's words at cls +
// c * nwords), rank-scanned together (one directory over all classes; nwords
// is a multiple of kScanBlockWords, so class c's first block is c * nwords /
// kScanBlockWords and its ranks are the directory's minus that block's
// offset).
struct ClassView {
    const u64* cls;      // class bitmaps, class-major
    const u32* dir;      // rank directory of all classes (one entry per word)
    const u64* boff;     // block offsets of all classes
    const u64* kbase;    // first word of each class in X (device)
    u64 nwords;          // bitmap words per class
    const u32* cls_of;   // class of each sample, or null for class 0
    const u32* row_of;   // row of X of each sample
};

// Single-pass packing into both class matrices of the block-sparse product:
// a value of sample i whose row is of class 0 goes to XM, one of class
// cls_of[i] (the sample's tile) to XS, at word kbase[c] + (rank within the
// class) / 64 of row row_of[i]; other rows are not packed.  Classes
// interleave along a sample's values, so the words are OR-ed in with atomics
// (lanes of a warp holding the same word combine first).
__global__ void __launch_bounds__(kIngestThreads)
k_pack_classes(const u64* __restrict__ ids, u64 n, Plan plan, u64 lo, u64 width, ClassView v, u64* XM,
               u64 stride_m, u64* XS, u64 stride_s)
{
    __shared__ ChunkDesc s_d[2];
    const u64 nch = plan.totals[1];
    const u64 blk0 = 0;
    if (threadIdx.x == 0) fetch_chunk(plan, n, nch, kTicketPack, s_d[0]);
    __syncthreads();
    for (int db = 0;; db ^= 1) {
        const ChunkDesc d = s_d[db];
        if (d.c >= nch) break;
        if (threadIdx.x == 0) fetch_chunk(plan, n, nch, kTicketPack, s_d[db ^ 1]);
        const u64 i = d.i, p0 = d.p0, p1 = d.p1;
        const u64 cs = v.cls_of[i];
        const u64 row = v.row_of[i];
        u64* rowm = XM ? XM + row * stride_m + v.kbase[0] : nullptr;
        u64* rows = XS + row * stride_s + v.kbase[cs];
        const u64 bm0 = blk0, bms = cs * v.nwords / kScanBlockWords;
        // two 32-value groups per warp in flight: both groups' values and
        // class-0 words are loaded before either is used
        for (u64 base = p0 + (threadIdx.x & ~31u); base < p1; base += 2 * kIngestThreads) {
            const u64 posA = base + (threadIdx.x & 31), posB = posA + kIngestThreads;
            u64 d[2] = {~0ull, ~0ull};
            if (posA < p1) d[0] = __ldcs(ids + posA) - lo;
            if (posB < p1) d[1] = __ldcs(ids + posB) - lo;
            u64 m0[2] = {0ull, 0ull};
            #pragma unroll
            for (int g = 0; g < 2; ++g)
                if (d[g] < width) m0[g] = v.cls[d[g] >> 6];
            #pragma unroll
            for (int g = 0; g < 2; ++g) {
                u64 key = ~0ull, bit = 0ull;
                if (d[g] < width) {
                    const u64 w0 = d[g] >> 6, sh = d[g] & 63, low = (1ull << sh) - 1ull;
                    if ((m0[g] >> sh) & 1ull) {
                        const u64 r = v.boff[w0 / kScanBlockWords] - v.boff[bm0] + (u64)v.dir[w0] +
                                      (u64)__popcll(m0[g] & low);
                        key = r >> 6;  // class 0: keys below 2^62
                        bit = 1ull << (r & 63);
                    } else {
                        const u64 ws = cs * v.nwords + w0, ms = v.cls[ws];
                        if ((ms >> sh) & 1ull) {
                            const u64 r = v.boff[ws / kScanBlockWords] - v.boff[bms] + (u64)v.dir[ws] +
                                          (u64)__popcll(ms & low);
                            key = (1ull << 62) | (r >> 6);
                            bit = 1ull << (r & 63);
                        }
                    }
                }
                const bool lead = segmented_or<u64>(key, bit);
                if (lead && bit) {
                    if (key >> 62) atomicOr((unsigned long long*)(rows + (key & ((1ull << 62) - 1))), bit);
                    else atomicOr((unsigned long long*)(rowm + key), bit);
                }
            }
        }
        __syncthreads();
    }
}

// The smallest first value and the largest last value over the non-empty
// samples (for sorted samples: the collection's minimum and maximum); out
// must hold {~0, 0} before.  One CTA.
__global__ void __launch_bounds__(kPlanThreads)
k_first_last(const u64* __restrict__ offsets, const u64* __restrict__ ids, u64 n, u64* out)
{
    __shared__ unsigned long long s_min, s_max;
    if (threadIdx.x == 0) { s_min = ~0ull; s_max = 0ull; }
    __syncthreads();
    unsigned long long mn = ~0ull, mx = 0ull;
    for (u64 i = threadIdx.x; i < n; i += blockDim.x) {
        const u64 a = offsets[i], e = offsets[i + 1];
        if (e > a) {
            mn = min(mn, (unsigned long long)ids[a]);
            mx = max(mx, (unsigned long long)ids[e - 1]);
        }
    }
    atomicMin(&s_min, mn);
    atomicMax(&s_max, mx);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMin((unsigned long long*)out, s_min);
        atomicMax((unsigned long long*)out + 1, s_max);
    }
}

inline unsigned grid_for_chunks(u64 max_chunks, int sms)
{
    u64 g = (u64)sms * 8;
    if (max_chunks < g) g = max_chunks;
    return (unsigned)(g ? g : 1);
}

}  // namespace

cudaError_t launch_plan(const u64* offsets, const u64* ids, u64 n, u64 lo, u64 hi, bool full,
                        Plan plan, cudaStream_t st, const u32* perm, const u64* ends)
{
    k_plan<<<1, kPlanThreads, 0, st>>>(offsets, ids, n, lo, hi, full ? 1 : 0, plan, perm, ends);
    return cudaGetLastError();
}

cudaError_t launch_validate(const u64* offsets, const u64* ids, u64 n, Plan plan, u64 max_chunks,
                            int id_bits, u64* sizes, u32* err, u64* maxid, u64* minid, int sms,
                            cudaStream_t st, u64 err_stride)
{
    k_validate<<<grid_for_chunks(max_chunks, sms), kIngestThreads, 0, st>>>(offsets, ids, n, plan, id_bits,
                                                                            sizes, err, maxid, minid, err_stride);
    return cudaGetLastError();
}

cudaError_t launch_filter_tiles(const u64* ids, u64 n, Plan plan, u64 max_chunks, u64 lo, u64 width,
                               u32* bitmaps, u32* twice, const u32* tile_of, int sms, cudaStream_t st)
{
    k_filter<<<grid_for_chunks(max_chunks, sms), kIngestThreads, 0, st>>>(ids, n, plan, lo, width, bitmaps, twice,
                                                                          tile_of, width / 32);
    return cudaGetLastError();
}

cudaError_t launch_filter(const u64* ids, u64 n, Plan plan, u64 max_chunks, u64 lo, u64 width,
                          u32* bitmap, int sms, cudaStream_t st, u32* twice)
{
    k_filter<<<grid_for_chunks(max_chunks, sms), kIngestThreads, 0, st>>>(ids, n, plan, lo, width, bitmap, twice,
                                                                          nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_scan(const u64* bitmap, u64 nwords, u32* dir, u64* bsum, u64* boff, u64* R,
                        cudaStream_t st, u64* ktotal, u64* kbase)
{
    u64 nb = (nwords + kScanBlockWords - 1) / kScanBlockWords;
    if (nb == 0) nb = 1;
    k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, st>>>(bitmap, nwords, dir, bsum);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan_top<<<1, 1024, 0, st>>>(bsum, nb, boff, R, ktotal, kbase);
    return cudaGetLastError();
}

cudaError_t launch_scan_top(const u64* bsum, u64 nb, u64* boff, u64* R, cudaStream_t st)
{
    k_scan_top<<<1, 1024, 0, st>>>(bsum, nb, boff, R, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_pack_full(const u64* ids, u64 n, Plan plan, u64 max_chunks, u64 lo, u64 width,
                             const u64* bitmap, const u32* dir, const u64* boff, u64* X, u64 stride,
                             const u64* Rdev, int sms, cudaStream_t st, const u64* kbase)
{
    k_pack_full<<<grid_for_chunks(max_chunks, sms), kIngestThreads, 0, st>>>(ids, n, plan, lo, width, bitmap, dir,
                                                                            boff, X, stride, kbase, Rdev);
    return cudaGetLastError();
}

cudaError_t launch_pack_classes(const u64* ids, u64 n, Plan plan, u64 max_chunks, u64 lo, u64 width, const u64* cls,
                                const u32* dir, const u64* boff, u64 nwords, const u64* kbase, const u32* cls_of,
                                const u32* row_of, u64* XM, u64 stride_m, u64* XS, u64 stride_s, int sms,
                                cudaStream_t st)
{
    ClassView v{cls, dir, boff, kbase, nwords, cls_of, row_of};
    k_pack_classes<<<grid_for_chunks(max_chunks, sms), kIngestThreads, 0, st>>>(ids, n, plan, lo, width, v, XM,
                                                                                stride_m, XS, stride_s);
    return cudaGetLastError();
}

cudaError_t launch_first_last(const u64* offsets, const u64* ids, u64 n, u64* out, cudaStream_t st)
{
    k_first_last<<<1, kPlanThreads, 0, st>>>(offsets, ids, n, out);
    return cudaGetLastError();
}

cudaError_t launch_zero_rows(u64* X, u64 rows, u64 stride, u64 words, int sms, cudaStream_t st)
{
    if (rows == 0 || words == 0) return cudaSuccess;
    u64 total = rows * words;
    u64 g = (total + 255) / 256;
    u64 cap = (u64)sms * 16;
    if (g > cap) g = cap;
    k_zero_rows<<<(unsigned)g, 256, 0, st>>>(X, rows, stride, words);
    return cudaGetLastError();
}

cudaError_t launch_pack(const u64* ids, u64 n, Plan plan, u64 max_chunks, u64 lo, u64 width,
                        const u64* bitmap, const u32* dir, const u64* boff, u64* X, u64 stride,
                        u64* batch_sizes, int sms, cudaStream_t st, const u64* kbase, u64 wstride)
{
    k_pack<<<grid_for_chunks(max_chunks, sms), kIngestThreads, 0, st>>>(ids, n, plan, lo, width, bitmap, dir,
                                                                        boff, X, stride, batch_sizes, kbase,
                                                                        wstride);
    return cudaGetLastError();
}

}  // namespace jsim
