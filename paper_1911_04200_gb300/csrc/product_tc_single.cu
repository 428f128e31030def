// Single-collection tcgen05 product (the all-pairs and product entry points).
// Same arithmetic and roles as the multi-collection kernel in product_tc.cu;
// this is the version validated for one collection per launch.
// Semiring product on the 5th-generation tensor cores (tcgen05, sm_103a):
// C += X X^T over (AND, popcount, +) (Eq. 7), computed exactly as an FP8
// matrix product of 0/1 values.
//
// Every bit of a packed word becomes one e4m3 byte, 0x00 (0.0) or 0x08
// (2^-6, the smallest normal); a product of two such values is 0 or 2^-12,
// and the tensor core sums them into FP32 accumulators held in tensor memory
// (TMEM).  A segment of work accumulates at most 2^22 bit-rows, so every
// accumulator is count * 2^-12 with count < 2^24 - a value FP32 holds
// exactly, as it holds every partial sum on the way; the epilogue scales by
// 2^12, converts to integers and adds them into C.
//
// Work: the tiles of C are 128 x 256 (128 rows on the A side, 256 on the B
// side, both read from X) that touch the upper triangle; each tile's word
// range is cut into stages of 128 bit-rows.  The (tile, stage) units are laid
// out tile-major and one persistent CTA per SM takes an equal contiguous
// share, split into segments at tile boundaries and at the exactness cap.
//
// Roles inside a CTA (17 warps):
//   warps 0-11  unpack: thread p owns row p of every stage (rows 0-127 A,
//               128-383 B); it keeps its packed words four stages ahead in
//               registers (one 16-byte load per stage), waits until the tensor core has released the
//               stage buffer, writes its 128-byte row in the canonical
//               K-major 128-byte-swizzle layout (16-byte chunk c of row r at
//               c ^ (r % 8)), fences the generic-to-async proxy; one lane per
//               warp then arrives on the buffer's `full` barrier;
//   warp 12     one lane issues 4 tcgen05.mma (M=128, N=256, K=32) per stage
//               into one of two TMEM accumulators and commits them to the
//               buffer's `empty` barrier, and each finished segment to the
//               accumulator's `acc_full` barrier;
//   warps 13-16 epilogue: wait for `acc_full`, read the accumulator with
//               tcgen05.ld (each warp its 32 TMEM lanes), add it into C and
//               release it through `acc_empty`.
// Four 48 KiB stage buffers; two 256-column accumulators, so the epilogue of
// one segment overlaps the MMAs of the next.  Every wait is bounded (clock64
// budget, plus a CTA-wide abort flag); on time-out the CTA raises the error
// word, waits (bounded) for its issued MMAs, frees its TMEM and leaves.
#include <algorithm>
#include "common.cuh"

namespace jsim {

namespace {

constexpr int kProducerWarps = 12;
constexpr int kMmaWarp = 12;
constexpr int kEpiWarp0 = 13;
constexpr int kWarps = 17;
constexpr int kThreads = kWarps * 32;          // 544
constexpr int kM = 128;                        // A-side rows per tile
constexpr int kN = 256;                        // B-side rows per tile
constexpr int kRows = kM + kN;                 // rows unpacked per stage (one per producer thread)
static_assert(kRows == kProducerWarps * 32, "one row per producer thread");
static_assert(kEpiWarp0 % 4 == 1, "epilogue warp e reads TMEM lanes of warp rank (kEpiWarp0 + e) % 4");
// Build-time tuning: bit-rows per stage (JSIM_TC_KBITS, 128 or 256; 256
// measured ~10 % faster on GB300: half the barrier round trips and fences
// per packed word, with two 96 KiB stage buffers instead of four of 48 KiB).
#ifndef JSIM_TC_KBITS
#define JSIM_TC_KBITS 256
#endif
constexpr int kStageBits = JSIM_TC_KBITS;      // bit-rows per stage: kAtoms 128-byte swizzle atom columns
constexpr int kAtoms = kStageBits / 128;
static_assert(kAtoms == 1 || kAtoms == 2, "one or two atom columns per stage");
constexpr int kStageWords = kStageBits / 64;
constexpr int kBlkBytes = 128;
constexpr int kAtomA = kM * kBlkBytes;         // one atom column of A: 16 KiB
constexpr int kAtomB = kN * kBlkBytes;         // one atom column of B: 32 KiB
constexpr int kABytes = kAtoms * kAtomA;
constexpr int kStageBytes = kAtoms * kRows * kBlkBytes;  // 48 KiB per atom column
constexpr int kBufs = 4 / kAtoms;
constexpr int kAhead = 4;                      // stages of packed words held in registers
constexpr int kSmemBytes = kBufs * kStageBytes + 1024;  // + alignment slack
static_assert(kSmemBytes <= 232448, "fits the per-CTA shared-memory limit");
constexpr int kTmemCols = 512;                 // two 256-column FP32 accumulators
constexpr u64 kMaxSegStages = (1ull << 22) / kStageBits;
constexpr u32 kErrTimeout = 4u;

// instruction descriptor: kind::f8f6f4, D = F32, A = B = E4M3, both K-major,
// N = 256 (bits 17..22 hold N/8), M = 128 (bits 24..28 hold M/16)
constexpr u32 kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((u32)(kN >> 3) << 17) | ((u32)(kM >> 4) << 24);

__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, K-major, 128-byte swizzle: start address,
// leading byte offset 16 (unused by swizzled K-major), stride byte offset
// 1024 (next 8-row group), descriptor version 1, layout SWIZZLE_128B (2)
__device__ __forceinline__ u64 sw128_desc(u32 saddr)
{
    return (u64)((saddr & 0x3FFFFu) >> 4) | ((u64)1 << 16) | ((u64)(1024 >> 4) << 32) | ((u64)1 << 46) |
           ((u64)2 << 61);
}

__device__ __forceinline__ void mbar_init(u64* bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(u64* bar)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" :: "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity)
{
    u32 ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `parity`; false on time-out or when another
// role has already aborted the CTA.
__device__ __forceinline__ bool mbar_wait(u64* bar, u32 parity, long long budget, volatile int* abort_flag)
{
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > budget) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// 4 bits -> 4 e4m3 bytes: bit i -> byte i = 0x08 (2^-6) or 0x00.  The
// multiplier's terms place bit i at 3 + i + 7j; only j = i lands on a byte's
// bit 3 (3 + 8i), and no two terms share a position, so nothing carries.
__device__ __forceinline__ u32 expand4(u32 nib)
{
    return (nib * 0x01020408u) & 0x08080808u;
}

__device__ __forceinline__ void tmem_ld32(u32 taddr, u32 (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// tile t -> first row and column over 128 x 256 tiles with rows [128 ti, +128)
// and columns [256 tj, +256) that hold at least one pair i <= j (ti <= 2 tj + 1)
__device__ __forceinline__ void tc_tile(u64 t, u64 TM, u64& r0, u64& c0)
{
    u64 j = 0;
    for (;;) {
        u64 cnt = min(TM, 2 * j + 2);
        if (t < cnt) break;
        t -= cnt;
        ++j;
    }
    r0 = t * kM;
    c0 = j * kN;
}

// The CTA's work.  The stage range of every tile is cut into chunks of L
// stages; chunk k's units (tile, stage) are laid out tile-major and CTA c
// takes the c-th of G equal contiguous shares.  Every CTA therefore walks the
// chunks in the same order and at the same pace, so at any time all CTAs
// read the same window of L stages of every row (it stays in L2), and a CTA
// meets the same one or two tiles in every chunk, so their accumulators
// persist across chunks.
struct WorkIter {
    u64 tiles, nst, L, G, c, KC;
    u64 k, Lk, u, uend;
    __device__ __forceinline__ void init(u64 tiles_, u64 nst_, u64 L_, u64 G_, u64 c_)
    {
        tiles = tiles_; nst = nst_; L = L_; G = G_; c = c_;
        KC = (nst + L - 1) / L;
        k = ~0ull; u = uend = Lk = 0;
    }
    // next segment (a run of stages of one tile); false at the end
    __device__ __forceinline__ bool next(u64& tile, u64& kst, u64& len)
    {
        while (u >= uend) {
            k = (k == ~0ull) ? 0 : k + 1;
            if (k >= KC) return false;
            Lk = min(L, nst - k * L);
            const u64 Uk = tiles * Lk;
            u = c * Uk / G;
            uend = (c + 1) * Uk / G;
        }
        tile = u / Lk;
        const u64 s_in = u - tile * Lk;
        const u64 e = min(uend, (tile + 1) * Lk);
        len = e - u;
        kst = k * L + s_in;
        u = e;
        return true;
    }
};

// Accumulator bookkeeping shared (replayed identically) by the MMA warp and
// the epilogue warps: two TMEM slots tagged with a tile; a segment of a tile
// already in a slot accumulates there, otherwise a free slot or the less
// recently used one is taken (flushing it first).  A slot is also flushed
// before its accumulated stages would pass the exactness cap.
struct Slots {
    u64 tile[2];
    u64 fill[2];
    u32 flushes[2];
    int last;
    __device__ __forceinline__ void init()
    {
        tile[0] = tile[1] = ~0ull;
        fill[0] = fill[1] = 0;
        flushes[0] = flushes[1] = 0;
        last = 1;
    }
    __device__ __forceinline__ int pick(u64 t) const
    {
        if (tile[0] == t) return 0;
        if (tile[1] == t) return 1;
        if (tile[0] == ~0ull) return 0;
        if (tile[1] == ~0ull) return 1;
        return 1 - last;
    }
    // does slot s have to be flushed before a segment of tile t, len stages?
    __device__ __forceinline__ bool needs_flush(int s, u64 t, u64 len) const
    {
        return tile[s] != ~0ull && (tile[s] != t || fill[s] + len > kMaxSegStages);
    }
};

template <typename CT>
__global__ void __launch_bounds__(kThreads, 1)
k_prod_tc1(const u64* __restrict__ X, u64 stride, u64 n, u64 W, u64 TM, u64 tiles, u64 L, CT* __restrict__ C,
          u64 ldc, u32* err, long long budget, int vec16)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) u64 full_bar[kBufs], empty_bar[kBufs], accf_bar[2], acce_bar[2], done_bar;
    __shared__ u32 tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const u64 nst = (W + kStageWords - 1) / kStageWords;
    // stages of this CTA (sum of its shares over all chunks)
    u64 T = 0;
    {
        const u64 KC = (nst + L - 1) / L;
        for (u64 k = 0; k < KC; ++k) {
            const u64 Uk = tiles * min(L, nst - k * L);
            T += (blockIdx.x + 1) * Uk / gridDim.x - blockIdx.x * Uk / gridDim.x;
        }
    }
    if (T == 0) return;  // uniform per CTA, before any TMEM or barrier use

    const u32 raw = smem_u32(smem_raw);
    const u32 base = (raw + 1023u) & ~1023u;
    unsigned char* sm = smem_raw + (base - raw);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_u32(&tmem_slot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 32) {
        for (int b = 0; b < kBufs; ++b) {
            mbar_init(&full_bar[b], kProducerWarps);
            mbar_init(&empty_bar[b], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf_bar[a], 1);
            mbar_init(&acce_bar[a], 4 * 32);
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const u32 tmem = tmem_slot;
    volatile int* abort_v = &abort_flag;

    if (warp < kProducerWarps) {
        // ---------------- unpack producers ----------------
        const int p = tid;  // row of every stage this thread writes
        const bool is_a = p < kM;
        const int row = is_a ? p : p - kM;
        // atom column a of this row: row_off + a * atom_step
        const u32 row_off = (u32)((is_a ? 0 : kABytes) + row * kBlkBytes);
        const u32 atom_step = (u32)(is_a ? kAtomA : kAtomB);
        u64 ring[kAhead][kStageWords];
        // position of the next fetch: the current segment's tile (first row
        // and column), stage, and stages left in it
        WorkIter fit;
        fit.init(tiles, nst, L, gridDim.x, blockIdx.x);
        u64 f_tile = ~0ull, f_kst = 0, f_left = 0, f_r0 = 0, f_c0 = 0;
        // packed words of this thread's row at the next fetch position (0 past the end)
        auto fetch = [&](u64 (&v)[kStageWords]) {
            #pragma unroll
            for (int q = 0; q < kStageWords; ++q) v[q] = 0ull;
            if (f_left == 0) {
                u64 tile;
                if (!fit.next(tile, f_kst, f_left)) return;
                if (tile != f_tile) { tc_tile(tile, TM, f_r0, f_c0); f_tile = tile; }
            }
            u64 grow = is_a ? f_r0 + row : f_c0 + row;
            u64 gk = f_kst * kStageWords;
            if (grow < n) {
                const u64* src = X + grow * stride + gk;
                #pragma unroll
                for (int q = 0; q < kStageWords; q += 2) {
                    if (vec16 && gk + q + 1 < W) {
                        // two words of the stage in one 16-byte load
                        asm volatile("ld.global.nc.v2.u64 {%0,%1}, [%2];\n"
                                     : "=l"(v[q]), "=l"(v[q + 1]) : "l"(src + q));
                    } else {
                        if (gk + q < W) v[q] = __ldg(src + q);
                        if (gk + q + 1 < W) v[q + 1] = __ldg(src + q + 1);
                    }
                }
            }
            --f_left;
            ++f_kst;
        };
        #pragma unroll
        for (int a = 0; a < kAhead; ++a) fetch(ring[a]);
        bool ok = true;
        for (u64 t0 = 0; t0 < T && ok; t0 += kAhead) {
            // ring slot a holds stage t0 + a; static indices keep the
            // prefetched words in registers without moves
            #pragma unroll
            for (int a = 0; a < kAhead; ++a) {
                const u64 t = t0 + a;
                if (t >= T || !ok) break;
                const int b = (int)(t % kBufs);
                if (t >= kBufs && !mbar_wait(&empty_bar[b], (u32)((t / kBufs - 1) & 1), budget, abort_v)) {
                    ok = false;
                    break;
                }
                #pragma unroll
                for (int at = 0; at < kAtoms; ++at) {
                    unsigned char* rowp = sm + b * kStageBytes + row_off + at * atom_step;
                    #pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        // bits 128 at + 16c .. +15 of the stage row -> 16 bytes
                        const u64 wv = ring[a][2 * at + (c >> 2)];
                        const u32 half = (c & 2) ? (u32)(wv >> 32) : (u32)wv;
                        const int sh = (c & 1) * 16;
                        uint4 o;
                        o.x = expand4((half >> sh) & 15u);
                        o.y = expand4((half >> (sh + 4)) & 15u);
                        o.z = expand4((half >> (sh + 8)) & 15u);
                        o.w = expand4((half >> (sh + 12)) & 15u);
                        *(uint4*)(rowp + ((c ^ (row & 7)) << 4)) = o;
                    }
                }
                // every writer fences its generic-proxy stores for the async
                // proxy; the warp converges, and one lane arrives for it
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&full_bar[b]);
                fetch(ring[a]);
            }
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            WorkIter it;
            it.init(tiles, nst, L, gridDim.x, blockIdx.x);
            Slots sl;
            sl.init();
            u64 t = 0, tile, kst, len;
            bool ok = true;
            while (ok && it.next(tile, kst, len)) {
                const int sidx = sl.pick(tile);
                if (sl.needs_flush(sidx, tile, len)) {
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                                 :: "r"(smem_u32(&accf_bar[sidx])) : "memory");
                    sl.flushes[sidx] += 1;
                    sl.tile[sidx] = ~0ull;
                }
                bool fresh = false;
                if (sl.tile[sidx] == ~0ull) {
                    // reuse of a flushed slot waits until the epilogue has read it
                    if (sl.flushes[sidx] > 0 &&
                        !mbar_wait(&acce_bar[sidx], (sl.flushes[sidx] - 1) & 1u, budget, abort_v)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    sl.tile[sidx] = tile;
                    sl.fill[sidx] = 0;
                    fresh = true;
                }
                const u32 dt = tmem + (u32)sidx * 256u;
                for (u64 q = 0; q < len; ++q, ++t) {
                    const int b = (int)(t % kBufs);
                    if (!mbar_wait(&full_bar[b], (u32)((t / kBufs) & 1), budget, abort_v)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const u32 abase = base + b * kStageBytes, bbase = abase + kABytes;
                    #pragma unroll
                    for (int k = 0; k < kStageBits / 32; ++k) {
                        // K step k: atom column k / 4, 32-byte slice k % 4
                        u64 da = sw128_desc(abase + (k >> 2) * kAtomA + (k & 3) * 32);
                        u64 db = sw128_desc(bbase + (k >> 2) * kAtomB + (k & 3) * 32);
                        u32 accum = (fresh && q == 0 && k == 0) ? 0u : 1u;
                        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
                                     :: "r"(dt), "l"(da), "l"(db), "r"(kIdesc), "r"(accum) : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                                 :: "r"(smem_u32(&empty_bar[b])) : "memory");
                }
                sl.fill[sidx] += len;
                sl.last = sidx;
            }
            if (ok) {
                for (int sidx = 0; sidx < 2; ++sidx) {
                    if (sl.tile[sidx] == ~0ull) continue;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                                 :: "r"(smem_u32(&accf_bar[sidx])) : "memory");
                }
            }
            // every MMA this thread issued completes before this arrival
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         :: "r"(smem_u32(&done_bar)) : "memory");
        }
        __syncwarp();
    } else {
        // ---------------- epilogue ----------------
        const int e = (warp - kEpiWarp0 + 1) & 3;  // TMEM lane quarter of this warp (warp % 4)
        // drain slot sidx holding `tile` (its n-th flush); false on abort
        auto drain = [&](int sidx, u64 tile, u32 nth) -> bool {
            int got = 0;
            if (lane == 0) got = mbar_wait(&accf_bar[sidx], nth & 1u, budget, abort_v) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);  // the warp follows one verdict
            if (!got) return false;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            u64 r0, c0;
            tc_tile(tile, TM, r0, c0);
            const u64 i = r0 + (u64)(e * 32 + lane);
            #pragma unroll 1
            for (int cb = 0; cb < kN / 32; ++cb) {
                u32 r[32];
                tmem_ld32(tmem + ((u32)(e * 32) << 16) + (u32)sidx * 256u + (u32)(cb * 32), r);
                if (i < n) {
                    #pragma unroll
                    for (int x = 0; x < 32; ++x) {
                        u64 j = c0 + cb * 32 + x;
                        // accumulator = count * 2^-12 (operands 2^-6), exact below 2^24 * 2^-12
                        u32 v = (u32)(__uint_as_float(r[x]) * 4096.0f);
                        if (j < n && i <= j && v) atomicAdd(C + i * ldc + j, (CT)v);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(&acce_bar[sidx]);
            return true;
        };
        WorkIter it;
        it.init(tiles, nst, L, gridDim.x, blockIdx.x);
        Slots sl;
        sl.init();
        u64 tile, kst, len;
        bool ok = true;
        while (ok && it.next(tile, kst, len)) {
            const int sidx = sl.pick(tile);
            if (sl.needs_flush(sidx, tile, len)) {
                ok = drain(sidx, sl.tile[sidx], sl.flushes[sidx]);
                sl.flushes[sidx] += 1;
                sl.tile[sidx] = ~0ull;
            }
            if (sl.tile[sidx] == ~0ull) {
                sl.tile[sidx] = tile;
                sl.fill[sidx] = 0;
            }
            sl.fill[sidx] += len;
            sl.last = sidx;
        }
        for (int sidx = 0; ok && sidx < 2; ++sidx) {
            if (sl.tile[sidx] == ~0ull) continue;
            ok = drain(sidx, sl.tile[sidx], sl.flushes[sidx]);
            sl.flushes[sidx] += 1;
        }
    }

    // wait (bounded) until every issued MMA has completed, then free TMEM
    if (warp == 0) {
        long long t0 = clock64();
        while (!mbar_try_wait(&done_bar, 0u)) {
            if (clock64() - t0 > budget) { *abort_v = 1; break; }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && *abort_v) atomicOr(err, kErrTimeout);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

template <typename CT>
cudaError_t run(ProductArgs& a, cudaStream_t st)
{
    const u64 TM = (a.n + kM - 1) / kM, TN = (a.n + kN - 1) / kN;
    u64 tiles = 0;
    for (u64 j = 0; j < TN; ++j) tiles += std::min<u64>(TM, 2 * j + 2);
    const u64 nst = (a.W + kStageWords - 1) / kStageWords;
    const u64 total = tiles * nst;
    if (total == 0) return cudaSuccess;
    const u64 grid = std::min<u64>((u64)a.sms, total);
    // chunk length: the window of L stages of all n rows (16 bytes per row
    // per stage) is about 48 MiB, so it stays in L2 while every CTA reads it
    u64 L = (48ull << 20) / ((u64)kStageWords * 8ull * std::max<u64>(a.n, 1));
    L = std::max<u64>(64, std::min<u64>(L, kMaxSegStages));
    cudaError_t e = cudaFuncSetAttribute(k_prod_tc1<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    int clk_khz = 0;
    int clk_dev = 0;
    cudaGetDevice(&clk_dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, clk_dev);
    long long budget = (long long)(clk_khz > 0 ? clk_khz : 2000000) * 1000LL * (long long)a.timeout_ms / 1000LL;
    // 16-byte loads when every stage's two words are 16-byte aligned
    const int vec16 = ((uintptr_t)a.X % 16 == 0 && a.stride % 2 == 0) ? 1 : 0;
    k_prod_tc1<CT><<<(unsigned)grid, kThreads, kSmemBytes, st>>>(a.X, a.stride, a.n, a.W, TM, tiles, L, (CT*)a.C,
                                                                a.ldc, a.err, budget, vec16);
    a.launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t product_tc_single(ProductArgs& a, cudaStream_t st)
{
    return a.count_bits == 64 ? run<u64>(a, st) : run<u32>(a, st);
}

}  // namespace jsim
