// Semiring product on pairs of SMs (tcgen05 with cta_group::2, sm_103a):
// C += X X^T over (AND, popcount, +) (Eq. 7), computed exactly as an FP8
// product of 0/1 values, with the same encoding as the one-SM kernel
// (product_tc_single.cu): a set bit is the e4m3 byte 0x08 = 2^-6, products
// are 2^-12, a segment accumulates at most 2^22 bit-rows, so every FP32
// accumulator is count * 2^-12 with count < 2^24, held exactly.
//
// Why pairs: the unpacking of bits into e4m3 bytes in shared memory is the
// cost that bounds the one-SM kernel.  A 2-SM MMA of M = 256, N = 256 reads
// its A operand as 128 rows from each SM and its B operand as 128 rows from
// each SM, and leaves each SM a 128 x 256 accumulator: every SM unpacks 256
// rows per stage for a 128 x 256 block of C, where the one-SM kernel unpacks
// 384 rows for the same block - a third less unpacking per count.
//
// A cluster of two CTAs (ranks 0 and 1) works on 256 x 256 tiles of C on or
// above the diagonal (tile rows [256 ti, +256), columns [256 tj, +256),
// ti <= tj).  Per stage of 128 bit-rows, CTA r unpacks A rows
// 256 ti + 128 r + [0, 128) and B rows 256 tj + 128 r + [0, 128) into its
// own stage buffer (same offsets in both CTAs).  Roles (kGroups = 1: 13
// warps per CTA):
//   warps 0-7   unpack (with kGroups = 2, two groups of 8 warps taking
//               alternate stages; thread p of a group: row p, A for p < 128,
//               else B), four of its stages of packed words ahead in
//               registers; after writing a stage
//               and fencing for the async proxy, one lane per warp arrives on
//               `full` (rank 0) or on the local `ready` (rank 1), whose
//               completion the rank-1 signal thread forwards to the rank-0
//               `full` (one cluster-scope release per stage, 9 arrivals);
//   warp 8      rank 1: the signal thread; rank 0: one lane issues 8 tcgen05.mma
//               (cta_group::2, M = 256, N = 256, K = 32) per stage into one of
//               two TMEM accumulators and commits them, multicast to both
//               CTAs, to `empty` (stage reusable) and, per finished segment,
//               to `acc_full`;
//   warps 9-12  epilogue in both CTAs: read this CTA's 128 accumulator rows
//               with tcgen05.ld, add them into C, and arrive (a lane per
//               warp) on the rank-0 CTA's `acc_empty` (8 arrivals).
// Three 64 KiB stage buffers per CTA (256 bit-rows: two atom columns).
// Every wait is bounded (clock64 budget,
// plus a CTA-wide abort flag); on time-out the CTA raises the error word,
// waits (bounded) for the MMAs already issued, and both CTAs meet at a
// cluster barrier before TMEM is freed and the CTAs exit.
#include <atomic>
#include <algorithm>
#include "common.cuh"

namespace jsim {

namespace {

// Build-time tuning (JSIM_TC2_GROUPS, JSIM_TC2_BUFS, JSIM_TC2_AHEAD,
// JSIM_TC2_KBITS).  Measured on GB300 (n = 1024 .. 4096): 256 bit-rows per
// stage in three 64 KiB buffers is fastest - 1.46x the 128-bit stages, whose
// per-stage barrier round trips and proxy fences bound the kernel; 384-bit
// stages (two buffers) and a second producer group change little.
#ifndef JSIM_TC2_GROUPS
#define JSIM_TC2_GROUPS 1
#endif
#ifndef JSIM_TC2_BUFS
#define JSIM_TC2_BUFS 3
#endif
// Stages of packed words each producer holds in registers ahead of its
// unpacking (Tbit-ops/s at n = 1024 / 2048 / 4096 / 10,000; 4 ahead:
// 1068 / 1206 / 1241 / 1258, 6: 1064 / 1203 / 1261 / 1287, 8: 1070 / 1203 /
// 1272 / 1289; 2: 983 at n = 1024).
#ifndef JSIM_TC2_AHEAD
#define JSIM_TC2_AHEAD 8
#endif
// L2 window shared by all clusters: JSIM_TC2_WINDOW_MIB of packed words of
// all rows, but at least JSIM_TC2_MIN_STAGES stages per chunk.  Every tile
// switch flushes an accumulator, so for many rows a window that fits L2 is
// too short (157 stages at n = 10,000); for few rows a window beyond L2
// re-reads the panels from DRAM (128 MiB at n = 1024: 2.1x the packed bytes).
// Swept with padded strides (Tbit-ops/s; n = 1024 / 2048 / 4096 / 10,000):
//   48 MiB, >= 512 stages   1063 / 1161 / 1182 / 1231
//   48 MiB, >= 768 stages   1063 / 1157 / 1250 / 1257
//   64 MiB, >= 512 stages   1065 / 1209 / 1180 / 1208
//   48 MiB, no minimum      1060 / 1156 / 1175 / 1077
#ifndef JSIM_TC2_WINDOW_MIB
#define JSIM_TC2_WINDOW_MIB 64
#endif
#ifndef JSIM_TC2_MIN_STAGES
#define JSIM_TC2_MIN_STAGES 768
#endif
#ifndef JSIM_TC2_KBITS
#define JSIM_TC2_KBITS 256
#endif
constexpr int kGroups = JSIM_TC2_GROUPS;          // producer groups, taking alternate stages
constexpr int kGroupWarps = 8;                    // warps per group: one row per thread
constexpr int kProducerWarps = kGroups * kGroupWarps;
constexpr int kMmaWarp = kProducerWarps;
constexpr int kEpiWarp0 = kProducerWarps + 1;
constexpr int kWarps = kProducerWarps + 5;
constexpr int kThreads = kWarps * 32;             // 672
constexpr int kHalf = 128;                        // A rows and B rows per CTA per tile
constexpr int kTile = 256;                        // tile side (rows and columns of C)
static_assert(2 * kHalf == kGroupWarps * 32, "one row per producer thread");

static_assert(kEpiWarp0 % 4 == 1, "epilogue warp e reads TMEM lanes of warp rank (kEpiWarp0 + e) % 4");
constexpr int kStageBits = JSIM_TC2_KBITS;        // bit-rows per stage: kAtoms 128-byte swizzle atom columns
constexpr int kAtoms = kStageBits / 128;
static_assert(kAtoms >= 1 && kAtoms <= 4 && kStageBits % 128 == 0, "whole atom columns per stage");
constexpr int kStageWords = kStageBits / 64;
constexpr int kBlkBytes = 128;
constexpr int kAtom = kHalf * kBlkBytes;          // one atom column of a half (A or B): 16 KiB
constexpr int kABytes = kAtoms * kAtom;
constexpr int kStageBytes = 2 * kAtoms * kAtom;   // 32 KiB per atom column
constexpr int kBufs = JSIM_TC2_BUFS;
constexpr int kAhead = JSIM_TC2_AHEAD;
static_assert(kBufs % kGroups == 0, "stage buffers split evenly over the groups");
constexpr int kSmemBytes = kBufs * kStageBytes + 1024;  // + alignment slack
static_assert(kSmemBytes <= 232448, "fits the per-CTA shared-memory limit");
constexpr int kTmemCols = 512;                    // two 256-column FP32 accumulators
constexpr u64 kMaxSegStages = (1ull << 22) / kStageBits;
constexpr u32 kErrTimeout = 4u;

// instruction descriptor: kind::f8f6f4, D = F32, A = B = E4M3, both K-major,
// N = 256 (bits 17..22 hold N/8), M = 256 across the pair (bits 24..28 hold M/16)
constexpr u32 kIdesc = (1u << 4) | ((u32)(kTile >> 3) << 17) | ((u32)(kTile >> 4) << 24);

__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ u32 cta_rank()
{
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}

// the same shared-memory variable in CTA `rank` of the cluster
__device__ __forceinline__ u32 peer_addr(const void* p, u32 rank)
{
    u32 r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release;\nbarrier.cluster.wait.acquire;\n" ::: "memory");
}

__device__ __forceinline__ u64 sw128_desc(u32 saddr)
{
    return (u64)((saddr & 0x3FFFFu) >> 4) | ((u64)1 << 16) | ((u64)(1024 >> 4) << 32) | ((u64)1 << 46) |
           ((u64)2 << 61);
}

__device__ __forceinline__ void mbar_init(u64* bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}

// arrive on the barrier at cluster address `caddr` (this CTA's or the peer's)
__device__ __forceinline__ void mbar_arrive_cluster(u32 caddr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];\n" :: "r"(caddr) : "memory");
}

__device__ __forceinline__ void mbar_arrive(u64* bar)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" :: "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity)
{
    u32 ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

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

// commit the MMAs issued so far to the barrier at `bar`'s offset in both CTAs
__device__ __forceinline__ void commit_both(u64* bar)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n"
                 :: "r"(smem_u32(bar)), "h"((unsigned short)3) : "memory");
}

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

// tile t -> (ti, tj), tiles ordered column by column: tj = 0, 1, ..., ti = 0..tj
__device__ __forceinline__ void pair_tile(u64 t, u64& r0, u64& c0)
{
    u64 j = 0;
    while (t > j) {
        t -= j + 1;
        ++j;
    }
    r0 = t * kTile;
    c0 = j * kTile;
}

// Work of a cluster: as in the one-SM kernel, the stage range is cut into
// chunks of L stages, chunk k's (tile, stage) units are laid out tile-major
// and cluster c takes the c-th of G equal contiguous shares; every cluster
// walks the chunks at the same pace, so the window of L stages of all rows is
// shared in L2.
struct WorkIter {
    u64 tiles, nst, L, G, c, KC;
    u64 k, Lk, u, uend;
    __device__ __forceinline__ void init(u64 tiles_, u64 nst_, u64 L_, u64 G_, u64 c_)
    {
        tiles = tiles_; nst = nst_; L = L_; G = G_; c = c_;
        KC = (nst + L - 1) / L;
        k = ~0ull; u = uend = Lk = 0;
    }
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
    __device__ __forceinline__ bool needs_flush(int s, u64 t, u64 len) const
    {
        return tile[s] != ~0ull && (tile[s] != t || fill[s] + len > kMaxSegStages);
    }
};

template <typename CT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
k_prod_tc2(const u64* __restrict__ X, u64 stride, u64 n, u64 W, u64 tiles, u64 L, CT* __restrict__ C, u64 ldc,
           u32* err, long long budget, int vec16)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) u64 full_bar[kBufs], ready_bar[kBufs], empty_bar[kBufs], accf_bar[2], acce_bar[2],
        done_bar;
    __shared__ u32 tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const u32 rank = cta_rank();
    const u64 G = gridDim.x / 2, c = blockIdx.x / 2;  // clusters and this CTA's cluster
    const u64 nst = (W + kStageWords - 1) / kStageWords;
    // stages of this cluster (the same in both CTAs)
    u64 T = 0;
    {
        const u64 KC = (nst + L - 1) / L;
        for (u64 k = 0; k < KC; ++k) {
            const u64 Uk = tiles * min(L, nst - k * L);
            T += (c + 1) * Uk / G - c * Uk / G;
        }
    }
    if (T == 0) return;  // uniform per cluster, before any TMEM, barrier or peer access

    const u32 raw = smem_u32(smem_raw);
    const u32 base = (raw + 1023u) & ~1023u;
    unsigned char* sm = smem_raw + (base - raw);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_u32(&tmem_slot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;\n" ::: "memory");
    }
    if (tid == 32) {
        for (int b = 0; b < kBufs; ++b) {
            mbar_init(&full_bar[b], kGroupWarps + 1);  // rank-0 producer warps + the rank-1 signal
            mbar_init(&ready_bar[b], kGroupWarps);      // rank-1 producer warps
            mbar_init(&empty_bar[b], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf_bar[a], 1);
            mbar_init(&acce_bar[a], 2 * 4);                // epilogue warps of both CTAs
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    cluster_sync();  // both CTAs' barriers exist before any remote arrival
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const u32 tmem = tmem_slot;
    volatile int* abort_v = &abort_flag;

    if (warp < kProducerWarps) {
        // ---------------- unpack producers ----------------
        // group g takes the stages t = g (mod kGroups), so kGroups stages are
        // unpacked at once; thread p of a group owns row p of its stages
        const int g = warp / kGroupWarps;
        const int p = tid - g * kGroupWarps * 32;
        const bool is_a = p < kHalf;
        const int row = is_a ? p : p - kHalf;
        const u32 row_off = (u32)((is_a ? 0 : kABytes) + row * kBlkBytes);
        u64 ring[kAhead][kStageWords];
        WorkIter fit;
        fit.init(tiles, nst, L, G, c);
        u64 f_tile = ~0ull, f_kst = 0, f_left = 0, f_r0 = 0, f_c0 = 0;
        // advance the fetch position by one stage; load this thread's words
        // of it when `load` (0 past the end)
        auto fetch = [&](u64 (&v)[kStageWords], bool load) {
            #pragma unroll
            for (int q = 0; q < kStageWords; ++q) v[q] = 0ull;
            if (f_left == 0) {
                u64 tile;
                if (!fit.next(tile, f_kst, f_left)) return;
                if (tile != f_tile) { pair_tile(tile, f_r0, f_c0); f_tile = tile; }
            }
            const u64 grow = (is_a ? f_r0 : f_c0) + (u64)rank * kHalf + (u64)row;
            const u64 gk = f_kst * kStageWords;
            if (load && grow < n) {
                const u64* src = X + grow * stride + gk;
                #pragma unroll
                for (int q = 0; q < kStageWords; q += 2) {
                    if (vec16 && gk + q + 1 < W) {
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
        // this group's next stage: load it, then skip the other groups' stages
        auto fetch_own = [&](u64 (&v)[kStageWords]) {
            fetch(v, true);
            u64 skip[kStageWords];
            #pragma unroll
            for (int q = 1; q < kGroups; ++q) fetch(skip, false);
        };
        {
            u64 skip[kStageWords];
            for (int q = 0; q < g; ++q) fetch(skip, false);
        }
        #pragma unroll
        for (int a = 0; a < kAhead; ++a) fetch_own(ring[a]);
        bool ok = true;
        for (u64 s0 = 0; ok; s0 += kAhead) {
            #pragma unroll
            for (int a = 0; a < kAhead; ++a) {
                const u64 t = (s0 + a) * kGroups + g;
                if (t >= T || !ok) { ok = false; break; }
                const int b = (int)(t % kBufs);
                if (t >= kBufs && !mbar_wait(&empty_bar[b], (u32)((t / kBufs - 1) & 1), budget, abort_v)) {
                    ok = false;
                    break;
                }
                #pragma unroll
                for (int at = 0; at < kAtoms; ++at) {
                    unsigned char* rowp = sm + b * kStageBytes + row_off + at * kAtom;
                    #pragma unroll
                    for (int cc = 0; cc < 8; ++cc) {
                        const u64 wv = ring[a][2 * at + (cc >> 2)];
                        const u32 half = (cc & 2) ? (u32)(wv >> 32) : (u32)wv;
                        const int sh = (cc & 1) * 16;
                        uint4 o;
                        o.x = expand4((half >> sh) & 15u);
                        o.y = expand4((half >> (sh + 4)) & 15u);
                        o.z = expand4((half >> (sh + 8)) & 15u);
                        o.w = expand4((half >> (sh + 12)) & 15u);
                        *(uint4*)(rowp + ((cc ^ (row & 7)) << 4)) = o;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();
                // rank 0: straight to the MMA's barrier; rank 1: to the local
                // barrier its signal thread forwards (one cluster-scope release
                // per stage instead of one per warp)
                if (lane == 0) mbar_arrive(rank == 0 ? &full_bar[b] : &ready_bar[b]);
                fetch_own(ring[a]);
            }
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer (rank-0 CTA) ----------------
        if (rank == 0 && lane == 0) {
            WorkIter it;
            it.init(tiles, nst, L, G, c);
            Slots sl;
            sl.init();
            u64 t = 0, tile, kst, len;
            bool ok = true;
            while (ok && it.next(tile, kst, len)) {
                const int sidx = sl.pick(tile);
                if (sl.needs_flush(sidx, tile, len)) {
                    commit_both(&accf_bar[sidx]);
                    sl.flushes[sidx] += 1;
                    sl.tile[sidx] = ~0ull;
                }
                bool fresh = false;
                if (sl.tile[sidx] == ~0ull) {
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
                        const u64 da = sw128_desc(abase + (k >> 2) * kAtom + (k & 3) * 32);
                        const u64 db = sw128_desc(bbase + (k >> 2) * kAtom + (k & 3) * 32);
                        const u32 accum = (fresh && q == 0 && k == 0) ? 0u : 1u;
                        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
                                     :: "r"(dt), "l"(da), "l"(db), "r"(kIdesc), "r"(accum) : "memory");
                    }
                    commit_both(&empty_bar[b]);
                }
                sl.fill[sidx] += len;
                sl.last = sidx;
            }
            if (ok) {
                for (int sidx = 0; sidx < 2; ++sidx) {
                    if (sl.tile[sidx] == ~0ull) continue;
                    commit_both(&accf_bar[sidx]);
                }
            }
            commit_both(&done_bar);
        } else if (rank == 1 && lane == 0) {
            // signal: forward each stage's local readiness to the MMA's barrier
            // in the rank-0 CTA (release at cluster scope, after acquiring the
            // producers' release at CTA scope)
            for (u64 t = 0; t < T; ++t) {
                const int b = (int)(t % kBufs);
                if (!mbar_wait(&ready_bar[b], (u32)((t / kBufs) & 1), budget, abort_v)) break;
                mbar_arrive_cluster(peer_addr(&full_bar[b], 0));
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (both CTAs) ----------------
        const int e = (warp - kEpiWarp0 + 1) & 3;  // TMEM lane quarter of this warp (warp % 4)
        auto drain = [&](int sidx, u64 tile, u32 nth) -> bool {
            int got = 0;
            if (lane == 0) got = mbar_wait(&accf_bar[sidx], nth & 1u, budget, abort_v) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) return false;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            u64 r0, c0;
            pair_tile(tile, r0, c0);
            const u64 i = r0 + (u64)rank * kHalf + (u64)(e * 32 + lane);
            #pragma unroll 1
            for (int cb = 0; cb < kTile / 32; ++cb) {
                u32 r[32];
                tmem_ld32(tmem + ((u32)(e * 32) << 16) + (u32)sidx * 256u + (u32)(cb * 32), r);
                if (i < n) {
                    #pragma unroll
                    for (int x = 0; x < 32; ++x) {
                        const u64 j = c0 + cb * 32 + x;
                        const u32 v = (u32)(__uint_as_float(r[x]) * 4096.0f);
                        if (j < n && i <= j && v) atomicAdd(C + i * ldc + j, (CT)v);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(peer_addr(&acce_bar[sidx], 0));
            return true;
        };
        WorkIter it;
        it.init(tiles, nst, L, G, c);
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

    // every MMA of the pair has completed (bounded wait), both CTAs are done
    // with each other's barriers, then TMEM is freed
    if (warp == 0) {
        long long t0 = clock64();
        while (!mbar_try_wait(&done_bar, 0u)) {
            if (clock64() - t0 > budget) { *abort_v = 1; break; }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && *abort_v) atomicOr(err, kErrTimeout);
    cluster_sync();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

template <typename CT>
cudaError_t run(ProductArgs& a, cudaStream_t st)
{
    const u64 TT = (a.n + kTile - 1) / kTile;
    const u64 tiles = TT * (TT + 1) / 2;
    const u64 nst = (a.W + kStageWords - 1) / kStageWords;
    const u64 total = tiles * nst;
    if (total == 0) return cudaSuccess;
    u64 L = ((u64)JSIM_TC2_WINDOW_MIB << 20) / ((u64)kStageWords * 8ull * std::max<u64>(a.n, 1));
    L = std::max<u64>(JSIM_TC2_MIN_STAGES, std::min<u64>(L, kMaxSegStages));
    cudaError_t e = cudaFuncSetAttribute(k_prod_tc2<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    // as many clusters as can be resident at once (a GPC with an odd number
    // of free SMs leaves one unused), so no cluster waits for another's SMs
    int dev = 0;
    cudaGetDevice(&dev);
    static std::atomic<int> resident_by_dev[kMaxDevices];
    int resident = dev < kMaxDevices ? resident_by_dev[dev].load(std::memory_order_relaxed) : 0;
    if (resident == 0) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)a.sms & ~1u);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = kSmemBytes;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k_prod_tc2<CT>, &cfg) != cudaSuccess || nc < 1) {
            cudaGetLastError();
            nc = a.sms / 2;
        }
        resident = nc;
        if (dev < kMaxDevices) resident_by_dev[dev].store(nc, std::memory_order_relaxed);
    }
    const u64 clusters = std::min<u64>((u64)std::min(resident, a.sms / 2), total);
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    long long budget = (long long)(clk_khz > 0 ? clk_khz : 2000000) * 1000LL * (long long)a.timeout_ms / 1000LL;
    const int vec16 = ((uintptr_t)a.X % 16 == 0 && a.stride % 2 == 0) ? 1 : 0;
    k_prod_tc2<CT><<<(unsigned)(2 * clusters), kThreads, kSmemBytes, st>>>(a.X, a.stride, a.n, a.W, tiles, L,
                                                                          (CT*)a.C, a.ldc, a.err, budget, vec16);
    a.launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t product_tc_pair(ProductArgs& a, cudaStream_t st)
{
    return a.count_bits == 64 ? run<u64>(a, st) : run<u32>(a, st);
}

}  // namespace jsim
