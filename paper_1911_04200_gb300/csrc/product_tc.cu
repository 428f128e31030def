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
// Work: the tiles of C are 128 x TN (TN = 256 or 128; 128 rows on the A
// side, TN on the B side, both read from X) that touch the upper triangle;
// each tile's word range is cut into stages of 256 bit-rows.  The (job, tile, stage) units of
// all collections of a launch are laid out job-major, then tile-major, and
// one persistent CTA per SM takes an equal contiguous share, split into
// segments at tile boundaries and at the exactness cap.
//
// Roles inside a CTA ((128 + TN) / 32 + 5 warps):
//   producers   unpack: thread p owns row p of every stage (rows 0-127 A,
//               the rest B); it keeps its packed words four stages ahead in
//               registers (16-byte loads), waits until the tensor core has
//               released the stage buffer, writes its row's two 128-byte
//               atom columns in the canonical K-major 128-byte-swizzle layout
//               (16-byte chunk c of row r at c ^ (r % 8)), fences the
//               generic-to-async proxy; one lane per warp then arrives on the
//               buffer's `full` barrier.  On a diagonal tile (TN = 128, rows
//               = columns) the B operand is the A operand, and the A-side and
//               B-side threads of a row write one atom column each;
//   MMA warp    one lane issues 8 tcgen05.mma (M=128, N=TN, K=32) per stage
//               into one of two TMEM accumulators and commits them to the
//               buffer's `empty` barrier, and each finished segment to the
//               accumulator's `acc_full` barrier;
//   4 epilogue  wait for `acc_full`, read the accumulator with tcgen05.ld
//   warps       (each warp its 32 TMEM lanes), add it into C and release it
//               through `acc_empty`.
// Two (TN = 256) or three (TN = 128) stage buffers; two TN-column
// accumulators, so the epilogue of one segment overlaps the MMAs of the
// next.  Every wait is bounded (clock64
// budget, plus a CTA-wide abort flag); on time-out the CTA raises the error
// word, waits (bounded) for its issued MMAs, frees its TMEM and leaves.
#include <algorithm>
#include <vector>
#include "common.cuh"
#include "product_tc_sched.cuh"

namespace jsim {

namespace {

using tcs::kM;
using tcs::kStageBits;
using tcs::kStageWords;
using tcs::kMaxSegStages;
using tcs::kMaxJobs;
using tcs::JobInfo;
using tcs::Seg;
using tcs::WorkIter;
using tcs::Slots;
using tcs::job_tiles;
using tcs::tc_tile;
constexpr int kAtoms = kStageBits / 128;
constexpr int kBlkBytes = 128;
constexpr int kAtomA = kM * kBlkBytes;         // one atom column of A: 16 KiB
constexpr int kABytes = kAtoms * kAtomA;
constexpr int kAhead = 4;                      // stages of packed words held in registers
constexpr u32 kErrTimeout = 4u;

// The kernel's shape for tiles of 128 x TN (TN = 256 or 128).  One producer
// thread per unpacked row (128 + TN), one MMA warp, four epilogue warps; two
// TMEM accumulators of TN columns.  With TN = 128 a stage is two thirds the
// size, so three stage buffers fit.  DG (TN = 128): every tile of the launch
// is diagonal and a stage holds the A rows only - of SB = 512 bit-rows (four
// atom columns, the two producer threads of a row writing two each), so the
// per-stage costs are paid half as often; three buffers.
template <int TN, bool DG = false, int SB = kStageBits>
struct Shape {
    static constexpr int kN = TN;
    static constexpr int kRows = kM + TN;                  // rows unpacked per stage
    static constexpr int kProducerWarps = kRows / 32;
    static constexpr int kMmaWarp = kProducerWarps;
    static constexpr int kEpiWarp0 = kProducerWarps + 1;
    static constexpr int kWarps = kEpiWarp0 + 4;
    static constexpr int kThreads = kWarps * 32;
    static constexpr int kAtomB = TN * kBlkBytes;          // one atom column of B
    static constexpr int kSB = SB;                         // bit-rows per stage
    static constexpr int kSW = SB / 64;                    // packed words per stage
    static constexpr int kAtomsS = SB / 128;               // atom columns per stage
    static constexpr int kStageBytes = DG ? kAtomsS * kAtomA : kAtoms * kRows * kBlkBytes;
    static constexpr int kBufs = DG ? 3 : TN == 128 ? 3 : 2;
    static constexpr int kSmemBytes = kBufs * kStageBytes + 1024;  // + alignment slack
    static constexpr int kTmemCols = 2 * TN;               // two TN-column FP32 accumulators
    // instruction descriptor: kind::f8f6f4, D = F32, A = B = E4M3, both
    // K-major, N = TN (bits 17..22 hold N/8), M = 128 (bits 24..28 hold M/16)
    static constexpr u32 kIdesc =
        (1u << 4) | (0u << 7) | (0u << 10) | ((u32)(TN >> 3) << 17) | ((u32)(kM >> 4) << 24);
    static_assert(kRows % 32 == 0, "one row per producer thread");
    static_assert(kEpiWarp0 % 4 == 1, "epilogue warp e reads TMEM lanes of warp rank (kEpiWarp0 + e) % 4");
    static_assert(kSmemBytes + 9 * 1024 <= 232448, "fits the per-CTA shared-memory limit");
    static_assert(TN == 128 || TN == 256, "tile widths");
    static_assert(!DG || TN == kM, "diagonal-only launches have square tiles");
    static_assert(SB == kStageBits || (DG && SB == 2 * kStageBits), "512-bit stages for diagonal-only launches");
};

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

// One independent collection of a launch: its packed words, word count
// (on the host, or on the device when Wdev is set) and count accumulator.
struct TcJob {
    const u64* X;
    const u64* Wdev;
    void* C;
    u64 stride, n, W, ldc;
};
// Kernel parameters: the job table lives in device memory.
struct TcJobs {
    const TcJob* job;
    u32 njobs;
    int vec16;  // 16-byte loads are safe for every job
};

template <typename CT, int TN, bool DG, int SB>
__global__ void __launch_bounds__(Shape<TN, DG, SB>::kThreads, 1)
k_prod_tc(const TcJobs P, u32* err, long long budget)
{
    using S = Shape<TN, DG, SB>;
    constexpr int kSW = S::kSW;                    // packed words per stage
    constexpr u64 kSeg = (1ull << 22) / SB;        // stages per segment under the exactness cap
    constexpr bool kWide = SB == 2 * kStageBits;   // a diagonal row split into two halves of two atom columns
    constexpr int kBufs = S::kBufs, kStageBytes = S::kStageBytes, kAtomB = S::kAtomB;
    constexpr int kProducerWarps = S::kProducerWarps, kMmaWarp = S::kMmaWarp, kEpiWarp0 = S::kEpiWarp0;
    constexpr int kTmemCols = S::kTmemCols;
    constexpr u32 kIdesc = S::kIdesc;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) u64 full_bar[kBufs], empty_bar[kBufs], accf_bar[2], acce_bar[2], done_bar;
    __shared__ u32 tmem_slot;
    __shared__ int abort_flag;
    __shared__ JobInfo ji[kMaxJobs];
    __shared__ u64 s_T;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const u32 njobs = P.njobs;
    if (tid == 0) {
        u64 U = 0;
        for (u32 j = 0; j < njobs; ++j) {
            const TcJob& J = P.job[j];
            const u64 W = J.Wdev ? *(volatile const u64*)J.Wdev : J.W;
            const JobInfo x = tcs::job_info(J.n, W, U, TN, kSW);
            U += x.tiles * x.nst;
            ji[j] = x;
        }
        // stages of this CTA
        s_T = tcs::cta_stages(U, gridDim.x, blockIdx.x);
    }
    __syncthreads();
    const u64 T = s_T;
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
        const u32 row_off = (u32)((is_a ? 0 : kABytes) + row * kBlkBytes);
        const u32 atom_step = (u32)(is_a ? kAtomA : kAtomB);
        u64 ring[kAhead][kStageWords];
        // per ring slot: the stage's tile is diagonal (TN = 128, rows = columns):
        // its B operand is the A operand, and the two threads of a row share
        // its unpack (the A-side thread the first atom column, the B-side
        // thread - which maps to the same row - the second)
        bool diag[kAhead];
        static_assert(kAtoms == 2, "a diagonal row is split into two atom columns");
        // position of the next fetch: the current segment's job, tile (first
        // row and column), stage, and stages left in it
        WorkIter fit;
        fit.init(ji, njobs, gridDim.x, blockIdx.x);
        fit.max_seg = kSeg;
        Seg fs;
        u64 f_key = ~0ull, f_kst = 0, f_left = 0, f_r0 = 0, f_c0 = 0, f_n = 0, f_W = 0, f_stride = 0;
        const u64* f_X = nullptr;
        // packed words of this thread's row at the next fetch position (0 past the end)
        auto fetch = [&](u64 (&v)[kStageWords], bool& dg) {
            #pragma unroll
            for (int q = 0; q < kStageWords; ++q) v[q] = 0ull;
            dg = false;
            if (f_left == 0) {
                if (!fit.next(fs)) return;
                f_kst = fs.kst;
                f_left = fs.len;
                const u64 key = ((u64)fs.job << 40) | fs.tile;
                if (key != f_key) {
                    const TcJob& J = P.job[fs.job];
                    f_X = J.X; f_n = J.n; f_stride = J.stride;
                    f_W = J.Wdev ? *(volatile const u64*)J.Wdev : J.W;
                    tc_tile(fs.tile, ji[fs.job].TM, f_r0, f_c0, TN);
                    f_key = key;
                }
            }
            dg = DG || (TN == kM && f_r0 == f_c0);
            const u64 grow = tcs::fetch_row(p, f_r0, f_c0);  // on a diagonal tile both sides map to row f_r0 + row
            if (grow < f_n) {
                const u64* src = f_X + grow * f_stride;
                #pragma unroll
                for (int q = 0; q < kStageWords; q += 2) {
                    // the words of this thread's atom columns: with 256-bit
                    // stages one column each on a diagonal tile, with 512-bit
                    // stages the A side's first two and the B side's last two
                    if (!kWide && dg && (q >> 1) != (is_a ? 0 : 1)) continue;
                    const int qw = kWide ? q + (is_a ? 0 : kStageWords) : q;
                    u64 w0, w1;
                    const bool in0 = tcs::fetch_word(f_kst, qw, f_W, w0, kSW);
                    const bool in1 = tcs::fetch_word(f_kst, qw + 1, f_W, w1, kSW);
                    if (P.vec16 && in1) {
                        // two words of the stage in one 16-byte load
                        asm volatile("ld.global.nc.v2.u64 {%0,%1}, [%2];\n"
                                     : "=l"(v[q]), "=l"(v[q + 1]) : "l"(src + w0));
                    } else {
                        if (in0) v[q] = __ldg(src + w0);
                        if (in1) v[q + 1] = __ldg(src + w1);
                    }
                }
            }
            --f_left;
            ++f_kst;
        };
        #pragma unroll
        for (int a = 0; a < kAhead; ++a) fetch(ring[a], diag[a]);
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
                    // a diagonal tile's rows go to the A operand only (the MMA
                    // reads them for both): with 256-bit stages atom column 0
                    // from the A-side thread and 1 from the B-side thread of
                    // the row; with 512-bit stages columns 0-1 and 2-3
                    if (!kWide && diag[a] && at != (is_a ? 0 : 1)) continue;
                    const int ga = kWide ? at + (is_a ? 0 : kAtoms) : at;
                    unsigned char* rowp = sm + b * kStageBytes +
                                          (diag[a] ? (u32)(row * kBlkBytes + ga * kAtomA) : row_off + at * atom_step);
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
                fetch(ring[a], diag[a]);
            }
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            WorkIter it;
            it.init(ji, njobs, gridDim.x, blockIdx.x);
            it.max_seg = kSeg;
            Slots sl;
            sl.init();
            sl.max_seg = kSeg;
            u64 t = 0;
            Seg sg;
            bool ok = true;
            while (ok && it.next(sg)) {
                const u64 tile = ((u64)sg.job << 40) | sg.tile, len = sg.len;
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
                const u32 dt = tmem + (u32)sidx * (u32)TN;
                // a diagonal tile (TN = 128, rows = columns) multiplies its A rows by themselves
                u64 r0, c0;
                tc_tile(sg.tile, ji[sg.job].TM, r0, c0, TN);
                const bool dg = DG || (TN == kM && r0 == c0);
                for (u64 q = 0; q < len; ++q, ++t) {
                    const int b = (int)(t % kBufs);
                    if (!mbar_wait(&full_bar[b], (u32)((t / kBufs) & 1), budget, abort_v)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const u32 abase = base + b * kStageBytes, bbase = dg ? abase : abase + kABytes;
                    #pragma unroll
                    for (int k = 0; k < SB / 32; ++k) {
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
        auto drain = [&](int sidx, u64 key, u32 nth) -> bool {
            int got = 0;
            if (lane == 0) got = mbar_wait(&accf_bar[sidx], nth & 1u, budget, abort_v) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);  // the warp follows one verdict
            if (!got) return false;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const u32 jb = (u32)(key >> 40);
            const TcJob& J = P.job[jb];
            CT* C = (CT*)J.C;
            const u64 n = J.n, ldc = J.ldc;
            u64 r0, c0;
            tc_tile(key & ((1ull << 40) - 1), ji[jb].TM, r0, c0, TN);
            const u64 i = r0 + (u64)(e * 32 + lane);
            #pragma unroll 1
            for (int cb = 0; cb < TN / 32; ++cb) {
                u32 r[32];
                tmem_ld32(tmem + ((u32)(e * 32) << 16) + (u32)sidx * (u32)TN + (u32)(cb * 32), r);
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
        it.init(ji, njobs, gridDim.x, blockIdx.x);
        it.max_seg = kSeg;
        Slots sl;
        sl.init();
        sl.max_seg = kSeg;
        Seg sg;
        bool ok = true;
        while (ok && it.next(sg)) {
            const u64 tile = ((u64)sg.job << 40) | sg.tile, len = sg.len;
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

long long wait_budget(int timeout_ms)
{
    int clk_khz = 0;
    int clk_dev = 0;
    cudaGetDevice(&clk_dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, clk_dev);
    return (long long)(clk_khz > 0 ? clk_khz : 2000000) * 1000LL * (long long)timeout_ms / 1000LL;
}

template <typename CT, int TN, bool DG = false, int SB = kStageBits>
cudaError_t launch(const TcJobs& P, int sms, u32* err, int timeout_ms, cudaStream_t st)
{
    using S = Shape<TN, DG, SB>;
    cudaError_t e =
        cudaFuncSetAttribute(k_prod_tc<CT, TN, DG, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmemBytes);
    if (e != cudaSuccess) return e;
    k_prod_tc<CT, TN, DG, SB><<<(unsigned)sms, S::kThreads, S::kSmemBytes, st>>>(P, err, wait_budget(timeout_ms));
    return cudaGetLastError();
}

}  // namespace

cudaError_t product_tc_jobs(const TcJobDesc* jobs, int njobs, void* dev_table, bool upload, int count_bits, int sms,
                            u32* err, int timeout_ms, cudaStream_t st, int* launches, int tile_n, bool diag_only)
{
    if (tile_n != 128 && tile_n != 256) return cudaErrorInvalidValue;
    if (diag_only) {
        // one 128 x 128 tile per job, on the diagonal
        if (tile_n != 128) return cudaErrorInvalidValue;
        for (int q = 0; q < njobs; ++q)
            if (jobs[q].n > (u64)kM) return cudaErrorInvalidValue;
    }
    // the table of every job, copied once to device memory (dev_table holds
    // njobs entries of TcJob); one launch per group of kMaxJobs jobs
    static_assert(sizeof(TcJob) == sizeof(TcJobDesc), "table entry layout");
    std::vector<TcJob> host((size_t)njobs);
    int vec16 = 1;
    for (int q = 0; q < njobs; ++q) {
        const TcJobDesc& d = jobs[q];
        host[q] = TcJob{d.X, d.Wdev, d.C, d.stride, d.n, d.W, d.ldc};
        if ((uintptr_t)d.X % 16 != 0 || d.stride % 2 != 0) vec16 = 0;
    }
    if (njobs == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (upload) {
        e = cudaMemcpyAsync(dev_table, host.data(), sizeof(TcJob) * (size_t)njobs, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    for (int j0 = 0; j0 < njobs; j0 += kMaxJobs) {
        TcJobs P;
        P.job = (const TcJob*)dev_table + j0;
        P.njobs = (u32)std::min(kMaxJobs, njobs - j0);
        P.vec16 = vec16;
        if (diag_only)
            e = count_bits == 64 ? launch<u64, 128, true, 2 * kStageBits>(P, sms, err, timeout_ms, st)
                                 : launch<u32, 128, true, 2 * kStageBits>(P, sms, err, timeout_ms, st);
        else if (tile_n == 128)
            e = count_bits == 64 ? launch<u64, 128>(P, sms, err, timeout_ms, st)
                                 : launch<u32, 128>(P, sms, err, timeout_ms, st);
        else
            e = count_bits == 64 ? launch<u64, 256>(P, sms, err, timeout_ms, st)
                                 : launch<u32, 256>(P, sms, err, timeout_ms, st);
        if (e != cudaSuccess) return e;
        if (launches) *launches += 1;
    }
    return cudaSuccess;
}

namespace {
}  // namespace

bool product_tc_supported(int device)
{
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) return false;
    return major == 10 && minor == 3;
}

cudaError_t product_tc(ProductArgs& a, cudaStream_t st)
{
    return product_tc_single(a, st);
}

}  // namespace jsim

// ---------------------------------------------------------------------------
// Host-side check of the schedule above (no GPU): replays, for every CTA of a
// launch, the unpack threads' fetches, the MMA thread's segments and
// accumulator slots, and the epilogue's drains and C writes, with the same
// __host__ __device__ functions the kernel runs, and checks every address
// against its buffer.
// ---------------------------------------------------------------------------
#include <cstdio>
#include <cstring>

namespace {

struct CheckMsg {
    char* buf;
    size_t cap;
    int fail(int code, const char* fmt, unsigned long long a, unsigned long long b, unsigned long long c)
    {
        if (buf && cap) snprintf(buf, cap, fmt, a, b, c);
        return code;
    }
};

}  // namespace

extern "C" JSIM_API int jsim_check_tc_schedule(uint32_t njobs, const uint64_t* n, const uint64_t* W,
                                               const uint64_t* stride, const uint64_t* rows, uint32_t grid,
                                               uint32_t tile_n, uint32_t stage_bits, char* msg, size_t cap)
{
    using namespace jsim;
    using namespace jsim::tcs;
    CheckMsg m{msg, cap};
    if (msg && cap) msg[0] = 0;
    if (stage_bits == 0) stage_bits = kStageBits;
    if (njobs == 0 || njobs > (uint32_t)kMaxJobs || grid == 0 || !n || !W || !stride || !rows ||
        (tile_n != 128 && tile_n != 256) || (stage_bits != kStageBits && !(stage_bits == 2 * kStageBits && tile_n == 128)))
        return JSIM_ERR_ARG;
    const u64 kn = tile_n;
    const u64 sw = stage_bits / 64, max_seg = (1ull << 22) / stage_bits;
    const int kRows = kM + (int)kn;
    std::vector<JobInfo> ji(njobs);
    u64 U = 0;
    for (u32 j = 0; j < njobs; ++j) {
        if (rows[j] < n[j] || (W[j] > stride[j] && n[j] > 0)) return m.fail(1, "job %llu: rows %llu or W beyond stride %llu", j, rows[j], stride[j]);
        ji[j] = job_info(n[j], W[j], U, kn, sw);
        U += ji[j].tiles * ji[j].nst;
    }
    // every (job, tile, stage) unit must be taken exactly once
    std::vector<unsigned char> seen(U, 0);
    // every pair i <= j of a job must lie in exactly one tile
    for (u32 jb = 0; jb < njobs; ++jb) {
        if (n[jb] == 0 || ji[jb].tiles == 0 || n[jb] > 8192) continue;
        const u64 N = n[jb];
        std::vector<unsigned char> cov(N * N, 0);
        for (u64 t = 0; t < ji[jb].tiles; ++t) {
            u64 r0, c0;
            tc_tile(t, ji[jb].TM, r0, c0, kn);
            for (u64 i = r0; i < r0 + kM && i < N; ++i)
                for (u64 j = std::max(i, c0); j < c0 + kn && j < N; ++j) {
                    if (cov[i * N + j]) return m.fail(2, "job %llu: pair (%llu, %llu) in two tiles", jb, i, j);
                    cov[i * N + j] = 1;
                }
        }
        for (u64 i = 0; i < N; ++i)
            for (u64 j = i; j < N; ++j)
                if (!cov[i * N + j]) return m.fail(3, "job %llu: pair (%llu, %llu) in no tile", jb, i, j);
    }
    for (u64 c = 0; c < grid; ++c) {
        const u64 T = cta_stages(U, grid, c);
        if (T == 0) continue;
        // unpack threads: T fetches that find a segment, then none
        {
            WorkIter fit;
            fit.init(ji.data(), njobs, grid, c);
            fit.max_seg = max_seg;
            Seg fs{};
            u64 left = 0, kst = 0, r0 = 0, c0 = 0;
            u32 job = 0;
            for (u64 t = 0; t < T + 4; ++t) {
                if (left == 0) {
                    if (!fit.next(fs)) {
                        if (t < T) return m.fail(4, "cta %llu: fetch %llu of %llu found no segment", c, t, T);
                        break;
                    }
                    if (t >= T) return m.fail(5, "cta %llu: fetch %llu beyond its %llu stages", c, t, T);
                    kst = fs.kst; left = fs.len; job = fs.job;
                    tc_tile(fs.tile, ji[job].TM, r0, c0, kn);
                }
                for (int p = 0; p < kRows; ++p) {
                    const u64 grow = fetch_row(p, r0, c0);
                    if (grow >= n[job]) continue;
                    for (int q = 0; q < (int)sw; ++q) {
                        u64 w;
                        if (!fetch_word(kst, q, W[job], w, sw)) continue;
                        if (grow >= rows[job] || w >= stride[job])
                            return m.fail(6, "cta %llu: read row %llu word %llu outside the matrix", c, grow, w);
                        if ((q & 1) == 0 && stride[job] % 2 == 0 && ((grow * stride[job] + w) & 1))
                            return m.fail(7, "cta %llu: 16-byte load at row %llu word %llu misaligned", c, grow, w);
                    }
                }
                --left;
                ++kst;
            }
        }
        // MMA thread and epilogue: the same segments and slot decisions
        {
            WorkIter it;
            it.init(ji.data(), njobs, grid, c);
            it.max_seg = max_seg;
            Slots sl;
            sl.init();
            sl.max_seg = max_seg;
            Seg sg{};
            u64 t = 0;
            u32 commits[2] = {0, 0};
            u32 drains[2] = {0, 0};
            auto drain = [&](int sidx, u64 key) -> int {
                const u32 jb = (u32)(key >> 40);
                u64 r0, c0;
                tc_tile(key & ((1ull << 40) - 1), ji[jb].TM, r0, c0, kn);
                for (u64 e = 0; e < 4; ++e)
                    for (u64 lane = 0; lane < 32; ++lane) {
                        const u64 i = r0 + e * 32 + lane;
                        for (u64 col = 0; col < kn; ++col) {
                            const u64 tcol = (u64)sidx * kn + col;
                            if (tcol >= 2 * kn) return m.fail(8, "cta %llu: TMEM column %llu of slot %llu", c, tcol, sidx);
                            const u64 j = c0 + col;
                            if (i < n[jb] && j < n[jb] && i <= j && i * n[jb] + j >= n[jb] * n[jb])
                                return m.fail(9, "cta %llu: C write (%llu, %llu) outside", c, i, j);
                        }
                    }
                drains[sidx] += 1;
                return 0;
            };
            while (it.next(sg)) {
                const u64 key = ((u64)sg.job << 40) | sg.tile;
                const u64 u0 = ji[sg.job].U0 + sg.tile * ji[sg.job].nst + sg.kst;
                for (u64 q = 0; q < sg.len; ++q) {
                    if (u0 + q >= U || seen[u0 + q]) return m.fail(10, "cta %llu: unit %llu taken twice (of %llu)", c, u0 + q, U);
                    seen[u0 + q] = 1;
                }
                const int sidx = sl.pick(key);
                if (sl.needs_flush(sidx, key, sg.len)) {
                    commits[sidx] += 1;
                    if (int r = drain(sidx, sl.tile[sidx])) return r;
                    sl.flushes[sidx] += 1;
                    sl.tile[sidx] = ~0ull;
                }
                if (sl.tile[sidx] == ~0ull) {
                    sl.tile[sidx] = key;
                    sl.fill[sidx] = 0;
                }
                sl.fill[sidx] += sg.len;
                if (sl.fill[sidx] > max_seg)
                    return m.fail(11, "cta %llu: slot %llu holds %llu stages (beyond the exact cap)", c, sidx, sl.fill[sidx]);
                sl.last = sidx;
                t += sg.len;
            }
            for (int sidx = 0; sidx < 2; ++sidx) {
                if (sl.tile[sidx] == ~0ull) continue;
                commits[sidx] += 1;
                if (int r = drain(sidx, sl.tile[sidx])) return r;
            }
            if (t != T) return m.fail(12, "cta %llu: MMA stages %llu, unpacked %llu", c, t, T);
            for (int s = 0; s < 2; ++s)
                if (commits[s] != drains[s]) return m.fail(13, "cta %llu: slot %llu commits %llu != drains", c, s, commits[s]);
        }
    }
    for (u64 u = 0; u < U; ++u)
        if (!seen[u]) return m.fail(14, "unit %llu of %llu taken by no CTA%llu", u, U, 0);
    return 0;
}
