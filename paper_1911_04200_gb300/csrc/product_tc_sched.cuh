// Work schedule of the job-table tcgen05 product (product_tc.cu): which
// (job, tile, stage) units a persistent CTA takes, which rows and words its
// unpack threads read, and how its two TMEM accumulators are assigned.
// Everything here is __host__ __device__, so the host-side schedule check
// (jsim_check_tc_schedule) walks exactly the schedule the kernel runs.
#pragma once
#include "common.cuh"

namespace jsim {
namespace tcs {

constexpr int kM = 128;                        // A-side rows per tile
// B-side rows per tile: 256 (tiles of 128 x 256) or 128 (tiles of 128 x 128,
// whose diagonal tiles unpack their rows once for both operands); the kernel
// and these functions take it as a parameter `kn`.
constexpr int kStageBits = 256;                // bit-rows per stage: two 128-byte swizzle atom columns
                                               // (512 for diagonal-only launches: four; the functions
                                               // below take the stage's words as a parameter)
constexpr int kStageWords = kStageBits / 64;
// a segment accumulates at most 2^22 bit-rows (exact FP32 counts)
constexpr u64 kMaxSegStages = (1ull << 22) / kStageBits;
constexpr int kMaxJobs = 256;

__host__ __device__ __forceinline__ u64 umin(u64 a, u64 b) { return a < b ? a : b; }

// 128 x kn tiles touching the upper triangle of an n x n result: column
// tile j (columns [kn j, +kn)) pairs with row tiles ti < (j + 1) kn / 128
__host__ __device__ __forceinline__ u64 job_tiles(u64 n, u64& TM, u64 kn)
{
    TM = (n + kM - 1) / kM;
    const u64 TN = (n + kn - 1) / kn;
    u64 t = 0;
    for (u64 j = 0; j < TN; ++j) t += umin(TM, (j + 1) * (kn / kM));
    return t;
}

// tile t -> first row r0 and column c0 (tiles column-major, as counted above)
__host__ __device__ __forceinline__ void tc_tile(u64 t, u64 TM, u64& r0, u64& c0, u64 kn)
{
    u64 j = 0;
    for (;;) {
        u64 cnt = umin(TM, (j + 1) * (kn / kM));
        if (t < cnt) break;
        t -= cnt;
        ++j;
    }
    r0 = t * kM;
    c0 = j * kn;
}

// Per-job quantities every CTA derives in its prologue.
struct JobInfo {
    u64 nst;    // stages of every tile of the job (ceil(W / kStageWords))
    u64 tiles;  // 128 x kn tiles touching the upper triangle
    u64 TM;     // 128-row tile count
    u64 U0;     // first unit of the job in the launch-wide unit order
};

__host__ __device__ __forceinline__ JobInfo job_info(u64 n, u64 W, u64 U0, u64 kn, u64 sw = kStageWords)
{
    JobInfo x;
    x.nst = (W + sw - 1) / sw;  // sw words a stage
    x.tiles = job_tiles(n, x.TM, kn);
    if (x.nst == 0) x.tiles = 0;
    x.U0 = U0;
    return x;
}

// stages of CTA c of G over U units
__host__ __device__ __forceinline__ u64 cta_stages(u64 U, u64 G, u64 c)
{
    return (c + 1) * U / G - c * U / G;
}

// A run of stages of one tile of one job.
struct Seg {
    u32 job;
    u64 tile, kst, len;
};

// The CTA's work: the units (job, tile, stage) of all jobs of the launch,
// job-major then tile-major, are split into G equal contiguous shares, one
// per persistent CTA; small collections share a CTA and large ones spread
// over many.  A segment never exceeds the exactness cap.
struct WorkIter {
    const JobInfo* ji;
    u32 njobs;
    u64 u, uend;
    u32 j;
    u64 max_seg = kMaxSegStages;  // stages a segment may hold (2^22 bit-rows)
    __host__ __device__ __forceinline__ void init(const JobInfo* ji_, u32 njobs_, u64 G, u64 c)
    {
        ji = ji_; njobs = njobs_;
        const u64 U = ji[njobs - 1].U0 + ji[njobs - 1].tiles * ji[njobs - 1].nst;
        u = c * U / G;
        uend = (c + 1) * U / G;
        // job holding unit u: last j with U0 <= u
        u32 lo = 0, hi = njobs - 1;
        while (lo < hi) {
            u32 mid = (lo + hi + 1) >> 1;
            if (ji[mid].U0 <= u) lo = mid; else hi = mid - 1;
        }
        j = lo;
    }
    // next segment; false at the end
    __host__ __device__ __forceinline__ bool next(Seg& sg)
    {
        while (u < uend) {
            const JobInfo& J = ji[j];
            const u64 jend = J.U0 + J.tiles * J.nst;
            if (u >= jend) { ++j; continue; }  // empty or finished job
            const u64 v = u - J.U0;
            sg.job = j;
            sg.tile = v / J.nst;
            sg.kst = v - sg.tile * J.nst;
            const u64 e = umin(umin(uend, J.U0 + (sg.tile + 1) * J.nst), u + max_seg);
            sg.len = e - u;
            u = e;
            return true;
        }
        return false;
    }
};

// Accumulator bookkeeping shared (replayed identically) by the MMA warp and
// the epilogue warps: two TMEM slots tagged with a tile; a segment of a tile
// already in a slot accumulates there, otherwise a free slot or the less
// recently used one is taken (flushing it first).  A slot is also flushed
// before its accumulated stages would pass the exactness cap.
struct Slots {
    u64 tile[2];  // key: job << 40 | tile
    u64 fill[2];
    u32 flushes[2];
    int last;
    u64 max_seg = kMaxSegStages;
    __host__ __device__ __forceinline__ void init()
    {
        tile[0] = tile[1] = ~0ull;
        fill[0] = fill[1] = 0;
        flushes[0] = flushes[1] = 0;
        last = 1;
    }
    __host__ __device__ __forceinline__ int pick(u64 t) const
    {
        if (tile[0] == t) return 0;
        if (tile[1] == t) return 1;
        if (tile[0] == ~0ull) return 0;
        if (tile[1] == ~0ull) return 1;
        return 1 - last;
    }
    // does slot s have to be flushed before a segment of tile t, len stages?
    __host__ __device__ __forceinline__ bool needs_flush(int s, u64 t, u64 len) const
    {
        return tile[s] != ~0ull && (tile[s] != t || fill[s] + len > max_seg);
    }
};

// Row of the packed matrix that unpack thread p (0 .. 128 + kn - 1) reads for
// a tile at (r0, c0): threads 0..127 the A side (rows r0 + p), the others the
// B side (rows c0 + p - 128).
__host__ __device__ __forceinline__ u64 fetch_row(int p, u64 r0, u64 c0)
{
    return p < kM ? r0 + (u64)p : c0 + (u64)(p - kM);
}

// Words q of stage kst that unpack thread p loads: word kst * kStageWords + q
// of its row, for q with that word < W; a 16-byte load takes q and q + 1 when
// both are < W (q even) and vec16 holds.  Rows >= n are not read.
__host__ __device__ __forceinline__ bool fetch_word(u64 kst, int q, u64 W, u64& word, u64 sw = kStageWords)
{
    word = kst * sw + (u64)q;
    return word < W;
}

}  // namespace tcs
}  // namespace jsim
