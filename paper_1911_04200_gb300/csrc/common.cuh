// Shared declarations of the jsim CUDA library (internal; not installed).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "jsim.h"

namespace jsim {

typedef unsigned long long u64;
typedef unsigned int u32;

// Values of one sample per chunk of the ingest kernels (filter, validate, pack).
constexpr u64 kChunk = 4096;
// Bitmap words covered by one directory block of the rank scan.
constexpr u64 kScanBlockWords = 4096;
// Row granularity of the packed matrix; every product tile is a multiple of it.
constexpr u64 kRowPad = 128;
// Devices for which launch-shape caches are kept (higher ordinals recompute).
constexpr int kMaxDevices = 64;
// Word granularity of a packed row (K padding of every product variant).
constexpr u64 kWordPad = 64;

// Row stride of a packed matrix of W words per row: a multiple of kWordPad
// holding W, made an odd number of granules (1024 words for rows of 2^16
// words or more, kWordPad below) so that rows do not all start on the same
// DRAM channel.  Measured on the SM-pair product: rows of 2^19 words (4 MiB
// apart) ran at 935 Tbit-ops/s, 1074 with the stride one 8 KiB granule
// longer; 2^18-word rows 974 -> 1043.
inline u64 row_stride_words(u64 W)
{
    const u64 w = W ? W : 1;
    const u64 g = w > (1ull << 16) - kWordPad ? 1024 : kWordPad;
    u64 k = (w + g - 1) / g;
    if (k % 2 == 0) ++k;
    return k * g;
}

// Error flags raised by device kernels.
constexpr u32 kFlagUnsorted = 1u;
constexpr u32 kFlagIdRange = 2u;

// Per-batch plan of which values of each sample fall in [lo, hi).
struct Plan {
    u64* beg;    // [n]   first position of the sample's batch values
    u64* len;    // [n]   number of them
    u64* cofs;   // [n+1] exclusive prefix of chunk counts
    u64* totals; // [kPlanTotals] total values, total chunks, first value after the batch, whether one
                 // exists; then the chunk tickets of the kernels that walk the plan (filter, pack,
                 // validation) and the windowed ingest's count of class rows, zeroed by the plan
};
constexpr u64 kPlanTotals = 8;
constexpr int kTicketFilter = 4, kTicketPack = 5, kTicketValidate = 6;
constexpr int kPlanRowsTotal = 7;
// u64 words of a plan over n samples: beg, len, cofs (n + 1), totals
__host__ __device__ inline u64 plan_words(u64 n) { return 3 * n + 1 + kPlanTotals; }

// ---- feed.cu ---------------------------------------------------------------
// One piece of page-locked host input (hv: its device-mapped address) copied
// to the same positions of dv: c1[i] = first position in [c0[i], off[i+1])
// with value >= bound (off[i+1] when last), pre = exclusive prefix of the
// slice lengths (n + 1 entries), then `grid` CTAs copy the slices.
cudaError_t launch_feed_piece(const u64* hv, u64* dv, const u64* off, u64 n, const u64* c0, u64* c1, u64 bound,
                              bool last, u64* pre, int grid, cudaStream_t st);

// ---- windows.cu ------------------------------------------------------------
// Windowed ingest of the block-sparse path: the batch [lo, lo + nwin 2^wl)
// of a plan over n samples in tile order (tiles of 128) is cut into nwin
// windows of 2^wl rows, and the windows into G ranges of wpc (the last one
// possibly shorter); both passes run one CTA per (range, tile).
// A range holds at most kWinRangeWords words (of 64 rows) per class: pass 2
// keeps two classes' words of a range in shared memory.
constexpr u64 kMaxWinPerRange = 16;
constexpr u64 kWinRangeWords = 4096;
struct WinGeom {
    u64 n, T, lo;
    u64 nwin, wpc, G;
    u64 nw;     // words per class bitmap: nwin 2^wl / 64
    int wl;     // log2 of the rows of a window, 12..16
    // per tile, the order its samples are handed to warps (tile-local
    // positions, largest sample first: entry 128t + j of the plan's order)
    const u32* lpt;
};
// Pass 1: B (B2 with the two-or-more filter; T x nw words, tile-major) = the
// tiles' filter bitmaps, cls ((T + 1) x nw, class-major) = the class
// bitmaps, pre (likewise) = every class word's rank within its window (the
// class's rows of the window below the word), cnt ((T + 1) x nwin) = every
// window's rows per class, agg
// ((T + 1) x G) = every range's rows per class rounded up to 64, curs
// ((G + 1) x n) = every sample's position at each range start and at the
// batch end; plan.totals[kPlanRowsTotal] += the rows of all classes (zeroed
// by the plan).
size_t win_tiles_smem(const WinGeom& g, bool twice);
cudaError_t launch_win_classes(const u64* ids, Plan plan, const WinGeom& g, bool twice, u64* B, u64* B2, u64* cls,
                               unsigned short* pre, u32* cnt, u64* agg, u64* curs, cudaStream_t st);
// Pass 2: with boff the exclusive prefix of agg (class c's range r at
// boff[c G + r] - boff[c G]), every word of the batch's class-0 part of XM
// (words [kbase[0], kbase[0] + W_0) of rows 0..n-1; null: no class-0 rows)
// and of tile t's part of XS (words [kbase[1 + t], ...) of rows 128t..) is
// stored once, with plain stores.
size_t win_pack_smem(const WinGeom& g);
cudaError_t launch_win_pack(const u64* ids, const WinGeom& g, const u64* cls, const unsigned short* pre,
                            const u32* cnt, const u64* boff, const u64* curs, const u64* kbase, u64* XM, u64 stride_m,
                            u64* XS, u64 stride_s, cudaStream_t st);

// ---- ingest.cu -------------------------------------------------------------
// perm (optional): entry i of the plan describes sample perm[i].  ends
// (optional): sample i's values are searched in [offsets[i], ends[i]) instead
// of [offsets[i], offsets[i + 1]) (a slice of every sample, e.g. the part of
// the input already copied to the device).
cudaError_t launch_plan(const u64* offsets, const u64* ids, u64 n, u64 lo, u64 hi, bool full,
                        Plan plan, cudaStream_t st, const u32* perm = nullptr, const u64* ends = nullptr);
// out[0] = smallest first value, out[1] = largest last value of the
// non-empty samples (the minimum and maximum when they are sorted); out must
// hold {~0, 0} before.
cudaError_t launch_first_last(const u64* offsets, const u64* ids, u64 n, u64* out, cudaStream_t st);
// err_stride 0: one error word for all samples; 1: err[i] per sample
cudaError_t launch_validate(const u64* offsets, const u64* ids, u64 n, Plan plan, u64 max_chunks,
                            int id_bits, u64* sizes, u32* err, u64* maxid, u64* minid, int sms,
                            cudaStream_t st, u64 err_stride = 0);
// Per-tile filter: sample i sets its rows in bitmap tile_of[i] (bitmaps of
// width/32 u32 words each, tile-major); twice likewise (optional).
cudaError_t launch_filter_tiles(const u64* ids, u64 n, Plan plan, u64 max_chunks, u64 lo, u64 width,
                               u32* bitmaps, u32* twice, const u32* tile_of, int sms, cudaStream_t st);
// Single pass into both matrices: class-0 values to XM (null: there are
// none), class cls_of[i] values to XS, atomically OR-ed.
cudaError_t launch_pack_classes(const u64* ids, u64 n, Plan plan, u64 max_chunks, u64 lo, u64 width, const u64* cls,
                                const u32* dir, const u64* boff, u64 nwords, const u64* kbase, const u32* cls_of,
                                const u32* row_of, u64* XM, u64 stride_m, u64* XS, u64 stride_s, int sms,
                                cudaStream_t st);
// twice (optional): also the bitmap of rows held by two or more samples
cudaError_t launch_filter(const u64* ids, u64 n, Plan plan, u64 max_chunks, u64 lo, u64 width,
                          u32* bitmap, int sms, cudaStream_t st, u32* twice = nullptr);
// ktotal/kbase (optional, device): append this batch's words after the
// running word total (kbase = total; total += ceil(R/64)).
cudaError_t launch_scan(const u64* bitmap, u64 nwords, u32* dir, u64* bsum, u64* boff, u64* R,
                        cudaStream_t st, u64* ktotal = nullptr, u64* kbase = nullptr);
// boff = exclusive prefix of the nb counts bsum, *R = their total (one CTA)
cudaError_t launch_scan_top(const u64* bsum, u64 nb, u64* boff, u64* R, cudaStream_t st);
cudaError_t launch_zero_rows(u64* X, u64 rows, u64 stride, u64 words, int sms, cudaStream_t st);
// Packing with plain stores: every nonzero word [kbase, kbase + W_l) of rows
// 0..n-1 (W_l = ceil(*Rdev / 64), device) is written once and complete, into
// a packed matrix the caller has zeroed.  Values whose bit the bitmap lacks
// are not packed (the two-or-more filter).
// Values outside [lo, lo + width) are not packed.
cudaError_t launch_pack_full(const u64* ids, u64 n, Plan plan, u64 max_chunks, u64 lo, u64 width,
                             const u64* bitmap, const u32* dir, const u64* boff, u64* X, u64 stride,
                             const u64* Rdev, int sms, cudaStream_t st, const u64* kbase = nullptr);
// Sample i's word q goes to X[i * stride + (kbase + q) * wstride]: row-major
// packed rows with wstride 1, word-major (one row per word) with stride 1.
cudaError_t launch_pack(const u64* ids, u64 n, Plan plan, u64 max_chunks, u64 lo, u64 width,
                        const u64* bitmap, const u32* dir, const u64* boff, u64* X, u64 stride,
                        u64* batch_sizes, int sms, cudaStream_t st, const u64* kbase = nullptr,
                        u64 wstride = 1);

// ---- product kernels ---------------------------------------------------------
// C (n x n, CT = u32 or u64, row-major with row stride ldc) += X X^T on the
// upper-triangle tiles (both halves of diagonal tiles).  X has rows of
// `stride` words; words at or beyond W, and rows at or beyond n, read as 0.
struct ProductArgs {
    const u64* X;
    u64 stride;
    u64 n;
    u64 W;           // word count, or an upper bound of it when Wdev is set
    const u64* Wdev; // optional: the word count in device memory (read by the kernel)
    void* C;
    u64 ldc;
    int count_bits;
    int word_bits;
    int sms;
    int timeout_ms;  // bound on device-side waits
    u32* err;        // device error word (bit 4: a bounded wait timed out)
    int launches;    // out: kernel launches made
};
cudaError_t product_popc(ProductArgs& a, cudaStream_t st);
cudaError_t product_mma(ProductArgs& a, int variant, cudaStream_t st);
cudaError_t product_tc(ProductArgs& a, cudaStream_t st);
cudaError_t product_tc_single(ProductArgs& a, cudaStream_t st);
// the same product on clusters of two CTAs (tcgen05 cta_group::2)
cudaError_t product_tc_pair(ProductArgs& a, cudaStream_t st);
// Several independent collections in one persistent tcgen05 launch (up to
// 256 per launch; more are launched in groups).  W is read from Wdev on the
// device when Wdev is set (no host synchronisation), else taken from W.
struct TcJobDesc {
    const u64* X;
    const u64* Wdev;
    void* C;
    u64 stride, n, W, ldc;
};
// dev_table: device memory for njobs table entries (sizeof(TcJobDesc) each),
// read by the kernels; with upload it is first written from `jobs`
// (stream-ordered; not allowed while the stream is being captured).
// tile_n: tiles of 128 x 256 (256) or 128 x 128 (128; a diagonal tile then
// unpacks its rows once for both operands).  diag_only (tile_n 128, every job
// of at most 128 samples: one diagonal tile each): stages of the A rows only,
// more of them in flight.
cudaError_t product_tc_jobs(const TcJobDesc* jobs, int njobs, void* dev_table, bool upload, int count_bits, int sms,
                            u32* err, int timeout_ms, cudaStream_t st, int* launches, int tile_n = 256,
                            bool diag_only = false);
bool product_tc_supported(int device);

// ---- query.cu (serving) ---------------------------------------------------------
// A resident reference index: the reference as one batch over [lo, lo+width)
// with filter bitmap, rank directory and the R kept rows of Abar_ref,
// rank-major (row r: ns64 = ceil(n_ref / 64) words, bit j = reference sample
// j holds row r).
struct QueryIndex {
    const u64* index;
    const u64* bm;           // filter words, rank directory and block offsets (build)
    const u32* dir;
    const u64* boff;
    const ulonglong2* fr;    // (filter word, rank of its first bit) per word (queries)
    u64 lo, width, R, n_ref, ns64;
};
// build: Xt (R x ns64, zeroed by the caller) gets bit i of row rank(x) for
// every value x of reference sample i
cudaError_t launch_pack_rows(const u64* ids, u64 n, Plan plan, u64 max_chunks, const QueryIndex& ix, u64* Xt,
                             int sms, cudaStream_t st);
// fr[w] = (bm[w], boff[w / kScanBlockWords] + dir[w]) for the width / 64 words
cudaError_t launch_rank_words(const QueryIndex& ix, ulonglong2* fr, int sms, cudaStream_t st);
// Cacc (S x n_ref u32, zeroed by the caller) += query x reference counts;
// *rows_read += query values found in the filter; ns64 <= 128 (n_ref <= 8192).
// The S samples lie back to back in ids (plan of offsets, full); values =
// their total (host copy).
cudaError_t launch_qrows(const u64* ids, u64 S, Plan plan, u64 values, const QueryIndex& ix, u32* Cacc,
                         u64* rows_read, int sms, cudaStream_t st);
// distance: J holds D = 1.0 - J instead (binary64; 0 for two empty sets)
cudaError_t launch_qepi(const u32* Cacc, u64 S, u64 n_ref, const u64* sq, const u64* sr, int count_bits, void* Cout,
                        double* J, int sms, cudaStream_t st, int distance = 0);

// ---- epilogue.cu ---------------------------------------------------------------
// Cout[i][j] = Cacc[min(i,j)][max(i,j)], J = C / (s_i + s_j - C) (binary64), 1 if 0.
// diag_sizes: C_ii = s_i (the product ran over rows held by two or more
// samples, so its diagonal lacks the rows only sample i holds).
// distance: J holds D = 1.0 - J instead (binary64; 0 for two empty sets).
// *acc (device) += sum over the W word columns of rows 0..n-1 of nnz (nnz + 1) / 2.
cudaError_t launch_useful(const u64* X, u64 n, u64 stride, u64 W, u64* acc, int sms, cudaStream_t st);
// skip_if (optional, device): the kernel writes nothing when *skip_if != 0
cudaError_t launch_epilogue(const void* Cacc, u64 n, int count_bits, const u64* sizes,
                            void* Cout, double* J, cudaStream_t st, int diag_sizes = 0, int distance = 0,
                            const u32* skip_if = nullptr);

}  // namespace jsim
