// Block-sparse all-pairs product (variant JSIM_VARIANT_SPARSE).
//
// The paper stores the bitmask matrix sparsely and notes that the product's
// operation count depends on the sparsity structure, and that rows and
// columns may be permuted freely (Sec. III-B, III-C; C is invariant under a
// relabelling of the rows and permutes with the samples).  On the tensor
// cores a block of 128 samples x 256 rows costs the same whether it holds
// one set bit or all of them, so the work only shrinks when whole blocks are
// empty.  This path arranges that:
//
//  1. Sample order.  A sketch - the product of a small range of the lowest
//     values (about 512 per sample; 2048 to 32768 per sample gave the same
//     order quality on 1024 clade samples) - gives every pair's similarity J; the
//     samples are ordered by a greedy chain (the next sample is the one most
//     similar to any sample already in the current tile of 128), so that
//     samples sharing many values land in the same tile.
//  2. Row classes.  Per row batch, every tile of 128 samples (in that order)
//     gets its own filter bitmap (Eq. 5 restricted to the tile's samples).
//     A row held by two or more tiles is of class 0; a row held by tile t
//     alone is of class 1 + t.  Every class is rank-scanned (Eq. 6), so the
//     packed matrix of the batch splits into a class-0 matrix (all samples)
//     and one matrix per tile holding only that tile's rows.
//  3. Product.  Class-0 words: the dense product over all samples (Eq. 7).
//     Class 1 + t words: a 128 x 128 product of tile t only, added to the
//     diagonal block of tile t - the only block they can change, since no
//     other sample holds those rows.  All tiles' blocks run in one launch of
//     the job-table product.  The words of successive batches are appended
//     (Eq. 4) and multiplied when the matrices fill and at the end.  C
//     accumulates in sample-order positions; the epilogue reads it back
//     through the order.
//  The pack is one pass over the values: a value goes to the class-0 matrix
//  or to its tile's, OR-ed in with atomics (warp lanes holding the same word
//  combine first), since the two classes interleave along a sample.
//
// Every count is the same integer as the dense product's (a sum over the
// same rows, Eq. 4, grouped differently), so C and J are bit-identical.  With
// AUTO the sketch's own rows are classified first, and the call goes on dense
// unless the estimated time of the whole call (product and ingest at rates
// measured on GB300) is at least 5 % below the dense call's.
//
// Internal header of the C-ABI translation unit (included once, after ctx.cuh).
#pragma once
#include <cmath>

namespace {

constexpr u64 kTile = 128;                // samples per tile: the rows of a one-SM tensor-core tile
constexpr u64 kMaxTiles = 16;             // n <= 2048
constexpr u64 kSketchPerSample = 512;     // values per sample in the sketch range, on average
constexpr u64 kMinClassRows = 1ull << 18; // batch width granule: one scan block of every class
constexpr u64 kTileBitmapBytes = 128ull << 20;  // all tiles' filter bitmaps of a batch together
// Rates measured on GB300 (1024 clade samples, 1.3e9 values; both filters)
// that the automatic choice weighs: dense SM-pair product and block-sparse
// products in bit-operations per ms; ingest (validation, filter, scan, pack)
// per value in ms, dense and block-sparse, one filter and two-or-more.
// Batch widths swept at 2^25..2^28 rows (with the samples planned in tile
// order, so only one or two tiles' structures are in use at a time): 62.8 /
// 58.4 / 61.4 ms per call at 2^26 / 2^27 / 2^28 rows with one filter, 69.6 /
// 61.9 / 62.3 ms at 2^25 / 2^26 / 2^27 with the two-or-more filter - the
// widths where all tiles' bitmaps take kTileBitmapBytes.
constexpr double kDenseBitopsPerMs = 1.1e12;
constexpr double kSparseBitopsPerMs = 0.75e12;
constexpr double kIngestDenseMs[2] = {2.8e-8, 2.5e-8};
constexpr double kIngestSparseMs[2] = {2.8e-8, 3.4e-8};
// Windowed ingest (windows.cu): windows of 2^kWinLog rows, used where a
// sample has kWinMinValues values in a window on average (below, most of a
// range's work would go to samples with no value in it).
constexpr int kWinLog = 16;
constexpr double kWinMinValues = 0.5;
constexpr u64 kWinMaxBatch = 1ull << 30;

// Row classes from the tiles' bitmaps: class 0 = rows of two or more tiles,
// class 1 + t = rows of tile t alone (with the two-or-more filter: rows tile
// t holds twice or more and no other tile holds).  One thread per word.
__global__ void k_classify(const u64* __restrict__ B, const u64* __restrict__ B2, u64 T, u64 nwords,
                           u64* __restrict__ cls)
{
    for (u64 w = blockIdx.x * (u64)blockDim.x + threadIdx.x; w < nwords; w += (u64)gridDim.x * blockDim.x) {
        u64 b[kMaxTiles];
        u64 ones = 0, twos = 0;
        #pragma unroll
        for (u64 t = 0; t < kMaxTiles; ++t) {
            b[t] = t < T ? B[t * nwords + w] : 0ull;
            twos |= ones & b[t];
            ones |= b[t];
        }
        cls[w] = twos;
        #pragma unroll
        for (u64 t = 0; t < kMaxTiles; ++t)
            if (t < T) cls[(t + 1) * nwords + w] = (B2 ? B2[t * nwords + w] : b[t]) & ~twos;
    }
}

// Output (i, j) from counts accumulated at positions (pos[i], pos[j]) (upper
// triangle); J as the dense epilogue forms it.  Nothing is written when
// *skip_if is set (a bounded wait of a product ran out).
template <typename CT>
__global__ void k_epilogue_perm(const CT* __restrict__ Cacc, u64 n, const u32* __restrict__ pos,
                                const u64* __restrict__ sizes, CT* __restrict__ Cout, double* __restrict__ J,
                                int diag_sizes, int distance, const u32* skip_if)
{
    if (skip_if && *(volatile const u32*)skip_if) return;
    const u64 total = n * n;
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < total; t += (u64)gridDim.x * blockDim.x) {
        const u64 i = t / n, j = t - i * n;
        const u64 a = pos[i], b = pos[j];
        CT c = a <= b ? Cacc[a * n + b] : Cacc[b * n + a];
        if (diag_sizes && i == j) c = (CT)sizes[i];
        if (Cout) Cout[t] = c;
        if (J) {
            const u64 u = sizes[i] + sizes[j] - (u64)c;
            const double s = u ? __ddiv_rn(__ull2double_rn((u64)c), __ull2double_rn(u)) : 1.0;
            J[t] = distance ? __dsub_rn(1.0, s) : s;
        }
    }
}

// Zero the words [base[c], base[c] + words[c]) of the rows of every tile
// (tile t: rows [kTile t, kTile t + kTile) of X, class c = 1 + t; c = 0:
// all rows, class 0), before a batch packs its words there.
__global__ void k_zero_classes(u64* X, u64 rows, u64 stride, const u64* __restrict__ base,
                               const u64* __restrict__ words, int per_tile)
{
    for (u64 r = blockIdx.y; r < rows; r += gridDim.y) {
        const u64 c = per_tile ? 1 + r / kTile : 0;
        const u64 b = base[c], w = words[c];
        u64* row = X + r * stride + b;
        for (u64 k = blockIdx.x * (u64)blockDim.x + threadIdx.x; k < w; k += (u64)gridDim.x * blockDim.x)
            row[k] = 0ull;
    }
}

unsigned grid_of(u64 items, int sms, unsigned threads)
{
    u64 g = (items + threads - 1) / threads;
    const u64 cap = (u64)sms * 8;
    return (unsigned)std::max<u64>(1, std::min(g, cap));
}

// Single-precision similarities of the sketch, for ordering the samples:
// Jf[i][j] = c / (s_i + s_j - c) from the upper-triangle counts (0 on the
// diagonal and for two empty sketches), and the sketch sizes s_i = C_ii.
// Sketch counts are far below 2^24, so c and u are exact floats and c / u is
// one correctly rounded division.
template <typename CT>
__global__ void k_sketch_j(const CT* __restrict__ Cs, u64 n, float* __restrict__ Jf, u64* __restrict__ sz)
{
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < n * n; t += (u64)gridDim.x * blockDim.x) {
        const u64 i = t / n, j = t - i * n;
        float v = 0.f;
        if (i != j) {
            const u64 a = i < j ? i : j, b = i < j ? j : i;
            const float c = (float)Cs[a * n + b], u = (float)Cs[i * n + i] + (float)Cs[j * n + j] - c;
            v = u > 0.f ? __fdiv_rn(c, u) : 0.f;
        }
        Jf[t] = v;
        if (i == j) sz[i] = (u64)Cs[t];
    }
}

// Sample order from the sketch's similarities Jm (n x n, symmetric) and
// sizes: a greedy chain.  Start at the largest sample; the next sample is
// the unplaced one with the largest J to any sample already in the current
// tile of kTile (a new tile starts from its predecessor's similarities);
// ties go to the smaller index, and a sample sharing nothing with the tile
// is taken largest first.  Each step is one pass: the scores take in the
// last placed sample's similarities and the best unplaced sample is found
// in the same loop.
std::vector<u32> sample_order(const float* Jm, const u64* sz, u64 n)
{
    std::vector<u32> order;
    order.reserve(n);
    std::vector<char> placed(n, 0);
    std::vector<float> score(n, 0.f);
    u64 first = 0;
    for (u64 i = 1; i < n; ++i)
        if (sz[i] > sz[first]) first = i;
    order.push_back((u32)first);
    placed[first] = 1;
    for (u64 step = 1; step < n; ++step) {
        // the scores: J to the current tile's samples (a new tile: to its
        // predecessor only), with the last placed sample taken in now
        const float* r = Jm + (u64)order.back() * n;
        const bool fresh = step == 1 || step % kTile == 0;
        u64 best = n;
        float bs = 0.f;
        for (u64 j = 0; j < n; ++j) {
            const float v = fresh ? r[j] : std::max(score[j], r[j]);
            score[j] = v;
            if (!placed[j] && v > bs) {
                bs = v;
                best = j;
            }
        }
        if (best == n)
            for (u64 j = 0; j < n; ++j)
                if (!placed[j] && (best == n || sz[j] > sz[best])) best = j;
        order.push_back((u32)best);
        placed[best] = 1;
    }
    return order;
}

// Bytes of the class-0 and per-tile matrices the block-sparse path appends
// its batches' words to: a fixed share of the device (12 GiB, or a sixteenth
// of a smaller one).
u64 sparse_matrix_budget(u64 total_bytes) { return std::min<u64>(12ull << 30, total_bytes / 16); }

// Batch width of the block-sparse path for n samples over a value span: a
// power of two and a whole scan block of every class (0: the context's
// batch_rows does not divide into scan blocks).  Per-value ingest: all
// tiles' bitmaps within kTileBitmapBytes (they are updated with L2 atomics).
// Windowed ingest: the span's width up to kWinMaxBatch rows (measured on the
// default workload: 44.0 / 43.3 / 43.1 / 42.8 ms per call at 2^27 / 2^28 /
// 2^29 / 2^30 rows - fewer batches, fewer fixed costs), with both slots'
// batch structures within a sixteenth of the device and a quarter of what is
// free.
u64 sparse_batch_rows(const jsim_ctx* ctx, u64 n, u64 span, bool windowed = false)
{
    const u64 T = (n + kTile - 1) / kTile;
    const u64 f2 = ctx->opt.filter_min == 2 ? 2 : 1;
    u64 mt = ctx->opt.batch_rows;
    if (mt) return mt % kMinClassRows ? 0 : mt;
    if (windowed) {
        mt = kMinClassRows;
        while (mt < kWinMaxBatch && mt - 1 < span) mt <<= 1;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); return kMinClassRows; }
        auto slots_bytes = [&](u64 m) {
            const u64 nwin = m >> kWinLog;
            return 2 * (m / 8 * (T * f2 + T + 1) + m / 64 * 2 * (T + 1) + (nwin + 1) * n * 8 + (T + 1) * nwin * 12);
        };
        while (mt > kMinClassRows && (slots_bytes(mt) > total_b / 16 || slots_bytes(mt) > free_b / 4)) mt >>= 1;
        return mt;
    }
    mt = auto_batch_rows(span + 1 ? span + 1 : ~0ull);
    while (mt > kMinClassRows && T * (mt / 8) * f2 > kTileBitmapBytes) mt >>= 1;
    return std::max(mt, kMinClassRows);
}

// The block-sparse path of jsim_all_pairs: JSIM_ERR_UNSUPPORTED where it does
// not apply (more than kMaxTiles tiles, no tensor cores, a batch width that
// is not a multiple of kMinClassRows); with may_decline, declined = true
// when the sketch shows the product would not be halved (nothing written).
// With a feed, the values arrive piece by piece while the batches run (st
// is validated when the last piece is in); with sv, the values are there and
// their validation runs beside the sketch and the batches.  Either way
// st.minid and st.maxid are every sample's first and last value until the
// verdict is read, before any output is written.
int all_pairs_sparse(jsim_ctx* ctx, Staged& st, void* C, uint64_t* sizes, double* J, int out_mem,
                     bool may_decline, bool& declined, InputFeed* feed = nullptr, SideValidation* sv = nullptr)
{
    declined = false;
    const u64 n = st.n;
    const u64 T = (n + kTile - 1) / kTile;
    if (n == 0 || T > kMaxTiles || !product_tc_supported(ctx->opt.device)) return JSIM_ERR_UNSUPPORTED;
    const size_t cb = ctx->opt.count_bits == 64 ? 8 : 4;
    const bool twice = ctx->opt.filter_min == 2;
    cudaStream_t cs = ctx->stream;
    const u64 n_pad = round_up(n, kRowPad);

    const u64 span = st.N ? st.maxid - st.minid : 0;
    // Windowed ingest where the values are dense enough for windows of
    // 2^wl rows, on device-resident input (the per-value ingest otherwise).
    // Input fed piece by piece keeps the per-value ingest: the windowed
    // kernels hold an SM's registers for tens of microseconds per CTA, which
    // holds back the copy CTAs that feed the link (measured on the default
    // workload from page-locked host memory: 70 to 75 ms per call windowed,
    // 67.5 ms per value).
    const int wl = kWinLog;
    const double per_window =
        st.N ? (double)st.N / (double)n / ((double)span + 1.0) * (double)(1ull << wl) : 0.0;
    const bool windowed = per_window >= kWinMinValues && !feed;
    const u64 mt = feed ? feed->mt : sparse_batch_rows(ctx, n, span, windowed);
    if (!mt) return JSIM_ERR_UNSUPPORTED;
    ctx->stats.batch_rows = mt;
    auto geom = [&](u64 lo, u64 width) {
        WinGeom g{};
        g.n = n;
        g.T = T;
        g.lo = lo;
        g.wl = wl;
        g.nwin = width >> wl;
        g.nw = width / 64;
        g.wpc = std::min<u64>(std::max<u64>(g.nwin, 1), std::min<u64>(kMaxWinPerRange, kWinRangeWords >> (wl - 6)));
        g.G = (g.nwin + g.wpc - 1) / g.wpc;
        return g;
    };

    // search bounds of a batch at lo: with a feed, the slices of lo's piece
    const u64* pb = st.d_off;
    const u64* pe = nullptr;
    auto bounds_for = [&](u64 lo) -> int {
        if (!feed) return JSIM_OK;
        const int g = feed->piece_of(lo);
        int r = feed->wait(g);
        if (r) return r;
        pb = feed->beg(g);
        pe = feed->end(g);
        return JSIM_OK;
    };

    // ---- sketch: the dense product of the lowest values, about
    // kSketchPerSample per sample ----
    std::vector<u32> order(n), pos(n);
    for (u64 i = 0; i < n; ++i) order[i] = (u32)i;
    DevBuf d_pos, d_order, d_tile, d_cls_of, d_rowk, d_lpt, jobtab, Wc, kbase;
    const u64 nw_max = mt / 64;
    const u64 nb_max = (T + 1) * nw_max / kScanBlockWords;
    // Two slots of batch structures: the next batch is classified while this
    // one's class totals travel to the host and its pack is enqueued, so the
    // device does not wait for the host between batches.  Slot s reads its
    // totals back into pinned scalars [64 + 32 s, +22) and uploads its class
    // bases from [128 + 64 s, +2(T + 1)).  Windowed: bsum holds the ranges'
    // rows per class, cnt the windows', curs the window-start cursors.
    struct Slot {
        DevBuf B, B2, cls, dir, bsum, boff, Rd, plan_buf, cnt, curs, pre;
        Plan plan{};
        WinGeom g{};
        cudaEvent_t done = nullptr;    // totals on the host
        cudaEvent_t packed = nullptr;  // the last pack that read the slot's structures
        bool pack_pending = false;
        ~Slot()
        {
            if (done) cudaEventDestroy(done);
            if (packed) cudaEventDestroy(packed);
        }
    } slot[2];
    const u64 nwin_max = mt >> wl;
    const u64 ranges_max = nwin_max;  // a range holds one window or more
    for (Slot& x : slot) {
        ALLOC(x.cls, (T + 1) * nw_max * sizeof(u64));
        if (windowed) {
            ALLOC(x.B, T * nw_max * sizeof(u64));
            if (twice) ALLOC(x.B2, T * nw_max * sizeof(u64));
            ALLOC(x.cnt, (T + 1) * nwin_max * sizeof(u32));
            ALLOC(x.pre, (T + 1) * nw_max * sizeof(unsigned short));
            ALLOC(x.bsum, (T + 1) * ranges_max * sizeof(u64));
            ALLOC(x.boff, ((T + 1) * ranges_max + 1) * sizeof(u64));
            ALLOC(x.curs, (nwin_max + 1) * n * sizeof(u64));
        } else {
            ALLOC(x.B, T * nw_max * sizeof(u64));
            if (twice) ALLOC(x.B2, T * nw_max * sizeof(u64));
            ALLOC(x.dir, (T + 1) * nw_max * sizeof(u32));
            ALLOC(x.bsum, nb_max * sizeof(u64));
            ALLOC(x.boff, (nb_max + 1) * sizeof(u64));
        }
        ALLOC(x.Rd, sizeof(u64));
        ALLOC(x.plan_buf, plan_words(n) * sizeof(u64));
        x.plan = carve_plan(x.plan_buf, n);
        CK(cudaEventCreateWithFlags(&x.done, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&x.packed, cudaEventDisableTiming));
    }
    // Windowed: the batches are classified on a side stream, so the next
    // batch's classification runs beside this batch's pack (both are bound
    // by latency and instruction issue, at about half the SMs' issue rate
    // each); slot s's classification waits for the pack that last read slot
    // s, and a pack for its slot's classification.  The side stream has the
    // device's highest priority: the pack of a batch waits for the next
    // classification, so the classification's CTAs go first and the pack
    // takes the SMs' remaining room.  Whatever way the call returns, the
    // context's stream then waits for the side stream (before the slots'
    // memory is released on it).
    cudaStream_t ccs = cs;
    if (windowed) {
        if (!ctx->class_stream) {
            int lo_p = 0, hi_p = 0;
            CK(cudaDeviceGetStreamPriorityRange(&lo_p, &hi_p));
            CK(cudaStreamCreateWithPriority(&ctx->class_stream, cudaStreamNonBlocking, hi_p));
        }
        ccs = ctx->class_stream;
    }
    struct Join {
        cudaStream_t a, b;
        cudaEvent_t e = nullptr;
        ~Join()
        {
            if (a == b) return;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(e, b);
                cudaStreamWaitEvent(a, e, 0);
                cudaEventDestroy(e);
            } else {
                cudaStreamSynchronize(b);
            }
            cudaGetLastError();
        }
    } join{cs, ccs};
    ALLOC(Wc, (T + 1) * sizeof(u64));
    ALLOC(kbase, (T + 1) * sizeof(u64));
    ALLOC(d_pos, n * sizeof(u32));
    ALLOC(d_order, n * sizeof(u32));
    ALLOC(d_rowk, n * sizeof(u32));
    ALLOC(d_lpt, n * sizeof(u32));
    ALLOC(d_tile, n * sizeof(u32));
    ALLOC(d_cls_of, n * sizeof(u32));
    ALLOC(jobtab, kMaxTiles * sizeof(TcJobDesc));
    CK(cudaMemsetAsync(kbase.p, 0, (T + 1) * sizeof(u64), cs));

    // classify the rows of [lo, lo + width) into slot s and scan them; the
    // totals go to the host behind the slot's event
    auto enqueue_classify = [&](int si, u64 lo, u64 width) -> int {
        Slot& x = slot[si];
        const u64 nw = width / 64;
        const u64 hi = lo + width;  // 0 on wrap-around: unbounded
        u64* hs = ctx->h_scalars + 64 + 32 * si;
        if (windowed) {
            x.g = geom(lo, width);
            x.g.lpt = d_lpt.as<u32>();
            if (x.g.nwin > nwin_max || x.g.G > ranges_max || x.g.nwin * (1ull << wl) != width)
                return JSIM_ERR_UNSUPPORTED;  // the slot's buffers are sized for nwin_max windows
            if (x.pack_pending) CK(cudaStreamWaitEvent(ccs, x.packed, 0));
            {
                StageTimer t(ctx, &ctx->stats.ms_filter, ccs);
                CK(launch_plan(pb, st.d_ids, n, lo, hi, false, x.plan, ccs, d_order.as<u32>(), pe));
                CK(launch_win_classes(st.d_ids, x.plan, x.g, twice, x.B.as<u64>(), twice ? x.B2.as<u64>() : nullptr,
                                      x.cls.as<u64>(), x.pre.as<unsigned short>(), x.cnt.as<u32>(),
                                      x.bsum.as<u64>(), x.curs.as<u64>(), ccs));
                ctx->stats.launches += 4;
                ctx->stats.windows += x.g.nwin;
            }
            {
                StageTimer t(ctx, &ctx->stats.ms_scan, ccs);
                CK(launch_scan_top(x.bsum.as<u64>(), (T + 1) * x.g.G, x.boff.as<u64>(), x.Rd.as<u64>(), ccs));
                ctx->stats.launches += 1;
            }
            CK(cudaMemcpy2DAsync(hs, sizeof(u64), x.boff.as<u64>(), x.g.G * sizeof(u64), sizeof(u64), T + 1,
                                 cudaMemcpyDeviceToHost, ccs));
            CK(cudaMemcpyAsync(hs + 17, x.Rd.p, sizeof(u64), cudaMemcpyDeviceToHost, ccs));
            CK(cudaMemcpyAsync(hs + 18, x.plan.totals + 2, 2 * sizeof(u64), cudaMemcpyDeviceToHost, ccs));
            CK(cudaMemcpyAsync(hs + 20, x.plan.totals, sizeof(u64), cudaMemcpyDeviceToHost, ccs));
            CK(cudaMemcpyAsync(hs + 21, x.plan.totals + kPlanRowsTotal, sizeof(u64), cudaMemcpyDeviceToHost, ccs));
            CK(cudaEventRecord(x.done, ccs));
            return JSIM_OK;
        }
        {
            StageTimer t(ctx, &ctx->stats.ms_filter);
            // the plan lists the samples in their order (entry k: the sample
            // at position k), so the chunks in flight belong to one or two
            // tiles and their bitmaps and directories stay in L2
            CK(launch_plan(pb, st.d_ids, n, lo, hi, false, x.plan, cs, d_order.as<u32>(), pe));
            CK(cudaMemsetAsync(x.B.p, 0, T * nw * sizeof(u64), cs));
            if (twice) CK(cudaMemsetAsync(x.B2.p, 0, T * nw * sizeof(u64), cs));
            CK(launch_filter_tiles(st.d_ids, n, x.plan, st.max_chunks, lo, width, x.B.as<u32>(),
                                   twice ? x.B2.as<u32>() : nullptr, d_tile.as<u32>(), ctx->sms, cs));
            // one word per thread: short CTAs that any free slot can take
            k_classify<<<(unsigned)std::max<u64>(1, (nw + 255) / 256), 256, 0, cs>>>(
                x.B.as<u64>(), twice ? x.B2.as<u64>() : nullptr, T, nw, x.cls.as<u64>());
            CK(cudaGetLastError());
            ctx->stats.launches += 3;
        }
        {
            StageTimer t(ctx, &ctx->stats.ms_scan);
            CK(launch_scan(x.cls.as<u64>(), (T + 1) * nw, x.dir.as<u32>(), x.bsum.as<u64>(), x.boff.as<u64>(),
                           x.Rd.as<u64>(), cs));
            ctx->stats.launches += 2;
        }
        // every class's first block offset, the total and the plan's next value
        const u64 nb = nw / kScanBlockWords;
        CK(cudaMemcpy2DAsync(hs, sizeof(u64), x.boff.as<u64>(), nb * sizeof(u64), sizeof(u64), T + 1,
                             cudaMemcpyDeviceToHost, cs));
        CK(cudaMemcpyAsync(hs + 17, x.Rd.p, sizeof(u64), cudaMemcpyDeviceToHost, cs));
        CK(cudaMemcpyAsync(hs + 18, x.plan.totals + 2, 2 * sizeof(u64), cudaMemcpyDeviceToHost, cs));
        CK(cudaMemcpyAsync(hs + 20, x.plan.totals, sizeof(u64), cudaMemcpyDeviceToHost, cs));
        CK(cudaEventRecord(x.done, cs));
        return JSIM_OK;
    };
    // R_c of the batch in slot s, its plan's next value and its value count
    // (windowed: rounded up per range) and its rows without the rounding
    std::vector<u64> Rc(T + 1, 0);
    u64 range_values = 0, range_rows = 0;
    auto read_classify = [&](int si, bool& has_next, u64& next) -> int {
        CK(cudaEventSynchronize(slot[si].done));
        const u64* hs = ctx->h_scalars + 64 + 32 * si;
        range_rows = 0;
        for (u64 c = 0; c <= T; ++c) {
            Rc[c] = (c < T ? hs[c + 1] : hs[17]) - hs[c];
            range_rows += Rc[c];
        }
        if (windowed) range_rows = hs[21];
        next = hs[18];
        has_next = hs[19] != 0;
        range_values = hs[20];
        return JSIM_OK;
    };

    std::vector<u64> ssz(n, 0);  // the samples' sketch sizes (by sample)
    if (st.N) {
        u64 ws = 1ull << 16;
        const double want = (double)kSketchPerSample * (double)n;
        while (ws < mt && (double)st.N * (double)ws / ((double)span + 1.0) < want) ws <<= 1;
        const u64 lo_s = st.minid / ws * ws;
        BatchBufs sb;
        u64 R_s = 0, stride_s = 0;
        int rc = bounds_for(lo_s);
        if (rc) return rc;
        rc = build_batch(ctx, st, sb, lo_s, ws, R_s, stride_s, nullptr, nullptr, nullptr, pb, pe);
        if (rc) return rc;
        if (R_s) {
            DevBuf Cs;
            ALLOC(Cs, n * n * cb);
            CK(cudaMemsetAsync(Cs.p, 0, n * n * cb, cs));
            const u64 W_s = (R_s + 63) / 64;
            rc = run_product(ctx, choose_variant(ctx, n, W_s), sb.X.as<u64>(), stride_s, n, W_s, Cs.p);
            if (rc) return rc;
            // the input's validation runs while the host orders the samples
            if (sv && !sv->started) {
                rc = sv->start(ctx, st);
                if (rc) return rc;
            }
            // the sizes (n u64) and then the similarities (n x n floats) into
            // page-locked memory kept by the context: the host only runs the
            // greedy chain
            const size_t hb = n * sizeof(u64) + n * n * sizeof(float);
            if (ctx->h_sketch_bytes < hb) {
                if (ctx->h_sketch) cudaFreeHost(ctx->h_sketch);
                ctx->h_sketch = nullptr;
                ctx->h_sketch_bytes = 0;
                CK(cudaMallocHost(&ctx->h_sketch, hb));
                ctx->h_sketch_bytes = hb;
            }
            DevBuf Jf;
            ALLOC(Jf, hb);
            const unsigned g = grid_of(n * n, ctx->sms, 256);
            u64* d_sz = Jf.as<u64>();
            float* d_jf = (float*)(d_sz + n);
            if (cb == 8)
                k_sketch_j<u64><<<g, 256, 0, cs>>>(Cs.as<u64>(), n, d_jf, d_sz);
            else
                k_sketch_j<u32><<<g, 256, 0, cs>>>(Cs.as<u32>(), n, d_jf, d_sz);
            CK(cudaGetLastError());
            ctx->stats.launches += 1;
            CK(cudaMemcpyAsync(ctx->h_sketch, Jf.p, hb, cudaMemcpyDeviceToHost, cs));
            CK(cudaStreamSynchronize(cs));
            const u64* h_sz = (const u64*)ctx->h_sketch;
            order = sample_order((const float*)(h_sz + n), h_sz, n);
            ssz.assign(h_sz, h_sz + n);
        }
        for (u64 k = 0; k < n; ++k) pos[order[k]] = (u32)k;
        // per plan entry k (the sample at position k): its tile, class and
        // row; and per tile the order its samples go to the windowed kernels'
        // warps: largest sketch first (sizes vary by two decades, and a large
        // sample taken last would hold its CTA up)
        std::vector<u32> tile(n), cls_of(n), rowk(n), lpt(n);
        for (u64 k = 0; k < n; ++k) {
            tile[k] = (u32)(k / kTile);
            cls_of[k] = 1 + tile[k];
            rowk[k] = (u32)k;
            lpt[k] = (u32)(k % kTile);
        }
        for (u64 k0 = 0; k0 < n; k0 += kTile) {
            u32* l = lpt.data() + k0;
            const u64 m = std::min<u64>(kTile, n - k0);
            std::stable_sort(l, l + m, [&](u32 a, u32 b) { return ssz[order[k0 + a]] > ssz[order[k0 + b]]; });
        }
        CK(cudaMemcpyAsync(d_lpt.p, lpt.data(), n * sizeof(u32), cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(d_pos.p, pos.data(), n * sizeof(u32), cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(d_order.p, order.data(), n * sizeof(u32), cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(d_tile.p, tile.data(), n * sizeof(u32), cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(d_cls_of.p, cls_of.data(), n * sizeof(u32), cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(d_rowk.p, rowk.data(), n * sizeof(u32), cudaMemcpyHostToDevice, cs));
        CK(cudaStreamSynchronize(cs));  // the host vectors are released at return

        if (may_decline && R_s) {
            // the sketch range's rows by class: is the product at least halved?
            bool hn;
            u64 nx;
            rc = enqueue_classify(0, lo_s, std::max(ws, kMinClassRows));  // inside the first batch: same piece
            if (rc) return rc;
            rc = read_classify(0, hn, nx);
            if (rc) return rc;
            // the call's product work, dense and block-sparse, scaled from the
            // sketch range's rows by values; with the ingest, the call's time
            // either way at the measured rates
            double rows = 0, sparse = 0;
            for (u64 c = 0; c <= T; ++c) {
                const double r = (double)Rc[c];
                rows += r;
                if (c == 0) {
                    sparse += r * (double)n * (double)(n + 1) / 2.0;
                } else {
                    const double m = (double)std::min<u64>(kTile, n - (c - 1) * kTile);
                    sparse += r * m * (m + 1) / 2.0;
                }
            }
            const double scale = range_values ? (double)st.N / (double)range_values : 1.0;
            const double dense_bitops = rows * scale * (double)n * (double)(n + 1) / 2.0;
            const double sparse_bitops = sparse * scale;
            const double t_dense = dense_bitops / kDenseBitopsPerMs + (double)st.N * kIngestDenseMs[twice];
            const double t_sparse = sparse_bitops / kSparseBitopsPerMs + (double)st.N * kIngestSparseMs[twice];
            if (t_sparse > 0.95 * t_dense) {
                declined = true;
                ctx->stats.windows = 0;
                return JSIM_OK;
            }
        }
    } else {
        for (u64 k = 0; k < n; ++k) pos[k] = (u32)k;
        CK(cudaMemcpyAsync(d_pos.p, pos.data(), n * sizeof(u32), cudaMemcpyHostToDevice, cs));
        CK(cudaStreamSynchronize(cs));
    }
    ctx->stats.variant = JSIM_VARIANT_SPARSE;

    // ---- the batch loop ----
    // The class-0 words of all samples (XM) and every tile's own words (XS,
    // tile t in rows [kTile t, kTile t + kTile)) are appended batch after
    // batch (C is a sum over batches, Eq. 4) and multiplied when a matrix is
    // full and at the end: few, deep products instead of two per batch.
    DevBuf Cacc, XM, XS;
    ALLOC(Cacc, n * n * cb);
    CK(cudaMemsetAsync(Cacc.p, 0, n * n * cb, cs));
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(u32), cs));
    // a fixed share of the device (not of what is free now, which moves with
    // other allocators' caches: sizes that change from call to call made
    // every fourth call reallocate and take twice as long)
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); total_b = 64ull << 30; }
    const u64 budget = sparse_matrix_budget(total_b);  // XM a third, XS two thirds
    u64 capM = std::max<u64>(1ull << 12, budget / 3 / (n_pad * 8) / 64 * 64);
    u64 capS = std::max<u64>(1ull << 12, budget * 2 / 3 / (n_pad * 8) / 64 * 64);
    u64 stride_m = 0, stride_s = 0;
    u64 totM = 0;
    std::vector<u64> totS(T, 0);
    auto flush = [&]() -> int {
        StageTimer t(ctx, &ctx->stats.ms_product);
        double done = 0;
        if (totM) {
            int r = run_product(ctx, choose_variant(ctx, n, totM), XM.as<u64>(), stride_m, n, totM, Cacc.p);
            if (r) return r;
            done += (double)totM * (double)n * (double)(n + 1) / 2.0;
        }
        std::vector<TcJobDesc> jobs;
        for (u64 t2 = 0; t2 < T; ++t2) {
            if (!totS[t2]) continue;
            const u64 m = std::min<u64>(kTile, n - t2 * kTile);
            jobs.push_back(TcJobDesc{XS.as<u64>() + t2 * kTile * stride_s, nullptr,
                                     (char*)Cacc.p + (t2 * kTile * n + t2 * kTile) * cb, stride_s, m, totS[t2], n});
            done += (double)totS[t2] * (double)m * (double)(m + 1) / 2.0;
        }
        if (!jobs.empty()) {
            int launches = 0;
            // every job is one diagonal 128 x 128 tile: its rows are unpacked
            // once for both operands
            CK(product_tc_jobs(jobs.data(), (int)jobs.size(), jobtab.p, true, ctx->opt.count_bits, ctx->sms,
                               ctx->d_err, ctx->opt.timeout_ms > 0 ? ctx->opt.timeout_ms : 2000, cs, &launches, 128,
                               true));
            ctx->stats.product_launches += launches;
            ctx->stats.launches += launches;
        }
        ctx->stats.bitops_done += 64.0 * done;
        totM = 0;
        std::fill(totS.begin(), totS.end(), 0ull);
        return JSIM_OK;
    };
    auto any_packed = [&]() { return totM || std::any_of(totS.begin(), totS.end(), [](u64 w) { return w; }); };
    if (st.N) {
        u64 lo = st.minid / mt * mt;
        int si = 0;
        int rc = bounds_for(lo);
        if (rc) return rc;
        rc = enqueue_classify(si, lo, mt);
        if (rc) return rc;
        bool dense_run = true;  // the last batch's values continued in the batch right after it
        for (;;) {
            // While the values run on from batch to batch, the next row batch
            // is taken to follow this one and classified before this one's
            // totals are read (were it empty after all, that costs one
            // classification); not when it lies in a piece of the input still
            // in flight, where the wait is better spent multiplying.
            const u64 lo_sp = lo + mt;
            bool queued = false;
            if (dense_run && lo_sp > lo && lo_sp <= st.maxid &&
                (!feed || feed->piece_of(lo_sp) == feed->piece_of(lo) || feed->arrived(feed->piece_of(lo_sp)))) {
                rc = bounds_for(lo_sp);
                if (rc) return rc;
                rc = enqueue_classify(1 - si, lo_sp, mt);
                if (rc) return rc;
                queued = true;
            }
            bool has_next = false;
            u64 next = 0;
            rc = read_classify(si, has_next, next);
            if (rc) return rc;
            dense_run = has_next && next / mt * mt == lo_sp;
            const Slot& x = slot[si];
            const u64 nw = mt / 64;
            std::vector<u64> W(T + 1);
            u64 R = 0, Wmax_s = 0;
            bool full = false;
            for (u64 c = 0; c <= T; ++c) {
                W[c] = (Rc[c] + 63) / 64;
                R += Rc[c];
                if (c) {
                    Wmax_s = std::max(Wmax_s, W[c]);
                    full = full || totS[c - 1] + W[c] > capS;
                }
            }
            full = full || totM + W[0] > capM;
            if (R) {
                if (full) {
                    rc = flush();
                    if (rc) return rc;
                }
                // a batch alone above the capacity widens the matrix (it is empty now)
                if (W[0] > capM) { capM = round_up(W[0], 64); stride_m = 0; }
                if (Wmax_s > capS) { capS = round_up(Wmax_s, 64); stride_s = 0; }
                if (!stride_m && W[0]) {
                    stride_m = row_stride_words(capM);
                    XM.release();
                    ALLOC(XM, n_pad * stride_m * sizeof(u64));
                }
                if (!stride_s && Wmax_s) {
                    stride_s = row_stride_words(capS);
                    XS.release();
                    ALLOC(XS, n_pad * stride_s * sizeof(u64));
                }
                // the class bases and widths of the batch, from page-locked
                // scratch of the slot (the upload that last read it precedes
                // this batch's classification on the stream)
                u64* hk = ctx->h_scalars + 128 + 64 * si;
                hk[0] = totM;
                hk[T + 1] = W[0];
                for (u64 t2 = 0; t2 < T; ++t2) {
                    hk[1 + t2] = totS[t2];
                    hk[T + 2 + t2] = W[1 + t2];
                }
                CK(cudaMemcpyAsync(kbase.p, hk, (T + 1) * sizeof(u64), cudaMemcpyHostToDevice, cs));
                CK(cudaMemcpyAsync(Wc.p, hk + T + 1, (T + 1) * sizeof(u64), cudaMemcpyHostToDevice, cs));
                if (windowed) {
                    StageTimer t(ctx, &ctx->stats.ms_pack);
                    CK(cudaStreamWaitEvent(cs, x.done, 0));
                    CK(launch_win_pack(st.d_ids, x.g, x.cls.as<u64>(), x.pre.as<unsigned short>(), x.cnt.as<u32>(),
                                       x.boff.as<u64>(), x.curs.as<u64>(), kbase.as<u64>(),
                                       W[0] ? XM.as<u64>() : nullptr, stride_m, Wmax_s ? XS.as<u64>() : nullptr,
                                       stride_s, cs));
                    CK(cudaEventRecord(slot[si].packed, cs));
                    slot[si].pack_pending = true;
                    ctx->stats.launches += 1;
                } else {
                    StageTimer t(ctx, &ctx->stats.ms_pack);
                    if (W[0]) {
                        dim3 g(std::max<unsigned>(1, (unsigned)std::min<u64>((W[0] + 255) / 256, 64)),
                               (unsigned)std::min<u64>(n_pad, 1024));
                        k_zero_classes<<<g, 256, 0, cs>>>(XM.as<u64>(), n_pad, stride_m, kbase.as<u64>(), Wc.as<u64>(), 0);
                        CK(cudaGetLastError());
                    }
                    if (Wmax_s) {
                        dim3 g(std::max<unsigned>(1, (unsigned)std::min<u64>((Wmax_s + 255) / 256, 64)),
                               (unsigned)std::min<u64>(T * kTile, 1024));
                        k_zero_classes<<<g, 256, 0, cs>>>(XS.as<u64>(), T * kTile, stride_s, kbase.as<u64>(),
                                                          Wc.as<u64>(), 1);
                        CK(cudaGetLastError());
                    }
                    CK(launch_pack_classes(st.d_ids, n, x.plan, st.max_chunks, lo, mt, x.cls.as<u64>(),
                                           x.dir.as<u32>(), x.boff.as<u64>(), nw, kbase.as<u64>(),
                                           d_cls_of.as<u32>(), d_rowk.as<u32>(), W[0] ? XM.as<u64>() : nullptr,
                                           stride_m, Wmax_s ? XS.as<u64>() : nullptr, stride_s, ctx->sms, cs));
                    ctx->stats.launches += 3;
                }
                totM += W[0];
                for (u64 t2 = 0; t2 < T; ++t2) totS[t2] += W[1 + t2];
                u64 ws_sum = 0;
                for (u64 t2 = 0; t2 < T; ++t2)
                    ws_sum += (windowed ? std::min<u64>(kTile, n - t2 * kTile) : kTile) * W[1 + t2];
                ctx->stats.pack_bytes += 8 * range_values + 8 * ((windowed ? n : n_pad) * W[0] + ws_sum);
                const u64 Wd = (range_rows + 63) / 64;  // the words of the dense packing of the batch
                ctx->stats.batches += 1;
                ctx->stats.rows_nonzero += range_rows;
                ctx->stats.words += Wd;
                ctx->stats.bitops_dense += 64.0 * (double)Wd * (double)n * (double)(n + 1) / 2.0;
            }
            if (queued) {
                // the batch after this one is classified already: it is next
                // (every value of this batch's successor lies at or above it)
                si = 1 - si;
                lo = lo_sp;
                continue;
            }
            // The next batch from this one's plan: its first value above the
            // batch; with a feed the plan saw only lo's piece, and past its
            // last value the next piece begins.  The cursor moves forward by
            // at least a batch and stops after the last value (what the input
            // holds is only checked when the whole of it is in).
            u64 nl = 0;
            if (!feed) {
                nl = has_next ? next / mt * mt : 0;
            } else {
                const int g = feed->piece_of(lo);
                nl = has_next ? std::max(next / mt * mt, lo + mt) : g + 1 < feed->K ? feed->P[g + 1] : 0;
            }
            if (nl <= lo || nl > st.maxid) break;
            // waiting for a piece still in flight: multiply what is packed
            // so far in the meantime
            if (feed && feed->piece_of(nl) != feed->piece_of(lo) && !feed->arrived(feed->piece_of(nl)) &&
                any_packed()) {
                rc = flush();
                if (rc) return rc;
            }
            rc = bounds_for(nl);
            if (rc) return rc;
            si = 1 - si;
            lo = nl;
            rc = enqueue_classify(si, lo, mt);
            if (rc) return rc;
        }
        rc = flush();
        if (rc) return rc;
    }
    if (feed || sv) {
        // the validation's verdict (and the sizes the epilogue reads)
        int rc = feed ? feed->finish(st) : sv->finish(ctx, st);
        if (rc) return rc;
    }
    ctx->stats.variant = JSIM_VARIANT_SPARSE;

    // ---- outputs, read back through the sample order ----
    int rc = check_device_waits(ctx, ctx->d_err);
    if (rc) return rc;
    DevBuf Cst, Jst;
    void* Cdst = C;
    double* Jdst = J;
    if (out_mem == JSIM_MEM_HOST) {
        if (C) { ALLOC(Cst, n * n * cb); Cdst = Cst.p; }
        if (J) { ALLOC(Jst, n * n * sizeof(double)); Jdst = Jst.as<double>(); }
    }
    {
        StageTimer t(ctx, &ctx->stats.ms_epilogue);
        if (Cdst || Jdst) {
            const unsigned g = grid_of(n * n, ctx->sms, 256);
            if (cb == 8)
                k_epilogue_perm<u64><<<g, 256, 0, cs>>>(Cacc.as<u64>(), n, d_pos.as<u32>(), st.sizes.as<u64>(),
                                                        (u64*)Cdst, Jdst, twice, ctx->opt.distance, ctx->d_err);
            else
                k_epilogue_perm<u32><<<g, 256, 0, cs>>>(Cacc.as<u32>(), n, d_pos.as<u32>(), st.sizes.as<u64>(),
                                                        (u32*)Cdst, Jdst, twice, ctx->opt.distance, ctx->d_err);
            CK(cudaGetLastError());
            ctx->stats.launches += 1;
        }
    }
    {
        StageTimer t(ctx, &ctx->stats.ms_d2h);
        const cudaMemcpyKind k = out_mem == JSIM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        if (out_mem == JSIM_MEM_HOST) {
            if (C) CK(cudaMemcpyAsync(C, Cst.p, n * n * cb, k, cs));
            if (J) CK(cudaMemcpyAsync(J, Jst.p, n * n * sizeof(double), k, cs));
        }
        if (sizes) CK(cudaMemcpyAsync(sizes, st.sizes.p, n * sizeof(u64), k, cs));
    }
    CK(cudaStreamSynchronize(cs));
    return JSIM_OK;
}

}  // namespace
