// Host input brought to the device in value-range pieces while the
// block-sparse batch loop works on the pieces already there.
//
// The batch loop (Sec. III-B; Eq. 3) reads, for row batch [lo, lo + m~), only
// the values of every sample that fall in it.  So the copy of page-locked
// host input need not finish before the first batch: the values keep their
// sample-major places (device offsets = host offsets), and piece g - every
// sample's values in [P_g, P_{g+1}), one contiguous slice per sample, with
// the P_g multiples of the batch width - is brought over by the GPU itself
// (feed.cu: a binary search per sample in host memory, then a copy grid of
// kFeedCtas CTAs reading the host's values through their device-mapped
// address).  Every piece is enqueued at the start on a copy stream of its
// own, each followed by an event; the batch loop makes the context's stream
// wait for a piece's event before it plans a batch of the piece, and plans
// it inside the piece's slices only (the cut rows the copy stream wrote), so
// nothing reads values that are not there yet.  The pieces grow from one
// batch to an eighth of the range and shrink back to one batch at the end, so
// little of the copy is exposed at the start and little of the batch loop is
// left when it ends.  The ingest kernels take their chunks by ticket, so the
// CTA slots the copy grid holds delay none of them.
//
// The input is validated piece by piece as the pieces arrive (on a side
// stream, while the batch loop goes on; the pieces' slices tile every
// sample, so every value is checked once), and the verdict is read before
// any output is written.  Until then the loop relies only on what holds for
// any input: plans stay inside their slices, the ingest kernels drop values
// outside the batch, and the batch cursor only moves forward.
//
// Internal header of the C-ABI translation unit (included once, after ctx.cuh).
#pragma once

namespace {

constexpr int kFeedCtas = 64;  // copy grid: 64 x 256 threads keep the host link busy
// input below this many bytes is copied whole (the pieces' fixed costs
// would not pay)
constexpr u64 kFeedMinBytes = 512ull << 20;

struct InputFeed {
    jsim_ctx* ctx = nullptr;
    u64 n = 0, mt = 0;
    std::vector<u64> P;         // P[g]: first value of piece g; piece K-1 is open above
    int K = 0;
    const u64* d_off = nullptr; // cut row 0: the offsets
    DevBuf d_cuts;              // cut rows 1..K (row g: first position of piece g; row K: the ends)
    DevBuf d_pre;               // per piece: exclusive prefix of its slice lengths (n + 1)
    cudaStream_t xs = nullptr;  // the copy stream
    cudaEvent_t ready = nullptr, t0 = nullptr;
    std::vector<cudaEvent_t> ev;  // piece g on the device
    SideValidation val;           // of every piece as it arrives

    InputFeed() = default;
    InputFeed(const InputFeed&) = delete;
    InputFeed& operator=(const InputFeed&) = delete;
    ~InputFeed() { shutdown(); }

    // waits for the copy and validation streams (before the device buffers
    // they write are released) and frees what the feed holds
    void shutdown()
    {
        if (xs) cudaStreamSynchronize(xs);
        if (val.vs) cudaStreamSynchronize(val.vs);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        ev.clear();
        for (cudaEvent_t* e : {&ready, &t0})
            if (*e) { cudaEventDestroy(*e); *e = nullptr; }
        if (xs) { cudaStreamDestroy(xs); xs = nullptr; }
        cudaGetLastError();
    }

    // piece holding value v (the last piece holds everything above)
    int piece_of(u64 v) const
    {
        int g = (int)(std::upper_bound(P.begin(), P.end(), v) - P.begin()) - 1;
        return g < 0 ? 0 : g;
    }
    const u64* row(int g) const { return g == 0 ? d_off : d_cuts.as<u64>() + (u64)(g - 1) * n; }
    const u64* beg(int g) const { return row(g); }
    const u64* end(int g) const { return row(g + 1); }

    // The pieces of the batches between minid and maxid, all enqueued on the
    // copy stream, and the validation behind the last one.  hv: the host
    // values' device-mapped address; st: the staged collection (offsets on
    // the device, values allocated, not yet copied).
    int start(jsim_ctx* c, Staged& st, const u64* hv, u64 mt_, u64 minid, u64 maxid)
    {
        ctx = c; n = st.n; mt = mt_; d_off = st.d_off;
        const u64 b_first = minid / mt, nb = maxid / mt - b_first + 1;
        const u64 cap = std::max<u64>(1, (nb + 7) / 8);
        // pieces of 1, 1, 2, 4, ... batches up to an eighth of the range, and
        // the last ones halved down to one batch, so that little of the copy
        // is exposed before the first batch and little of the batch loop is
        // left when the copy ends
        std::vector<u64> len;
        for (u64 b = 0, l = 1; b < nb; b += l, l = std::min(cap, l * (b >= 2 ? 2 : 1))) len.push_back(std::min(l, nb - b));
        while (len.back() > 1 && len.size() < 32) {
            const u64 x = len.back();
            len.back() = x - x / 2;
            len.push_back(x / 2);
        }
        for (u64 b = 0, g = 0; g < len.size(); b += len[g], ++g) P.push_back((b_first + b) * mt);
        K = (int)P.size();
        ALLOC(d_cuts, (u64)K * n * sizeof(u64));
        ALLOC(d_pre, (u64)K * (n + 1) * sizeof(u64));
        int lo_prio = 0, hi_prio = 0;
        CK(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
        CK(cudaStreamCreateWithPriority(&xs, cudaStreamNonBlocking, hi_prio));
        CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        CK(cudaEventCreate(&t0));
        ev.assign(K, nullptr);
        for (int g = 0; g < K; ++g) CK(cudaEventCreate(&ev[g]));
        // the copies write buffers the context's stream allocated
        CK(cudaEventRecord(ready, ctx->stream));
        CK(cudaStreamWaitEvent(xs, ready, 0));
        CK(cudaEventRecord(t0, xs));
        for (int g = 0; g < K; ++g) {
            const bool last = g + 1 == K;
            CK(launch_feed_piece(hv, st.ids_buf.as<u64>(), d_off, n, row(g), d_cuts.as<u64>() + (u64)g * n,
                                 last ? 0 : P[g + 1], last, d_pre.as<u64>() + (u64)g * (n + 1), kFeedCtas, xs));
            CK(cudaEventRecord(ev[g], xs));
        }
        ctx->stats.launches += 2 * (u64)K;
        // every piece validated as it arrives, beside the batch loop: the
        // pieces' slices tile every sample, so each value is checked once,
        // against the value before it in its sample (in an earlier piece at a
        // slice's start), and only the last piece's check is left when the
        // copy ends
        int rc = val.open(ctx);
        if (rc) return rc;
        rc = validate_init(ctx, st, val.vs);
        if (rc) return rc;
        for (int g = 0; g < K; ++g) {
            CK(cudaStreamWaitEvent(val.vs, ev[g], 0));
            rc = validate_slices(ctx, st, val.vs, beg(g), end(g));
            if (rc) return rc;
        }
        return val.close();
    }

    // the context's stream waits for piece g
    int wait(int g)
    {
        CK(cudaStreamWaitEvent(ctx->stream, ev[g], 0));
        return JSIM_OK;
    }

    // has piece g arrived on the device?
    bool arrived(int g)
    {
        const cudaError_t e = cudaEventQuery(ev[g]);
        if (e != cudaSuccess) cudaGetLastError();
        return e == cudaSuccess;
    }

    // the context's stream waits for the validation; its verdict and the
    // copy statistics
    int finish(Staged& st)
    {
        int rc = val.finish(ctx, st);
        if (rc) return rc;
        ctx->stats.h2d_pieces += (u64)K;
        ctx->stats.h2d_bytes += st.N * sizeof(u64);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t0, ev[K - 1]) == cudaSuccess) ctx->stats.ms_h2d += ms;
        cudaGetLastError();
        return JSIM_OK;
    }
};

}  // namespace
