// Streamed all-pairs for inputs held in host memory that are too large to
// copy to the device at once (the batch loop of Sec. III-B, Eq. 3 and Eq. 4,
// with each batch's values brought over from host memory as it is needed).
//
// The value range is cut into super-batches: runs of consecutive row batches
// (aligned to m~) whose values fit one pinned staging buffer and whose filter
// bitmaps fit a device budget.  Two staging buffers and two device buffers
// alternate:
//   host:    gather super-batch g+1's values (one contiguous slice of each
//            sample, found by binary search) into pinned staging, with
//            several host threads, while the device multiplies g;
//   copy:    on a second stream, staging -> device buffer, once the device
//            has finished reading that buffer (two super-batches back);
//   compute: validate the slice (distinct counts accumulate: equal values
//            never straddle a boundary); filter and rank-scan the whole
//            super-batch as one batch of the method (Eq. 5, Eq. 6); one
//            synchronisation learns its row count; pack it; one product
//            launch adds its AND+popcount counts into C (Eq. 7, Eq. 4).
// C is accumulated over all super-batches; the epilogue runs once.
//
// Sortedness is checked in two places: on the device inside every slice,
// and on the host across slices (every sample's slices must tile it).  Both
// together imply that every sample is sorted, because a binary search that
// cuts a sample at position q has seen a[q-1] < boundary <= a[q].
//
// Checkpoints: after whole super-batches the state of the call is C so far,
// the sizes, the input-error flags and the statistics; a checkpoint file
// holds them with a header that identifies the call, and a resumed call
// starts at the first super-batch the file does not hold.  C is a sum over
// super-batches (Eq. 4), so the order of additions, and with it every count,
// is that of one uninterrupted call.
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include "ctx.cuh"

// Copy streams of a streamed call: page-locked input is copied slice by
// slice, and slices spread over several streams keep several copy engines
// busy (small copies one after another on one stream leave the link idle
// between them).
constexpr int kCopyStreams = 4;

struct StreamState {
    int device = -1;
    cudaStream_t xs = nullptr;  // copy stream (the first of kCopyStreams)
    cudaStream_t xs_more[kCopyStreams - 1] = {};
    cudaEvent_t fork[2] = {nullptr, nullptr};
    cudaEvent_t joined[2][kCopyStreams - 1] = {};
    u64* pin[2] = {nullptr, nullptr};
    size_t pin_words = 0;
    cudaEvent_t copied[2] = {nullptr, nullptr}, released[2] = {nullptr, nullptr};
};

void jsim_streamed_release(jsim_ctx* ctx)
{
    StreamState* s = ctx->streamed;
    if (!s) return;
    if (s->xs) cudaStreamSynchronize(s->xs);
    for (cudaStream_t x : s->xs_more)
        if (x) cudaStreamSynchronize(x);
    for (int k = 0; k < 2; ++k) {
        if (s->pin[k]) cudaFreeHost(s->pin[k]);
        if (s->copied[k]) cudaEventDestroy(s->copied[k]);
        if (s->released[k]) cudaEventDestroy(s->released[k]);
        if (s->fork[k]) cudaEventDestroy(s->fork[k]);
        for (cudaEvent_t e : s->joined[k])
            if (e) cudaEventDestroy(e);
    }
    if (s->xs) cudaStreamDestroy(s->xs);
    for (cudaStream_t x : s->xs_more)
        if (x) cudaStreamDestroy(x);
    cudaGetLastError();
    delete s;
    ctx->streamed = nullptr;
}

namespace {

// pinned staging of at least `words` u64 each, a copy stream and events
int stream_state(jsim_ctx* ctx, size_t words, StreamState*& out)
{
    if (!ctx->streamed) {
        StreamState* s = new StreamState;
        s->device = ctx->opt.device;
        ctx->streamed = s;
        CK(cudaStreamCreateWithFlags(&s->xs, cudaStreamNonBlocking));
        for (cudaStream_t& x : s->xs_more) CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) {
            CK(cudaEventCreateWithFlags(&s->copied[k], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&s->released[k], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&s->fork[k], cudaEventDisableTiming));
            for (cudaEvent_t& e : s->joined[k]) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
    }
    StreamState* s = ctx->streamed;
    if (s->pin_words < words) {
        CK(cudaStreamSynchronize(s->xs));
        for (int k = 0; k < 2; ++k) {
            if (s->pin[k]) cudaFreeHost(s->pin[k]);
            s->pin[k] = nullptr;
        }
        s->pin_words = 0;
        for (int k = 0; k < 2; ++k) CK(cudaMallocHost((void**)&s->pin[k], words * sizeof(u64)));
        s->pin_words = words;
    }
    out = s;
    return JSIM_OK;
}

struct Super {
    u64 b0 = 0, b1 = 0;  // row batches [b0, b1)
    u64 count = 0;       // values in the super-batch
    std::vector<u64> beg, len, off;  // per sample: slice start, length, staging offset
};

// Per-sample slices of the values below hi (hi == 0: unbounded above), each
// starting at pos[i], the sample's previous cut.  The searches of different
// samples are independent and run on several host threads for large n.
void slice(const std::vector<u64>& hoff, const uint64_t* ids, u64 n, const std::vector<u64>& pos, u64 hi, Super& s)
{
    s.beg.resize(n);
    s.len.resize(n);
    s.off.resize(n + 1);
    auto cut = [&](u64 i0, u64 i1) {
        for (u64 i = i0; i < i1; ++i) {
            const u64 p = pos[i], b = hoff[i + 1];
            const u64 q = hi == 0 ? b : gallop_host(ids, p, b, hi);
            s.beg[i] = p;
            s.len[i] = q - p;
        }
    };
    const unsigned nt = n >= 512 ? std::max(1u, std::min(8u, std::thread::hardware_concurrency())) : 1u;
    if (nt == 1) {
        cut(0, n);
    } else {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t) th.emplace_back(cut, n * t / nt, n * (t + 1) / nt);
        for (auto& x : th) x.join();
    }
    u64 acc = 0;
    for (u64 i = 0; i < n; ++i) {
        s.off[i] = acc;
        acc += s.len[i];
    }
    s.off[n] = acc;
    s.count = acc;
}

// Cuts [min value, max value] into super-batches of at most `cap_vals` values
// and `rb_cap` row batches of `mt` rows each, one at a time (the next one is
// planned on the host while the device multiplies the current one); ranges
// without values are skipped.  Every sample is cut where its values reach a
// boundary, searching forward from its previous cut; together with the
// device's check that every slice is sorted, the cut property (the value
// before a cut is below the boundary, the one at it is not) proves the whole
// sample sorted, and values left over after the last super-batch give
// JSIM_ERR_UNSORTED.  JSIM_ERR_OOM when one row batch alone holds more values
// than the staging.
struct SuperPlanner {
    const std::vector<u64>& hoff;
    const uint64_t* ids;
    u64 n, mt, cap_vals, rb_cap;
    u64 first = 0, last = 0, per0 = 1, b = 0;
    std::vector<u64> pos;
    bool done = false;

    SuperPlanner(const std::vector<u64>& hoff_, const uint64_t* ids_, u64 n_, u64 mt_, u64 cap_vals_, u64 rb_cap_)
        : hoff(hoff_), ids(ids_), n(n_), mt(mt_), cap_vals(cap_vals_), rb_cap(rb_cap_)
    {
    }

    int init()
    {
        u64 minid = ~0ull, maxid = 0;
        for (u64 i = 0; i < n; ++i) {
            const u64 a = hoff[i], e = hoff[i + 1];
            if (e == a) continue;
            if (ids[a] > ids[e - 1]) return JSIM_ERR_UNSORTED;
            minid = std::min<u64>(minid, ids[a]);
            maxid = std::max<u64>(maxid, ids[e - 1]);
        }
        const u64 N = hoff[n];
        pos.assign(hoff.begin(), hoff.end() - 1);
        if (N == 0) {
            done = true;
            return JSIM_OK;
        }
        first = minid / mt;
        last = maxid / mt;
        // row batches per super-batch from the average density, 25 % headroom
        const double per_d = (double)cap_vals / ((double)N / (double)(last - first + 1)) / 1.25;
        per0 = per_d >= (double)rb_cap ? rb_cap : std::max<u64>(1, (u64)per_d);
        b = first;
        return JSIM_OK;
    }

    // the next non-empty super-batch into s (have = false after the last)
    int next(Super& s, bool& have)
    {
        have = false;
        u64 per = per0;
        while (!done) {
            const u64 e = std::min(last + 1, b + per);
            s = Super();
            s.b0 = b;
            s.b1 = e;
            slice(hoff, ids, n, pos, e * mt, s);  // e * mt wraps to 0 only at the top of the range
            if (s.count > cap_vals) {
                if (e - b == 1) return JSIM_ERR_OOM;
                per = (e - b) / 2;  // the same start with half the row batches
                continue;
            }
            u64 maxv = 0;
            for (u64 i = 0; i < n; ++i) {
                pos[i] += s.len[i];
                if (s.len[i]) maxv = std::max<u64>(maxv, ids[s.beg[i] + s.len[i] - 1]);
            }
            if (s.count) s.b1 = std::max(b + 1, std::min(e, maxv / mt + 1));  // drop empty trailing row batches
            // first value at or above the range, to skip empty row batches
            u64 nv = ~0ull;
            bool more = false;
            if (e <= last)
                for (u64 i = 0; i < n; ++i)
                    if (pos[i] < hoff[i + 1]) { more = true; nv = std::min<u64>(nv, ids[pos[i]]); }
            if (!more) {
                done = true;
                for (u64 i = 0; i < n; ++i)
                    if (pos[i] != hoff[i + 1]) return JSIM_ERR_UNSORTED;
            } else {
                b = std::max(e, nv / mt);
            }
            if (s.count) {
                have = true;
                return JSIM_OK;
            }
            per = per0;
        }
        return JSIM_OK;
    }
};

// gather a super-batch's slices into `dst` (pinned) with several host threads
void gather(const uint64_t* ids, const Super& s, u64* dst)
{
    const u64 n = s.beg.size();
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (s.count < (1u << 20)) nt = 1;
    auto work = [&](unsigned t) {
        for (u64 i = t; i < n; i += nt)
            if (s.len[i]) memcpy(dst + s.off[i], ids + s.beg[i], s.len[i] * sizeof(u64));
    };
    if (nt == 1) { work(0); return; }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) th.emplace_back(work, t);
    for (auto& x : th) x.join();
}

// ---- checkpoint file --------------------------------------------------------

// the splitmix64 finaliser (Steele, Lea and Flood, OOPSLA 2014) as a mixer
inline u64 ck_mix(u64 z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct CkHash {
    u64 h = 0x6A09E667F3BCC909ull;
    void word(u64 w) { h = ck_mix(h ^ w); }
    void bytes(const void* p, size_t len)
    {
        const unsigned char* b = (const unsigned char*)p;
        size_t k = 0;
        for (; k + 8 <= len; k += 8) {
            u64 w;
            memcpy(&w, b + k, 8);
            word(w);
        }
        u64 t = 0;
        if (k < len) {
            memcpy(&t, b + k, len - k);
            word(t ^ ((u64)(len - k) << 56));
        }
    }
};

// the collection's identity: offsets, every sample's first and last value
// and 4096 evenly spaced values
u64 ck_fingerprint(const std::vector<u64>& hoff, const uint64_t* ids, u64 n)
{
    CkHash h;
    h.word(n);
    const u64 N = hoff[n];
    h.word(N);
    for (u64 i = 0; i <= n; ++i) h.word(hoff[i]);
    for (u64 i = 0; i < n; ++i)
        if (hoff[i + 1] > hoff[i]) {
            h.word(ids[hoff[i]]);
            h.word(ids[hoff[i + 1] - 1]);
        }
    if (N)
        for (u64 k = 0; k < 4096; ++k) h.word(ids[N * k / 4096]);
    return h.h;
}

struct CkHeader {
    char magic[8];
    u64 version, n, N, mt, cap_vals, count_bits, filter_min, id_bits, distance, supers, fingerprint;
    u64 done;  // super-batches whose counts C holds
    u64 rows_nonzero, batches, words;
    double bitops;
    u64 flags[3];
};
constexpr char kCkMagic[8] = {'J', 'S', 'I', 'M', 'C', 'K', 'P', '1'};

// same call: every identifying field equal
bool ck_same_call(const CkHeader& a, const CkHeader& b)
{
    return memcmp(a.magic, b.magic, 8) == 0 && a.version == b.version && a.n == b.n && a.N == b.N &&
           a.mt == b.mt && a.cap_vals == b.cap_vals && a.count_bits == b.count_bits &&
           a.filter_min == b.filter_min && a.id_bits == b.id_bits && a.distance == b.distance &&
           a.supers == b.supers && a.fingerprint == b.fingerprint;
}

// write header, sizes, C and a checksum to path.tmp, then rename it to path
int ck_write(const char* path, const CkHeader& h, const std::vector<u64>& sizes, const std::vector<unsigned char>& C)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return JSIM_ERR_CHECKPOINT;
    CkHash sum;
    sum.bytes(&h, sizeof h);
    sum.bytes(sizes.data(), sizes.size() * sizeof(u64));
    sum.bytes(C.data(), C.size());
    bool ok = fwrite(&h, sizeof h, 1, f) == 1;
    ok = ok && (sizes.empty() || fwrite(sizes.data(), sizeof(u64), sizes.size(), f) == sizes.size());
    ok = ok && (C.empty() || fwrite(C.data(), 1, C.size(), f) == C.size());
    ok = ok && fwrite(&sum.h, sizeof(u64), 1, f) == 1;
    ok = (fflush(f) == 0) && ok;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return JSIM_ERR_CHECKPOINT;
    }
    return JSIM_OK;
}

// read path into h, sizes and C if it exists (found = false otherwise);
// JSIM_ERR_CHECKPOINT when it is short, corrupt or of another call
int ck_read(const char* path, const CkHeader& want, CkHeader& h, std::vector<u64>& sizes,
            std::vector<unsigned char>& C, bool& found)
{
    found = false;
    FILE* f = fopen(path, "rb");
    if (!f) return JSIM_OK;
    found = true;
    u64 stored = 0;
    bool ok = fread(&h, sizeof h, 1, f) == 1 && ck_same_call(h, want) && h.done <= h.supers;
    if (ok) {
        sizes.resize(h.n);
        C.resize(h.n * h.n * (h.count_bits == 64 ? 8 : 4));
        ok = (sizes.empty() || fread(sizes.data(), sizeof(u64), sizes.size(), f) == sizes.size()) &&
             (C.empty() || fread(C.data(), 1, C.size(), f) == C.size()) && fread(&stored, sizeof(u64), 1, f) == 1;
    }
    if (ok) {
        char extra;
        ok = fread(&extra, 1, 1, f) == 0;  // nothing after the checksum
    }
    fclose(f);
    if (!ok) return JSIM_ERR_CHECKPOINT;
    CkHash sum;
    sum.bytes(&h, sizeof h);
    sum.bytes(sizes.data(), sizes.size() * sizeof(u64));
    sum.bytes(C.data(), C.size());
    return sum.h == stored ? JSIM_OK : JSIM_ERR_CHECKPOINT;
}

// samples up to which page-locked input is copied one slice per sample
constexpr u64 kDirectSlicesMax = 16384;

// waits for the copy stream before device buffers that its copies may still
// write are released (declared after them, so destroyed first)
struct CopyFence {
    StreamState* ss;
    ~CopyFence()
    {
        if (!ss) return;
        if (ss->xs) cudaStreamSynchronize(ss->xs);
        for (cudaStream_t x : ss->xs_more)
            if (x) cudaStreamSynchronize(x);
    }
};

}  // namespace

extern "C" int jsim_all_pairs_streamed(jsim_ctx* ctx, const jsim_sets* sets, void* C, uint64_t* sizes, double* J,
                                       int out_mem, uint64_t staging_bytes)
{
    return jsim_all_pairs_streamed_ckpt(ctx, sets, C, sizes, J, out_mem, staging_bytes, nullptr);
}

extern "C" int jsim_all_pairs_streamed_ckpt(jsim_ctx* ctx, const jsim_sets* sets, void* C, uint64_t* sizes,
                                            double* J, int out_mem, uint64_t staging_bytes,
                                            const jsim_checkpoint* ck)
{
    if (!ctx) return JSIM_ERR_ARG;
    const bool ck_on = ck && ck->path && ck->path[0];
    if (ck && !ck_on && ck->max_supers) return JSIM_ERR_CHECKPOINT;  // progress would be lost
    if (ck && ck->resume != 0 && ck->resume != 1) return JSIM_ERR_ARG;
    int rc = check_sets(sets);
    if (rc) return rc;
    if (sets->mem != JSIM_MEM_HOST) return JSIM_ERR_ARG;  // streaming reads host memory
    if (out_mem != JSIM_MEM_HOST && out_mem != JSIM_MEM_DEVICE) return JSIM_ERR_ARG;
    if (staging_bytes < (1u << 20)) return JSIM_ERR_ARG;
    CK(cudaSetDevice(ctx->opt.device));
    CallScope scope(ctx);
    StageTimer total(ctx, &ctx->stats.ms_total);
    const u64 n = sets->n;
    if (n == 0) return JSIM_OK;
    if (n > (1ull << 20)) return JSIM_ERR_ARG;
    std::vector<u64> hoff;
    rc = load_offsets(ctx, sets, hoff);
    if (rc) return rc;
    const u64 N = hoff[n];
    const uint64_t* ids = sets->ids;
    const size_t cb = ctx->opt.count_bits == 64 ? 8 : 4;
    const u64 cap_vals = staging_bytes / sizeof(u64);
    const u64 head = round_up(n + 1, 32);  // staging: offsets, then values at a 256-byte boundary

    // value range of the call (samples sorted: first and last values)
    u64 minid = ~0ull, maxid = 0;
    for (u64 i = 0; i < n; ++i)
        if (hoff[i + 1] > hoff[i]) {
            minid = std::min<u64>(minid, ids[hoff[i]]);
            maxid = std::max<u64>(maxid, ids[hoff[i + 1] - 1]);
        }
    const u64 span = N && maxid >= minid ? maxid - minid : 0;
    u64 mt = ctx->opt.batch_rows;
    if (!mt) {
        // the automatic batch, halved until a row batch of average density
        // fills at most a quarter of the staging
        mt = auto_batch_rows(span + 1 ? span + 1 : ~0ull);
        const double dens = (double)N / ((double)span + 1.0);
        while (mt > 64 && dens * (double)mt > (double)cap_vals / 4) mt >>= 1;
    }
    ctx->stats.batch_rows = mt;
    // per row batch of the super-batch: bitmap (m~/8 B), rank directory
    // (m~/16 B) and block offsets; at most twice the staging in total
    const u64 nwords = mt / 64;
    const u64 rb_bytes = nwords * (ctx->opt.filter_min == 2 ? 20 : 12) +
                         (nwords + kScanBlockWords - 1) / kScanBlockWords * 16;
    const u64 rb_cap = std::max<u64>(1, std::min<u64>(2 * staging_bytes / rb_bytes, 1u << 16));
    // super-batches: planned one ahead of the device (all of them first when
    // checkpointing, whose file names their count)
    std::deque<Super> sup;  // references stay valid while it grows
    SuperPlanner planner(hoff, ids, n, mt, cap_vals, rb_cap);
    rc = planner.init();
    if (rc) return rc;
    auto plan_upto = [&](size_t g) -> int {
        while (sup.size() <= g && !planner.done) {
            Super x;
            bool have = false;
            int r = planner.next(x, have);
            if (r) return r;
            if (have) sup.push_back(std::move(x));
        }
        return JSIM_OK;
    };
    rc = plan_upto(ck_on ? ~(size_t)0 : 0);
    if (rc) return rc;

    // ---- checkpoint: the call's identity, and the state to resume from ----
    CkHeader ckh{};
    std::vector<u64> ck_sizes;
    std::vector<unsigned char> ck_C;
    bool resumed = false;
    if (ck_on) {
        memcpy(ckh.magic, kCkMagic, 8);
        ckh.version = 1;
        ckh.n = n;
        ckh.N = N;
        ckh.mt = mt;
        ckh.cap_vals = cap_vals;
        ckh.count_bits = (u64)ctx->opt.count_bits;
        ckh.filter_min = (u64)ctx->opt.filter_min;
        ckh.id_bits = (u64)ctx->opt.id_bits;
        ckh.distance = (u64)ctx->opt.distance;
        ckh.supers = sup.size();
        ckh.fingerprint = ck_fingerprint(hoff, ids, n);
        if (ck->resume) {
            CkHeader got{};
            rc = ck_read(ck->path, ckh, got, ck_sizes, ck_C, resumed);
            if (rc) return rc;
            if (resumed) ckh = got;
        }
    }

    // ---- buffers ----
    StreamState* ss = nullptr;
    rc = stream_state(ctx, head + cap_vals, ss);
    if (rc) return rc;
    cudaStream_t cs = ctx->stream, xs = ss->xs;
    // a super-batch spans at most per0 row batches and cap_vals values
    const u64 rb_max = std::max<u64>(1, planner.per0), count_max = cap_vals;
    const u64 nw_max = rb_max * nwords;  // bitmap words of the widest super-batch
    const u64 nbk_max = std::max<u64>((nw_max + kScanBlockWords - 1) / kScanBlockWords, 1);
    DevBuf dbuf[2], Cacc, sizes_d, flags, plan_buf, X, bm, seen, dir, bsum, boff, Rd, Cst, Jst, useful;
    ALLOC(dbuf[0], (head + count_max) * sizeof(u64));
    ALLOC(dbuf[1], (head + count_max) * sizeof(u64));
    CopyFence fence{ss};
    ALLOC(Cacc, n * n * cb);
    ALLOC(sizes_d, n * sizeof(u64));
    ALLOC(flags, 3 * sizeof(u64));
    ALLOC(plan_buf, plan_words(n) * sizeof(u64));
    ALLOC(bm, nw_max * sizeof(u64));  // the rows kept
    const bool twice = ctx->opt.filter_min == 2;
    if (twice) ALLOC(seen, nw_max * sizeof(u64));
    ALLOC(dir, nw_max * sizeof(u32));
    ALLOC(bsum, nbk_max * sizeof(u64));
    ALLOC(boff, nbk_max * sizeof(u64));
    ALLOC(Rd, sizeof(u64));
    if (ctx->opt.count_useful) {
        ALLOC(useful, sizeof(u64));
        CK(cudaMemsetAsync(useful.p, 0, sizeof(u64), cs));
    }
    u64 g0 = 0;  // first super-batch of this call
    if (resumed) {
        g0 = ckh.done;
        CK(cudaMemcpyAsync(Cacc.p, ck_C.data(), n * n * cb, cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(sizes_d.p, ck_sizes.data(), n * sizeof(u64), cudaMemcpyHostToDevice, cs));
        CK(cudaMemcpyAsync(flags.p, ckh.flags, 3 * sizeof(u64), cudaMemcpyHostToDevice, cs));
        CK(cudaStreamSynchronize(cs));  // the host copies are pageable and are released below
        ctx->stats.rows_nonzero = ckh.rows_nonzero;
        ctx->stats.batches = ckh.batches;
        ctx->stats.words = ckh.words;
        ctx->stats.bitops_dense = ckh.bitops;
        std::vector<unsigned char>().swap(ck_C);
    } else {
        CK(cudaMemsetAsync(Cacc.p, 0, n * n * cb, cs));
        CK(cudaMemsetAsync(sizes_d.p, 0, n * sizeof(u64), cs));
        CK(cudaMemsetAsync(flags.p, 0, 2 * sizeof(u64), cs));
        CK(cudaMemsetAsync(flags.as<u64>() + 2, 0xff, sizeof(u64), cs));
    }
    // the state after super-batch g (its product enqueued) into the file
    auto save = [&](u64 done) -> int {
        ckh.done = done;
        ckh.rows_nonzero = ctx->stats.rows_nonzero;
        ckh.batches = ctx->stats.batches;
        ckh.words = ctx->stats.words;
        ckh.bitops = ctx->stats.bitops_dense;
        std::vector<u64> hsz(n);
        std::vector<unsigned char> hc(n * n * cb);
        CK(cudaMemcpyAsync(hc.data(), Cacc.p, n * n * cb, cudaMemcpyDeviceToHost, cs));
        CK(cudaMemcpyAsync(hsz.data(), sizes_d.p, n * sizeof(u64), cudaMemcpyDeviceToHost, cs));
        CK(cudaMemcpyAsync(ctx->h_scalars, flags.p, 3 * sizeof(u64), cudaMemcpyDeviceToHost, cs));
        CK(cudaStreamSynchronize(cs));
        for (int q = 0; q < 3; ++q) ckh.flags[q] = ctx->h_scalars[q];
        return ck_write(ck->path, ckh, hsz, hc);
    };
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(u32), cs));
    const Plan plan = carve_plan(plan_buf, n);
    const u64 n_pad = round_up(n, kRowPad);

    // copy super-batch g into device buffer g & 1 once the device has read
    // what that buffer held two super-batches earlier
    // Page-locked input is copied slice by slice straight from the caller's
    // memory (DMA, no host gather); pageable input is gathered into the
    // pinned staging by host threads first.
    bool direct = false;
    if (N && n <= kDirectSlicesMax) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, ids) == cudaSuccess && pa.type == cudaMemoryTypeHost) direct = true;
        cudaGetLastError();
    }
    auto stage = [&](size_t g) -> int {
        const int k = (int)(g & 1);
        const Super& s = sup[g];
        memcpy(ss->pin[k], s.off.data(), (n + 1) * sizeof(u64));
        if (!direct) gather(ids, s, ss->pin[k] + head);
        CK(cudaStreamWaitEvent(xs, ss->released[k], 0));
        cudaEvent_t a = nullptr;
        if (ctx->opt.profile && (a = take_event(ctx))) cudaEventRecord(a, xs);
        if (direct) {
            // slices in kCopyStreams contiguous groups of about equal bytes,
            // one group per copy stream (forked from and joined back to xs)
            CK(cudaMemcpyAsync(dbuf[k].p, ss->pin[k], head * sizeof(u64), cudaMemcpyHostToDevice, xs));
            ctx->stats.h2d_copies += 1;
            CK(cudaEventRecord(ss->fork[k], xs));
            for (cudaStream_t x : ss->xs_more) CK(cudaStreamWaitEvent(x, ss->fork[k], 0));
            u64 i = 0;
            for (int q = 0; q < kCopyStreams; ++q) {
                cudaStream_t x = q == 0 ? xs : ss->xs_more[q - 1];
                const u64 upto = s.count * (u64)(q + 1) / kCopyStreams;  // this group ends at offset `upto`
                for (; i < n && (q == kCopyStreams - 1 || s.off[i] < upto); ++i)
                    if (s.len[i]) {
                        CK(cudaMemcpyAsync(dbuf[k].as<u64>() + head + s.off[i], ids + s.beg[i],
                                           s.len[i] * sizeof(u64), cudaMemcpyHostToDevice, x));
                        ctx->stats.h2d_copies += 1;
                    }
            }
            for (int q = 1; q < kCopyStreams; ++q) {
                CK(cudaEventRecord(ss->joined[k][q - 1], ss->xs_more[q - 1]));
                CK(cudaStreamWaitEvent(xs, ss->joined[k][q - 1], 0));
            }
        } else {
            CK(cudaMemcpyAsync(dbuf[k].p, ss->pin[k], (head + s.count) * sizeof(u64), cudaMemcpyHostToDevice, xs));
            ctx->stats.h2d_copies += 1;
        }
        ctx->stats.h2d_bytes += (head + s.count) * sizeof(u64);
        if (a) {
            cudaEvent_t b = take_event(ctx);
            if (b) {
                cudaEventRecord(b, xs);
                ctx->pending.push_back({a, b, &ctx->stats.ms_h2d});
            }
        }
        CK(cudaEventRecord(ss->copied[k], xs));
        return JSIM_OK;
    };
    for (int k = 0; k < 2; ++k) CK(cudaEventRecord(ss->released[k], cs));
    if (g0 < sup.size()) {
        rc = stage(g0);
        if (rc) return rc;
    }
    // Every super-batch is one batch of the method (Eq. 3) spanning its row
    // batches: one filter, one rank scan and one pack over [lo, lo + width).
    // C is additive over any partition of the rows (Eq. 4), so grouping row
    // batches changes no count; it only packs fewer, longer rows.
    for (size_t g = g0; g < sup.size(); ++g) {
        const int k = (int)(g & 1);
        const Super& s = sup[g];
        const u64* d_off = dbuf[k].as<u64>();
        const u64* d_ids = dbuf[k].as<u64>() + head;
        const u64 max_chunks = s.count / kChunk + n + 1;
        const u64 lo = s.b0 * mt, width = (s.b1 - s.b0) * mt, nw = width / 64;
        CK(cudaStreamWaitEvent(cs, ss->copied[k], 0));
        {
            // the plan covers every value of the slice, all inside [lo, lo + width)
            StageTimer t(ctx, &ctx->stats.ms_validate);
            CK(launch_plan(d_off, d_ids, n, 0, 0, true, plan, cs));
            CK(launch_validate(d_off, d_ids, n, plan, max_chunks, ctx->opt.id_bits, sizes_d.as<u64>(),
                               flags.as<u32>(), flags.as<u64>() + 1, flags.as<u64>() + 2, ctx->sms, cs));
            ctx->stats.launches += 2;
        }
        {
            StageTimer t(ctx, &ctx->stats.ms_filter);
            CK(cudaMemsetAsync(bm.p, 0, nw * sizeof(u64), cs));
            if (twice) {
                CK(cudaMemsetAsync(seen.p, 0, nw * sizeof(u64), cs));
                CK(launch_filter(d_ids, n, plan, max_chunks, lo, width, seen.as<u32>(), ctx->sms, cs, bm.as<u32>()));
            } else {
                CK(launch_filter(d_ids, n, plan, max_chunks, lo, width, bm.as<u32>(), ctx->sms, cs));
            }
            ctx->stats.launches += 1;
        }
        {
            StageTimer t(ctx, &ctx->stats.ms_scan);
            CK(launch_scan(bm.as<u64>(), nw, dir.as<u32>(), bsum.as<u64>(), boff.as<u64>(), Rd.as<u64>(), cs));
            ctx->stats.launches += 2;
        }
        CK(cudaMemcpyAsync(ctx->h_scalars, Rd.p, sizeof(u64), cudaMemcpyDeviceToHost, cs));
        CK(cudaMemcpyAsync(ctx->h_scalars + 1, flags.p, sizeof(u64), cudaMemcpyDeviceToHost, cs));
        CK(cudaStreamSynchronize(cs));
        {
            // an input error found by this or an earlier slice's validation
            // ends the call before the pack (an unsorted slice may hold values
            // outside the super-batch's range)
            const u32 f = (u32)ctx->h_scalars[1];
            if (f & kFlagUnsorted) return JSIM_ERR_UNSORTED;
            if (f & kFlagIdRange) return JSIM_ERR_ID_RANGE;
        }
        const u64 R = ctx->h_scalars[0], W = (R + 63) / 64;
        ctx->stats.rows_nonzero += R;
        ctx->stats.batches += R != 0;
        const u64 stride = row_stride_words(W);
        if (W) {
            ALLOC(X, n_pad * stride * sizeof(u64));
            StageTimer t(ctx, &ctx->stats.ms_pack);
            CK(launch_zero_rows(X.as<u64>(), n_pad, stride, stride, ctx->sms, cs));
            CK(launch_pack_full(d_ids, n, plan, max_chunks, lo, width, bm.as<u64>(), dir.as<u32>(),
                                boff.as<u64>(), X.as<u64>(), stride, Rd.as<u64>(), ctx->sms, cs));
            ctx->stats.launches += 2;
            ctx->stats.pack_bytes += 8 * s.count + 8 * n_pad * stride;
        }
        CK(cudaEventRecord(ss->released[k], cs));  // the slice's values are no longer read
        if (W) {
            const int v = ctx->opt.variant == JSIM_VARIANT_AUTO ? choose_variant(ctx, n, W) : ctx->opt.variant;
            StageTimer t(ctx, &ctx->stats.ms_product);
            rc = run_product(ctx, v, X.as<u64>(), stride, n, W, Cacc.p);
            if (rc) return rc;
            if (ctx->opt.count_useful)
                CK(launch_useful(X.as<u64>(), n, stride, W, useful.as<u64>(), ctx->sms, cs));
            ctx->stats.words += W;
            ctx->stats.bitops_dense += 64.0 * (double)W * (double)n * (double)(n + 1) / 2.0;
        }
        if (ck_on && g + 1 < sup.size()) {
            const bool stop = ck->max_supers && g + 1 - g0 >= ck->max_supers;
            if (stop || (ck->every && (g + 1) % ck->every == 0)) {
                rc = save(g + 1);
                if (rc) return rc;
            }
            if (stop) return JSIM_ERR_INCOMPLETE;
        }
        // the next super-batch is planned, gathered and copied while this one
        // multiplies
        rc = plan_upto(g + 1);
        if (rc) return rc;
        if (g + 1 < sup.size()) {
            rc = stage(g + 1);
            if (rc) return rc;
        }
    }

    // ---- input errors, epilogue ----
    CK(cudaMemcpyAsync(ctx->h_scalars, flags.p, sizeof(u64), cudaMemcpyDeviceToHost, cs));
    CK(cudaMemcpyAsync(ctx->h_scalars + 2, ctx->d_err, sizeof(u32), cudaMemcpyDeviceToHost, cs));
    std::vector<u64> hs(n);
    CK(cudaMemcpyAsync(hs.data(), sizes_d.p, n * sizeof(u64), cudaMemcpyDeviceToHost, cs));
    CK(cudaStreamSynchronize(cs));
    const u32 f = (u32)ctx->h_scalars[0];
    if (f & kFlagUnsorted) return JSIM_ERR_UNSORTED;
    if (f & kFlagIdRange) return JSIM_ERR_ID_RANGE;
    // nothing is written when a bounded device wait ran out
    if ((u32)ctx->h_scalars[2] != 0) return JSIM_ERR_TIMEOUT;
    if (ctx->opt.count_bits == 32)
        for (u64 v : hs)
            if (v > 0xffffffffull) return JSIM_ERR_OVERFLOW;
    void* Cdst = C;
    double* Jdst = J;
    if (out_mem == JSIM_MEM_HOST) {
        if (C) { ALLOC(Cst, n * n * cb); Cdst = Cst.p; }
        if (J) { ALLOC(Jst, n * n * sizeof(double)); Jdst = Jst.as<double>(); }
    }
    {
        StageTimer t(ctx, &ctx->stats.ms_epilogue);
        if (Cdst || Jdst) {
            CK(launch_epilogue(Cacc.p, n, ctx->opt.count_bits, sizes_d.as<u64>(), Cdst, Jdst, cs, twice,
                               ctx->opt.distance));
            ctx->stats.launches += 1;
        }
    }
    {
        StageTimer t(ctx, &ctx->stats.ms_d2h);
        const cudaMemcpyKind kind = out_mem == JSIM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        if (out_mem == JSIM_MEM_HOST) {
            if (C) CK(cudaMemcpyAsync(C, Cst.p, n * n * cb, kind, cs));
            if (J) CK(cudaMemcpyAsync(J, Jst.p, n * n * sizeof(double), kind, cs));
        }
        if (sizes) CK(cudaMemcpyAsync(sizes, sizes_d.p, n * sizeof(u64), kind, cs));
    }
    CK(cudaMemcpyAsync(ctx->h_scalars, ctx->d_err, sizeof(u32), cudaMemcpyDeviceToHost, cs));
    if (ctx->opt.count_useful)
        CK(cudaMemcpyAsync(ctx->h_scalars + 1, useful.p, sizeof(u64), cudaMemcpyDeviceToHost, cs));
    CK(cudaStreamSynchronize(cs));
    if (ctx->opt.count_useful) ctx->stats.bitops_useful = 64.0 * (double)ctx->h_scalars[1];
    if ((u32)ctx->h_scalars[0] != 0) return JSIM_ERR_TIMEOUT;
    return JSIM_OK;
}
