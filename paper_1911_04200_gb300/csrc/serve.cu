// Serving: a resident reference index and a continuous-batching query
// server (one worker thread per index).
//
// jsim_index_build packs the reference once, as one batch of the method
// (Sec. III-B): filter over its whole value range (Eq. 5), rank directory
// (Eq. 6), and the kept rows of Abar_ref rank-major (row r: which reference
// samples hold it).  Queries against it need no pass over the reference:
// each query value is ranked against the resident filter (values the
// reference lacks count in |Q| only) and reads one row.
//
// Requests are submitted from any thread.  The worker owns `slots` device
// batches; whenever a slot is free it admits queued requests in arrival
// order while the batch's sample and value capacity allow, gathers their
// values into the slot's pinned staging and launches copy, validation,
// ranking, product and epilogue on the slot's stream.  Requests that arrive
// while batches run wait only for a free slot, and the slots' work overlaps
// on the device.  A request's results depend only on its own samples: the
// batch it lands in changes no count.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <functional>
#include <mutex>
#include <memory>
#include <thread>
#include <unordered_set>
#include "ctx.cuh"

namespace {

enum { kReqQueued = 0, kReqRunning = 1, kReqDone = 2 };

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct jsim_request {
    jsim_index* idx = nullptr;
    u64 q = 0, nvals = 0;
    std::vector<u64> off;      // q + 1 (the caller's offsets, copied)
    const uint64_t* ids = nullptr;  // the caller's values (read until completion)
    std::vector<unsigned char> C;
    std::vector<u64> sizes;
    std::vector<double> J;
    int state = kReqQueued;
    int status = JSIM_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
};

namespace {

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evp0 = nullptr, evp1 = nullptr;
    u64* pin_in = nullptr;     // [offsets S+1][pad][values]
    unsigned char* pin_out = nullptr;
    size_t out_bytes = 0;
    DevBuf din, plan_buf, sq, qerr, mm, Ud, Cacc, Cout, Jd;
    std::vector<jsim_request*> reqs;
    u64 S = 0;
    bool busy = false;
};

}  // namespace

struct GatherPool;

struct jsim_index {
    jsim_ctx* ctx = nullptr;
    jsim_serve_options opt{};
    u64 n_ref = 0, ns64 = 0, lo = 0, width = 0, R = 0;
    DevBuf X, bm, dir, boff, fr, sizes_ref;
    std::vector<u64> h_sizes_ref;
    std::vector<std::unique_ptr<Slot>> slots;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<jsim_request*> queue;
    std::unordered_set<jsim_request*> live;  // requests not yet freed
    bool stop = false;
    jsim_serve_stats stats{};
    int device = 0, sms = 0, count_bits = 32, distance = 0;
    std::unique_ptr<GatherPool> gather;  // host threads that gather query values
    ~jsim_index();
};

namespace {

QueryIndex view(const jsim_index* ix)
{
    QueryIndex q;
    q.index = ix->X.as<u64>();
    q.bm = ix->bm.as<u64>();
    q.dir = ix->dir.as<u32>();
    q.boff = ix->boff.as<u64>();
    q.fr = ix->fr.as<ulonglong2>();
    q.lo = ix->lo;
    q.width = ix->width;
    q.R = ix->R;
    q.n_ref = ix->n_ref;
    q.ns64 = ix->ns64;
    return q;
}

// layout of a slot's pinned output: C, J, sizes, per-sample flags, U
struct OutLayout {
    size_t c, j, s, f, u, total;
};

OutLayout out_layout(u64 S, u64 n_ref, size_t cb)
{
    OutLayout o;
    o.c = 0;
    o.j = round_up(S * n_ref * cb, 256);
    o.s = o.j + round_up(S * n_ref * sizeof(double), 256);
    o.f = o.s + round_up(S * sizeof(u64), 256);
    o.u = o.f + round_up(S * sizeof(u32), 256);
    o.total = o.u + 256;
    return o;
}

// Build-time tuning: host threads that gather a batch's query values (the
// server thread and JSIM_GATHER_THREADS - 1 pool threads started with the
// index) and the batch size below which one thread copies alone.
#ifndef JSIM_GATHER_THREADS
#define JSIM_GATHER_THREADS 16
#endif
#ifndef JSIM_GATHER_MIN_PER_THREAD
#define JSIM_GATHER_MIN_PER_THREAD (1u << 18)
#endif

}  // namespace

// Threads that copy parts of a batch's query values, started with the index
// and idle between batches (no thread start per batch).
struct GatherPool {
    std::vector<std::thread> th;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::function<void(unsigned)> job;
    unsigned parts = 0, next = 0, done = 0;
    bool stop = false;
    void start(unsigned n)
    {
        for (unsigned t = 0; t < n; ++t) th.emplace_back([this] { loop(); });
    }
    void loop()
    {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv.wait(lk, [&] { return stop || next < parts; });
            if (stop) return;
            const unsigned p = next++;
            lk.unlock();
            job(p);
            lk.lock();
            if (++done == parts) cv_done.notify_all();
        }
    }
    // run f(0) .. f(parts - 1), part 0 on the calling thread
    void run(unsigned nparts, const std::function<void(unsigned)>& f)
    {
        {
            std::lock_guard<std::mutex> lk(mu);
            job = f;
            parts = nparts;
            next = 1;
            done = 0;
        }
        cv.notify_all();
        f(0);
        std::unique_lock<std::mutex> lk(mu);
        if (++done != parts) cv_done.wait(lk, [&] { return done == parts; });
        parts = next = 0;
    }
    ~GatherPool()
    {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv.notify_all();
        for (auto& t : th) t.join();
    }
};

jsim_index::~jsim_index() = default;

namespace {

void gather_values(GatherPool& pool, const std::vector<jsim_request*>& reqs, u64* dst)
{
    u64 total = 0;
    for (auto* r : reqs) total += r->nvals;
    struct Piece { const uint64_t* src; u64* dst; u64 n; };
    std::vector<Piece> pieces;
    u64 at = 0;
    for (auto* r : reqs) {
        if (r->nvals) pieces.push_back({r->ids, dst + at, r->nvals});
        at += r->nvals;
    }
    const u64 want = std::max<u64>(1, total / JSIM_GATHER_MIN_PER_THREAD);
    const unsigned nt = (unsigned)std::min<u64>(want, pool.th.size() + 1);
    // split every piece into nt parts so one large request is copied in parallel
    auto work = [&](unsigned t) {
        for (auto& p : pieces) {
            const u64 a = p.n * t / nt, b = p.n * (t + 1) / nt;
            if (b > a) memcpy(p.dst + a, p.src + a, (b - a) * sizeof(u64));
        }
    };
    if (nt == 1) {
        work(0);
        return;
    }
    pool.run(nt, work);
}

// Launch one batch on a free slot (worker thread; the slot's pinned input is
// not in use).  Returns a jsim error code.
int launch_batch(jsim_index* ix, Slot& sl)
{
    jsim_ctx* ctx = ix->ctx;
    const size_t cb = ix->count_bits == 64 ? 8 : 4;
    u64 S = 0, V = 0;
    for (auto* r : sl.reqs) { S += r->q; V += r->nvals; }
    sl.S = S;
    const u64 head = round_up(S + 1, 32);
    // offsets of the concatenated query samples
    u64* off = sl.pin_in;
    u64 at = 0, k = 0;
    for (auto* r : sl.reqs) {
        for (u64 i = 0; i < r->q; ++i) off[k++] = at + r->off[i];
        at += r->nvals;
    }
    off[S] = V;
    gather_values(*ix->gather, sl.reqs, sl.pin_in + head);
    cudaStream_t st = sl.st;
    const u64* d_off = sl.din.as<u64>();
    const u64* d_ids = sl.din.as<u64>() + head;
    const u64 max_chunks = V / kChunk + S + 1;
    const Plan plan = carve_plan(sl.plan_buf, S);
    const QueryIndex qi = view(ix);
    const OutLayout ol = out_layout(S, ix->n_ref, cb);
    CK(cudaEventRecord(sl.ev0, st));
    CK(cudaMemcpyAsync(sl.din.p, sl.pin_in, (head + V) * sizeof(u64), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(sl.sq.p, 0, S * sizeof(u64), st));
    CK(cudaMemsetAsync(sl.qerr.p, 0, S * sizeof(u32), st));
    CK(launch_plan(d_off, d_ids, S, 0, 0, true, plan, st));
    CK(launch_validate(d_off, d_ids, S, plan, max_chunks, ctx->opt.id_bits, sl.sq.as<u64>(), sl.qerr.as<u32>(),
                       sl.mm.as<u64>(), sl.mm.as<u64>() + 1, ix->sms, st, 1));
    CK(cudaMemsetAsync(sl.Cacc.p, 0, S * ix->n_ref * sizeof(u32), st));
    CK(cudaMemsetAsync(sl.Ud.p, 0, sizeof(u64), st));
    CK(cudaEventRecord(sl.evp0, st));
    CK(launch_qrows(d_ids, S, plan, V, qi, sl.Cacc.as<u32>(), sl.Ud.as<u64>(), ix->sms, st));
    CK(cudaEventRecord(sl.evp1, st));
    CK(launch_qepi(sl.Cacc.as<u32>(), S, ix->n_ref, sl.sq.as<u64>(), ix->sizes_ref.as<u64>(), ix->count_bits,
                   sl.Cout.p, sl.Jd.as<double>(), ix->sms, st, ix->distance));
    unsigned char* po = sl.pin_out;
    CK(cudaMemcpyAsync(po + ol.c, sl.Cout.p, S * ix->n_ref * cb, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(po + ol.j, sl.Jd.p, S * ix->n_ref * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(po + ol.s, sl.sq.p, S * sizeof(u64), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(po + ol.f, sl.qerr.p, S * sizeof(u32), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(po + ol.u, sl.Ud.p, sizeof(u64), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(sl.ev1, st));
    return JSIM_OK;
}

// Hand a finished batch's results to its requests (worker thread, lock not held).
void retire(jsim_index* ix, Slot& sl, cudaError_t done)
{
    const size_t cb = ix->count_bits == 64 ? 8 : 4;
    const u64 n_ref = ix->n_ref;
    const OutLayout ol = out_layout(sl.S, n_ref, cb);
    const unsigned char* po = sl.pin_out;
    float ms = 0.f, msp = 0.f;
    if (done == cudaSuccess) {
        cudaEventElapsedTime(&ms, sl.ev0, sl.ev1);
        cudaEventElapsedTime(&msp, sl.evp0, sl.evp1);
    }
    cudaGetLastError();
    u64 s0 = 0;
    for (auto* r : sl.reqs) {
        if (done != cudaSuccess) {
            r->status = JSIM_ERR_CUDA;
        } else {
            u32 f = 0;
            for (u64 i = 0; i < r->q; ++i) f |= ((const u32*)(po + ol.f))[s0 + i];
            if (f & kFlagUnsorted) r->status = JSIM_ERR_UNSORTED;
            else if (f & kFlagIdRange) r->status = JSIM_ERR_ID_RANGE;
            else {
                r->C.resize(r->q * n_ref * cb);
                r->J.resize(r->q * n_ref);
                r->sizes.resize(r->q);
                memcpy(r->C.data(), po + ol.c + s0 * n_ref * cb, r->q * n_ref * cb);
                memcpy(r->J.data(), po + ol.j + s0 * n_ref * sizeof(double), r->q * n_ref * sizeof(double));
                memcpy(r->sizes.data(), po + ol.s + s0 * sizeof(u64), r->q * sizeof(u64));
                if (ix->count_bits == 32)
                    for (u64 v : r->sizes)
                        if (v > 0xffffffffull) r->status = JSIM_ERR_OVERFLOW;
            }
        }
        s0 += r->q;
    }
    const u64 rows = done == cudaSuccess ? *(const u64*)(po + ol.u) : 0;
    std::lock_guard<std::mutex> lk(ix->mu);
    const double t = now_ms();
    for (auto* r : sl.reqs) {
        r->state = kReqDone;
        r->t_done = t;
        ix->stats.requests_done += 1;
        ix->stats.samples_done += r->q;
        ix->stats.values_done += r->nvals;
    }
    ix->stats.batches += 1;
    ix->stats.ms_device += ms;
    ix->stats.ms_product += msp;
    ix->stats.rows_read += rows;
    ix->stats.index_bytes_read += (double)rows * (double)ix->ns64 * 8.0;
    ix->stats.bitops_dense += (double)rows * (double)n_ref;
    sl.reqs.clear();
    sl.busy = false;
    ix->cv_done.notify_all();
}

void worker_main(jsim_index* ix)
{
    cudaSetDevice(ix->device);
    std::unique_lock<std::mutex> lk(ix->mu);
    for (;;) {
        bool progressed = false;
        for (auto& sp : ix->slots) {
            Slot& sl = *sp;
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev1);
            if (q == cudaErrorNotReady) continue;
            lk.unlock();
            retire(ix, sl, q);
            lk.lock();
            progressed = true;
        }
        for (auto& sp : ix->slots) {
            Slot& sl = *sp;
            if (sl.busy || ix->queue.empty()) continue;
            u64 S = 0, V = 0;
            const double t = now_ms();
            while (!ix->queue.empty()) {
                jsim_request* r = ix->queue.front();
                if (!sl.reqs.empty() && (S + r->q > ix->opt.max_batch_samples || V + r->nvals > ix->opt.max_batch_values))
                    break;
                ix->queue.pop_front();
                r->state = kReqRunning;
                r->t_start = t;
                sl.reqs.push_back(r);
                S += r->q;
                V += r->nvals;
            }
            sl.busy = true;
            lk.unlock();
            const int rc = launch_batch(ix, sl);
            if (rc != JSIM_OK) {
                cudaStreamSynchronize(sl.st);
                cudaGetLastError();
                lk.lock();
                for (auto* r : sl.reqs) {
                    r->status = rc;
                    r->state = kReqDone;
                    r->t_done = now_ms();
                }
                sl.reqs.clear();
                sl.busy = false;
                ix->cv_done.notify_all();
            } else {
                lk.lock();
            }
            progressed = true;
        }
        bool any_busy = false;
        for (auto& sp : ix->slots) any_busy |= sp->busy;
        if (ix->stop && ix->queue.empty() && !any_busy) break;
        if (progressed) continue;
        if (!any_busy)
            ix->cv_work.wait(lk, [&] { return ix->stop || !ix->queue.empty(); });
        else
            ix->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
}

void free_slots(jsim_index* ix)
{
    for (auto& sp : ix->slots) {
        Slot& sl = *sp;
        if (sl.st) cudaStreamSynchronize(sl.st);
        for (DevBuf* b : {&sl.din, &sl.plan_buf, &sl.sq, &sl.qerr, &sl.mm, &sl.Ud, &sl.Cacc, &sl.Cout, &sl.Jd})
            b->release();
        if (sl.pin_in) cudaFreeHost(sl.pin_in);
        if (sl.pin_out) cudaFreeHost(sl.pin_out);
        if (sl.ev0) cudaEventDestroy(sl.ev0);
        if (sl.ev1) cudaEventDestroy(sl.ev1);
        if (sl.evp0) cudaEventDestroy(sl.evp0);
        if (sl.evp1) cudaEventDestroy(sl.evp1);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    ix->slots.clear();
    cudaGetLastError();
}

}  // namespace

extern "C" {

void jsim_serve_default_options(jsim_serve_options* o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->max_batch_samples = 64;
    o->max_batch_values = 1ull << 27;
    o->slots = 3;
}

int jsim_index_build(jsim_ctx* ctx, const jsim_sets* ref, const jsim_serve_options* opt, jsim_index** out)
{
    if (!ctx || !out) return JSIM_ERR_ARG;
    *out = nullptr;
    int rc = check_sets(ref);
    if (rc) return rc;
    jsim_serve_options o;
    if (opt) o = *opt; else jsim_serve_default_options(&o);
    if (o.max_batch_samples < 1 || o.max_batch_samples > 64 || o.max_batch_values < 1 ||
        o.max_batch_values >= (1ull << 32) || o.slots < 1 || o.slots > 8)
        return JSIM_ERR_ARG;
    CK(cudaSetDevice(ctx->opt.device));
    CallScope scope(ctx);
    std::vector<u64> hoff;
    rc = load_offsets(ctx, ref, hoff);
    if (rc) return rc;
    if (ref->n == 0) return JSIM_ERR_ARG;
    Staged st;
    rc = stage_and_validate(ctx, ref, st, hoff);
    if (rc) return rc;
    jsim_index* ix = new jsim_index;
    struct Guard { jsim_index*& p; ~Guard() { if (p) { free_slots(p); delete p; } } } guard{ix};
    ix->ctx = ctx;
    ix->opt = o;
    ix->device = ctx->opt.device;
    ix->sms = ctx->sms;
    ix->count_bits = ctx->opt.count_bits;
    ix->distance = ctx->opt.distance;
    const u64 n = ref->n;
    ix->n_ref = n;
    ix->ns64 = (n + 63) / 64;
    if (ix->ns64 > 128) return JSIM_ERR_UNSUPPORTED;  // rows of more than 8192 reference samples
    cudaStream_t cs = ctx->stream;
    // the reference as one batch over its value range
    if (st.N) {
        const u64 span = st.maxid - st.minid;
        if (span >= (1ull << 36)) return JSIM_ERR_UNSUPPORTED;  // filter bitmap above 8 GiB
        ix->lo = st.minid / 64 * 64;
        ix->width = round_up(st.maxid - ix->lo + 1, 64);
        const u64 nw = ix->width / 64, nbk = (nw + kScanBlockWords - 1) / kScanBlockWords;
        DevBuf bsum, R;
        ALLOC(ix->bm, nw * sizeof(u64));
        ALLOC(ix->dir, nw * sizeof(u32));
        ALLOC(ix->boff, nbk * sizeof(u64));
        ALLOC(bsum, nbk * sizeof(u64));
        ALLOC(R, sizeof(u64));
        CK(cudaMemsetAsync(ix->bm.p, 0, nw * sizeof(u64), cs));
        CK(launch_plan(st.d_off, st.d_ids, n, 0, 0, true, st.plan, cs));
        CK(launch_filter(st.d_ids, n, st.plan, st.max_chunks, ix->lo, ix->width, ix->bm.as<u32>(), ctx->sms, cs));
        CK(launch_scan(ix->bm.as<u64>(), nw, ix->dir.as<u32>(), bsum.as<u64>(), ix->boff.as<u64>(), R.as<u64>(), cs));
        CK(cudaMemcpyAsync(ctx->h_scalars, R.p, sizeof(u64), cudaMemcpyDeviceToHost, cs));
        CK(cudaStreamSynchronize(cs));
        ix->R = ctx->h_scalars[0];
        ALLOC(ix->X, std::max<u64>(ix->R, 1) * ix->ns64 * sizeof(u64));
        CK(cudaMemsetAsync(ix->X.p, 0, ix->R * ix->ns64 * sizeof(u64), cs));
        CK(launch_pack_rows(st.d_ids, n, st.plan, st.max_chunks, view(ix), ix->X.as<u64>(), ctx->sms, cs));
        // queries rank through one 16-byte entry per filter word; the
        // separate bitmap, directory and block offsets are build-only
        ALLOC(ix->fr, nw * sizeof(ulonglong2));
        CK(launch_rank_words(view(ix), ix->fr.as<ulonglong2>(), ctx->sms, cs));
        CK(cudaStreamSynchronize(cs));
        ix->bm.release();
        ix->dir.release();
        ix->boff.release();
    }
    ALLOC(ix->sizes_ref, n * sizeof(u64));
    CK(cudaMemcpyAsync(ix->sizes_ref.p, st.sizes.p, n * sizeof(u64), cudaMemcpyDeviceToDevice, cs));
    ix->h_sizes_ref.resize(n);
    CK(cudaMemcpyAsync(ix->h_sizes_ref.data(), st.sizes.p, n * sizeof(u64), cudaMemcpyDeviceToHost, cs));
    // slots
    const u64 S = o.max_batch_samples, V = o.max_batch_values;
    const size_t cb = ix->count_bits == 64 ? 8 : 4;
    const u64 head = round_up(S + 1, 32);
    for (int k = 0; k < o.slots; ++k) ix->slots.emplace_back(new Slot);
    for (auto& sp : ix->slots) {
        Slot& sl = *sp;
        CK(cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking));
        CK(cudaEventCreate(&sl.ev0));
        CK(cudaEventCreate(&sl.ev1));
        CK(cudaEventCreate(&sl.evp0));
        CK(cudaEventCreate(&sl.evp1));
        CK(cudaMallocHost((void**)&sl.pin_in, (head + V) * sizeof(u64)));
        sl.out_bytes = out_layout(S, n, cb).total;
        CK(cudaMallocHost((void**)&sl.pin_out, sl.out_bytes));
        ALLOC(sl.din, (head + V) * sizeof(u64));
        ALLOC(sl.plan_buf, plan_words(S) * sizeof(u64));
        ALLOC(sl.sq, S * sizeof(u64));
        ALLOC(sl.qerr, S * sizeof(u32));
        ALLOC(sl.mm, 2 * sizeof(u64));
        ALLOC(sl.Ud, sizeof(u64));
        ALLOC(sl.Cacc, S * n * sizeof(u32));
        ALLOC(sl.Cout, S * n * cb);
        ALLOC(sl.Jd, S * n * sizeof(double));
    }
    CK(cudaStreamSynchronize(cs));
    ix->gather.reset(new GatherPool);
    ix->gather->start(std::max(1u, std::min((unsigned)JSIM_GATHER_THREADS, std::thread::hardware_concurrency())) - 1);
    ix->worker = std::thread(worker_main, ix);
    *out = ix;
    ix = nullptr;  // the guard keeps it
    return JSIM_OK;
}

void jsim_index_destroy(jsim_index* ix)
{
    if (!ix) return;
    {
        std::lock_guard<std::mutex> lk(ix->mu);
        for (auto* r : ix->queue) {
            r->status = JSIM_ERR_CANCELLED;
            r->state = kReqDone;
            r->t_done = now_ms();
            r->idx = nullptr;
        }
        ix->queue.clear();
        ix->stop = true;
        ix->cv_work.notify_all();
        ix->cv_done.notify_all();
    }
    if (ix->worker.joinable()) ix->worker.join();
    for (auto* r : ix->live) r->idx = nullptr;  // they outlive the index
    cudaSetDevice(ix->device);
    free_slots(ix);
    cudaStreamSynchronize(ix->ctx->stream);
    delete ix;
}

int jsim_index_info(const jsim_index* ix, uint64_t* n_ref, uint64_t* words, uint64_t* ref_sizes)
{
    if (!ix) return JSIM_ERR_ARG;
    if (n_ref) *n_ref = ix->n_ref;
    if (words) *words = ix->R;
    if (ref_sizes) memcpy(ref_sizes, ix->h_sizes_ref.data(), ix->n_ref * sizeof(u64));
    return JSIM_OK;
}

int jsim_index_stats(jsim_index* ix, jsim_serve_stats* out)
{
    if (!ix || !out) return JSIM_ERR_ARG;
    std::lock_guard<std::mutex> lk(ix->mu);
    *out = ix->stats;
    out->queued = ix->queue.size();
    return JSIM_OK;
}

int jsim_query_submit(jsim_index* ix, const jsim_sets* q, jsim_request** out)
{
    if (!ix || !q || !out) return JSIM_ERR_ARG;
    *out = nullptr;
    if (q->mem != JSIM_MEM_HOST || !q->offsets) return JSIM_ERR_ARG;
    const double t0 = now_ms();
    jsim_request* r = new jsim_request;
    r->idx = ix;
    r->q = q->n;
    r->off.assign(q->offsets, q->offsets + q->n + 1);
    if (r->off[0] != 0) { delete r; return JSIM_ERR_ARG; }
    for (u64 i = 0; i < r->q; ++i)
        if (r->off[i + 1] < r->off[i]) { delete r; return JSIM_ERR_ARG; }
    r->nvals = r->off[r->q];
    if (r->nvals && !q->ids) { delete r; return JSIM_ERR_ARG; }
    if (r->q > ix->opt.max_batch_samples || r->nvals > ix->opt.max_batch_values) { delete r; return JSIM_ERR_ARG; }
    r->ids = q->ids;
    r->t_submit = t0;
    std::lock_guard<std::mutex> lk(ix->mu);
    if (ix->stop) { delete r; return JSIM_ERR_CANCELLED; }
    ix->live.insert(r);
    if (r->q == 0) {
        r->state = kReqDone;
        r->t_start = r->t_done = t0;
    } else {
        ix->queue.push_back(r);
        ix->stats.requests_submitted += 1;
        ix->cv_work.notify_one();
    }
    *out = r;
    return JSIM_OK;
}

int jsim_request_wait(jsim_request* r, void* C, uint64_t* qsizes, double* J, int timeout_ms)
{
    if (!r) return JSIM_ERR_ARG;
    jsim_index* ix = r->idx;
    if (ix) {
        std::unique_lock<std::mutex> lk(ix->mu);
        auto ready = [&] { return r->state == kReqDone; };
        if (timeout_ms < 0) ix->cv_done.wait(lk, ready);
        else if (!ix->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return JSIM_ERR_TIMEOUT;
    }
    if (r->state != kReqDone) return JSIM_ERR_CANCELLED;
    if (r->status != JSIM_OK) return r->status;
    if (C && !r->C.empty()) memcpy(C, r->C.data(), r->C.size());
    if (J && !r->J.empty()) memcpy(J, r->J.data(), r->J.size() * sizeof(double));
    if (qsizes && !r->sizes.empty()) memcpy(qsizes, r->sizes.data(), r->sizes.size() * sizeof(u64));
    return JSIM_OK;
}

int jsim_request_latency(const jsim_request* r, double* queued_ms, double* total_ms)
{
    if (!r) return JSIM_ERR_ARG;
    if (r->state != kReqDone) return JSIM_ERR_TIMEOUT;
    if (queued_ms) *queued_ms = r->t_start - r->t_submit;
    if (total_ms) *total_ms = r->t_done - r->t_submit;
    return JSIM_OK;
}

void jsim_request_free(jsim_request* r)
{
    if (!r) return;
    jsim_index* ix = r->idx;
    if (ix) {
        std::unique_lock<std::mutex> lk(ix->mu);
        if (r->state == kReqQueued) {
            for (auto it = ix->queue.begin(); it != ix->queue.end(); ++it)
                if (*it == r) { ix->queue.erase(it); break; }
        } else {
            ix->cv_done.wait(lk, [&] { return r->state == kReqDone; });
        }
        ix->live.erase(r);
    }
    delete r;
}

}  // extern "C"
