// Internal: the context object and host-side helpers shared by the C-ABI
// translation units (not installed).
#pragma once
#include <cstdio>
#include <cstring>
#include <vector>
#include <algorithm>
#include "common.cuh"

using namespace jsim;

struct jsim_ctx;
// The plain all-pairs call (api.cu).  own_scope = false when it runs as one
// collection of a batched call, whose statistics it then adds to.
// (C linkage, as the C-ABI translation unit defines it; not exported)
extern "C" int all_pairs_impl(jsim_ctx* ctx, const jsim_sets* sets, void* C, uint64_t* sizes, double* J,
                              int out_mem, u64 part, u64 parts, bool counts_only, bool own_scope);
// releases the batched-call state (captured graphs and buffers) of a context
void jsim_batched_release(jsim_ctx* ctx);
// releases the streamed-call state (pinned staging, copy stream) of a context
void jsim_streamed_release(jsim_ctx* ctx);
struct StreamState;

struct jsim_ctx {
    jsim_options opt;
    cudaStream_t stream;
    bool own_stream;
    int sms;
    int cc_major, cc_minor;
    jsim_stats stats;
    char cuda_err[256];
    // small pinned host scratch (256 u64) for device <-> host scalars
    unsigned long long* h_scalars;
    // page-locked scratch for the block-sparse path's sketch similarities (grown on demand)
    void* h_sketch = nullptr;
    size_t h_sketch_bytes = 0;
    // the block-sparse path's classification stream, at the device's highest priority (created on demand)
    cudaStream_t class_stream = nullptr;
    // device error word of kernels with bounded waits
    unsigned int* d_err;
    // the context's own stream-ordered memory pool (default allocator only)
    cudaMemPool_t pool = nullptr;
    // stage timing (profile = 1): events recorded on the stream, resolved at
    // the end of each call, so timing adds no host synchronisation
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    struct Pending { cudaEvent_t a, b; double* acc; };
    std::vector<Pending> pending;
    // streamed calls: pinned staging buffers kept between calls
    StreamState* streamed = nullptr;
    // side streams for independent per-collection work (batched calls), with
    // a fork event on the context's stream and one join event per lane
    std::vector<cudaStream_t> lanes;
    cudaEvent_t lane_fork = nullptr;
    std::vector<cudaEvent_t> lane_join;
};

namespace {

// The default allocator: stream-ordered allocations from the context's own
// memory pool (user = the pool).  The pool keeps freed memory for reuse
// instead of returning it at every synchronisation (as the device's default
// pool does), so the buffers a call frees and the next call allocates again
// cost no new mappings: on 1024 clade samples streamed from host memory the
// call took 229 ms per call from the default pool, 216 ms from a keeping pool.
void* default_alloc(size_t bytes, void* stream, void* user)
{
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, (cudaMemPool_t)user, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void default_free(void* p, size_t, void* stream, void*)
{
    if (p) cudaFreeAsync(p, (cudaStream_t)stream);
}

struct Status {
    int code = JSIM_OK;
};

// A device allocation freed (in stream order) when it leaves scope.
struct DevBuf {
    jsim_ctx* ctx = nullptr;
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (p && ctx) ctx->opt.free(p, bytes, (void*)ctx->stream, ctx->opt.alloc_user);
        p = nullptr;
        bytes = 0;
    }
    // (re)allocate at least `b` bytes; contents undefined
    bool ensure(jsim_ctx* c, size_t b)
    {
        if (p && bytes >= b) return true;
        release();
        ctx = c;
        size_t bb = b ? b : 16;
        p = c->opt.alloc(bb, (void*)c->stream, c->opt.alloc_user);
        if (!p) return false;
        bytes = bb;
        return true;
    }
    template <typename T> T* as() const { return (T*)p; }
};

int cuda_fail(jsim_ctx* ctx, cudaError_t e, const char* what)
{
    snprintf(ctx->cuda_err, sizeof ctx->cuda_err, "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return JSIM_ERR_CUDA;
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

#define ALLOC(buf, bytes)                                          \
    do {                                                           \
        if (!(buf).ensure(ctx, (bytes))) return JSIM_ERR_OOM;      \
    } while (0)

// Optional per-stage CUDA-event timing.
cudaEvent_t take_event(jsim_ctx* ctx)
{
    if (ctx->events_used == ctx->events.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        ctx->events.push_back(e);
    }
    return ctx->events[ctx->events_used++];
}

struct StageTimer {
    jsim_ctx* ctx;
    cudaEvent_t a = nullptr;
    double* acc;
    cudaStream_t s;  // the stream the stage runs on (the context's by default)
    StageTimer(jsim_ctx* c, double* target, cudaStream_t on = nullptr) : ctx(c), acc(target), s(on ? on : c->stream)
    {
        if (ctx->opt.profile) {
            a = take_event(ctx);
            if (a) cudaEventRecord(a, s);
        }
    }
    void stop()
    {
        if (a) {
            cudaEvent_t b = take_event(ctx);
            if (b) {
                cudaEventRecord(b, s);
                ctx->pending.push_back({a, b, acc});
            }
            a = nullptr;
        }
    }
    ~StageTimer() { stop(); }
};

// Resolves the stage timers of one API call when it returns.
struct CallScope {
    jsim_ctx* ctx;
    explicit CallScope(jsim_ctx* c) : ctx(c)
    {
        memset(&ctx->stats, 0, sizeof ctx->stats);
        ctx->events_used = 0;
        ctx->pending.clear();
    }
    ~CallScope()
    {
        for (auto& p : ctx->pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
                *p.acc += ms;
            else
                cudaGetLastError();
        }
        ctx->pending.clear();
        ctx->events_used = 0;
    }
};

u64 round_up(u64 x, u64 m) { return (x + m - 1) / m * m; }

// Waits for the context's stream and reads the device error word `err` (a
// bounded device wait ran out when it is nonzero), so that a call can return
// JSIM_ERR_TIMEOUT before it writes any output.
int check_device_waits(jsim_ctx* ctx, const u32* err)
{
    cudaError_t e = cudaMemcpyAsync(ctx->h_scalars, err, sizeof(u32), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error word");
    return (u32)ctx->h_scalars[0] != 0 ? JSIM_ERR_TIMEOUT : JSIM_OK;
}

// Side streams: work on lane l is ordered after everything queued on the
// context's stream before lanes_fork, and everything queued on it after
// lanes_join waits for all lanes.  Under stream capture the lanes become
// parallel branches of the graph.
int lanes_ensure(jsim_ctx* ctx, int k)
{
    if (!ctx->lane_fork) CK(cudaEventCreateWithFlags(&ctx->lane_fork, cudaEventDisableTiming));
    while ((int)ctx->lanes.size() < k) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        ctx->lanes.push_back(s);
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->lane_join.push_back(e);
    }
    return JSIM_OK;
}

int lanes_fork(jsim_ctx* ctx, int k)
{
    CK(cudaEventRecord(ctx->lane_fork, ctx->stream));
    for (int l = 0; l < k; ++l) CK(cudaStreamWaitEvent(ctx->lanes[l], ctx->lane_fork, 0));
    return JSIM_OK;
}

int lanes_join(jsim_ctx* ctx, int k)
{
    for (int l = 0; l < k; ++l) {
        CK(cudaEventRecord(ctx->lane_join[l], ctx->lanes[l]));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->lane_join[l], 0));
    }
    return JSIM_OK;
}

int check_sets(const jsim_sets* s)
{
    if (!s) return JSIM_ERR_ARG;
    if (s->mem != JSIM_MEM_HOST && s->mem != JSIM_MEM_DEVICE) return JSIM_ERR_ARG;
    if (!s->offsets) return JSIM_ERR_ARG;
    return JSIM_OK;
}

// Host copy of offsets, checked: offsets[0] == 0 and non-decreasing.
int load_offsets(jsim_ctx* ctx, const jsim_sets* s, std::vector<u64>& h)
{
    h.resize(s->n + 1);
    if (s->mem == JSIM_MEM_HOST) {
        memcpy(h.data(), s->offsets, (s->n + 1) * sizeof(u64));
    } else {
        CK(cudaMemcpyAsync(h.data(), s->offsets, (s->n + 1) * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (h[0] != 0) return JSIM_ERR_ARG;
    for (u64 i = 0; i < s->n; ++i)
        if (h[i + 1] < h[i]) return JSIM_ERR_ARG;
    if (h[s->n] > 0 && !s->ids) return JSIM_ERR_ARG;
    return JSIM_OK;
}

// Device-resident inputs of one collection plus the results of validation.
struct Staged {
    const u64* d_off = nullptr;
    const u64* d_ids = nullptr;
    DevBuf off_buf, ids_buf;
    DevBuf sizes;     // [n] distinct counts
    DevBuf plan_buf;  // beg, len, cofs, totals
    DevBuf flags;     // validation: error word, max value, min value
    Plan plan{};
    u64 n = 0, N = 0, maxid = 0, minid = 0, max_size = 0, max_chunks = 0;
};

Plan carve_plan(DevBuf& b, u64 n)
{
    Plan p;
    u64* base = b.as<u64>();
    p.beg = base;
    p.len = base + n;
    p.cofs = base + 2 * n;
    p.totals = base + 3 * n + 1;
    return p;
}

// Device buffers of a collection: offsets and values (copied from host
// memory, the values only when copy_ids), sizes, a plan and the validation
// flags.
int stage_input(jsim_ctx* ctx, const jsim_sets* s, Staged& st, const std::vector<u64>& hoff, bool copy_ids)
{
    st.n = s->n;
    st.N = hoff[s->n];
    {
        StageTimer t(ctx, &ctx->stats.ms_h2d);
        if (s->mem == JSIM_MEM_HOST) {
            ALLOC(st.off_buf, (st.n + 1) * sizeof(u64));
            ALLOC(st.ids_buf, std::max<u64>(st.N, 1) * sizeof(u64));
            CK(cudaMemcpyAsync(st.off_buf.p, hoff.data(), (st.n + 1) * sizeof(u64), cudaMemcpyHostToDevice,
                               ctx->stream));
            ctx->stats.h2d_copies += 1;
            ctx->stats.h2d_bytes += (st.n + 1) * sizeof(u64);
            if (st.N && copy_ids) {
                CK(cudaMemcpyAsync(st.ids_buf.p, s->ids, st.N * sizeof(u64), cudaMemcpyHostToDevice, ctx->stream));
                ctx->stats.h2d_copies += 1;
                ctx->stats.h2d_bytes += st.N * sizeof(u64);
            }
            st.d_off = st.off_buf.as<u64>();
            st.d_ids = st.ids_buf.as<u64>();
        } else {
            st.d_off = (const u64*)s->offsets;
            st.d_ids = (const u64*)s->ids;
        }
    }
    ALLOC(st.sizes, std::max<u64>(st.n, 1) * sizeof(u64));
    ALLOC(st.plan_buf, plan_words(st.n) * sizeof(u64));
    ALLOC(st.flags, 3 * sizeof(u64));  // err (u32 in a u64), max value, min value
    st.plan = carve_plan(st.plan_buf, st.n);
    st.max_chunks = st.N / kChunk + st.n + 1;
    return JSIM_OK;
}

// Validation of the staged values on stream `vs`: sorted segments, value
// range, distinct counts per sample (into st.sizes), min and max value.
// First the validation's sizes and flags cleared (on vs).
int validate_init(jsim_ctx* ctx, Staged& st, cudaStream_t vs)
{
    CK(cudaMemsetAsync(st.sizes.p, 0, st.n * sizeof(u64), vs));
    CK(cudaMemsetAsync(st.flags.p, 0, 2 * sizeof(u64), vs));
    CK(cudaMemsetAsync(st.flags.as<u64>() + 2, 0xff, sizeof(u64), vs));
    return JSIM_OK;
}

// Validation of the values [begs[i], ends[i]) of every sample i (on vs;
// ends null: to the sample's end), adding to the sizes and flags; slices of
// several calls that tile every sample validate it as one call would (a
// value is compared with the one before it in its sample, wherever that is).
int validate_slices(jsim_ctx* ctx, Staged& st, cudaStream_t vs, const u64* begs, const u64* ends)
{
    CK(launch_plan(begs, st.d_ids, st.n, 0, 0, true, st.plan, vs, nullptr, ends));
    CK(launch_validate(st.d_off, st.d_ids, st.n, st.plan, st.max_chunks, ctx->opt.id_bits, st.sizes.as<u64>(),
                       st.flags.as<u32>(), st.flags.as<u64>() + 1, st.flags.as<u64>() + 2, ctx->sms, vs));
    ctx->stats.launches += 2;
    return JSIM_OK;
}

int validate_staged(jsim_ctx* ctx, Staged& st, cudaStream_t vs)
{
    int rc = validate_init(ctx, st, vs);
    if (rc) return rc;
    return validate_slices(ctx, st, vs, st.d_off, nullptr);
}

// The validation's verdict (after the context's stream has waited for it):
// JSIM_ERR_UNSORTED, JSIM_ERR_ID_RANGE, JSIM_ERR_OVERFLOW (a size that 32-bit
// counts cannot hold), or st.minid, st.maxid and st.max_size.
int check_staged(jsim_ctx* ctx, Staged& st)
{
    std::vector<u64> hs(st.n);
    CK(cudaMemcpyAsync(ctx->h_scalars, st.flags.p, 3 * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hs.data(), st.sizes.p, st.n * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    u32 f = (u32)ctx->h_scalars[0];
    if (f & kFlagUnsorted) return JSIM_ERR_UNSORTED;
    if (f & kFlagIdRange) return JSIM_ERR_ID_RANGE;
    st.maxid = ctx->h_scalars[1];
    st.minid = ctx->h_scalars[2];
    st.max_size = 0;
    for (u64 v : hs) st.max_size = std::max(st.max_size, v);
    if (ctx->opt.count_bits == 32 && st.max_size > 0xffffffffull) return JSIM_ERR_OVERFLOW;
    return JSIM_OK;
}

// Validation of a staged collection on a side stream, beside the work that
// follows it on the context's stream: started after `after` (an event on
// another stream) or after what the context's stream has enqueued so far;
// finish() makes the context's stream wait for it and returns its verdict
// (check_staged).  Until then the work on the context's stream may read
// unvalidated values and must stay memory-safe on any input.
struct SideValidation {
    jsim_ctx* ctx = nullptr;
    cudaStream_t vs = nullptr;
    cudaEvent_t ready = nullptr, validated = nullptr;
    bool started = false;
    SideValidation() = default;
    SideValidation(const SideValidation&) = delete;
    SideValidation& operator=(const SideValidation&) = delete;
    ~SideValidation()
    {
        if (vs) { cudaStreamSynchronize(vs); cudaStreamDestroy(vs); }
        if (ready) cudaEventDestroy(ready);
        if (validated) cudaEventDestroy(validated);
        cudaGetLastError();
    }
    // the side stream, ordered after what the context's stream has enqueued so far
    int open(jsim_ctx* c)
    {
        ctx = c;
        CK(cudaStreamCreateWithFlags(&vs, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&validated, cudaEventDisableTiming));
        CK(cudaEventRecord(ready, ctx->stream));
        CK(cudaStreamWaitEvent(vs, ready, 0));
        return JSIM_OK;
    }
    // what the side stream holds so far is the validation
    int close()
    {
        CK(cudaEventRecord(validated, vs));
        started = true;
        return JSIM_OK;
    }
    int start(jsim_ctx* c, Staged& st, cudaEvent_t after = nullptr)
    {
        int rc = open(c);
        if (rc) return rc;
        if (after) CK(cudaStreamWaitEvent(vs, after, 0));
        rc = validate_staged(ctx, st, vs);
        if (rc) return rc;
        return close();
    }
    int finish(jsim_ctx* c, Staged& st)
    {
        if (!started) {
            int rc = start(c, st);
            if (rc) return rc;
        }
        CK(cudaStreamWaitEvent(ctx->stream, validated, 0));
        return check_staged(ctx, st);
    }
};

// The smallest first and largest last value of the staged samples (their
// minimum and maximum when sorted) into st.minid and st.maxid; none: {~0, 0}.
int first_last_values(jsim_ctx* ctx, Staged& st)
{
    DevBuf fl;
    ALLOC(fl, 2 * sizeof(u64));
    CK(cudaMemsetAsync(fl.p, 0xff, sizeof(u64), ctx->stream));
    CK(cudaMemsetAsync(fl.as<u64>() + 1, 0, sizeof(u64), ctx->stream));
    CK(launch_first_last(st.d_off, st.d_ids, st.n, fl.as<u64>(), ctx->stream));
    ctx->stats.launches += 1;
    CK(cudaMemcpyAsync(ctx->h_scalars, fl.p, 2 * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    st.minid = ctx->h_scalars[0];
    st.maxid = ctx->h_scalars[1];
    return JSIM_OK;
}

// Copy (if needed) and validate a collection.  On success st.sizes holds
// |X_i|.
int stage_and_validate(jsim_ctx* ctx, const jsim_sets* s, Staged& st, const std::vector<u64>& hoff)
{
    int rc = stage_input(ctx, s, st, hoff, true);
    if (rc) return rc;
    {
        StageTimer t(ctx, &ctx->stats.ms_validate);
        rc = validate_staged(ctx, st, ctx->stream);
        if (rc) return rc;
    }
    return check_staged(ctx, st);
}

// Largest power-of-two batch up to 2^28 rows (its 32 MiB filter bitmap and
// 16 MiB rank directory stay in L2), or the whole value range when it is
// smaller.  A sweep of the batch size on 1024 clade samples of 1.3e9 values
// (2^22 .. 2^32 rows) has its minimum at 2^28 with either filter: smaller
// batches multiply the product launches, larger ones move the filter, scan
// and pack out of L2.
u64 auto_batch_rows(u64 domain)
{
    const u64 cap = 1ull << 28;
    u64 m = 64;
    while (m < domain && m < cap) m <<= 1;
    return m;
}

// Variant choice, from a sweep on GB300 (random packed words, Tbit-ops/s):
//   n      64    128   192   256   512   1024  2048
//   POPC   71    92    104   111   123   130   142
//   TC     32    124   193   333   491   654   831
//   TC2    24    95    211   377   601   848   1069
// (the legacy mma.sync kernels stay at or below POPC).  Tensor tiles of 128
// or 256 samples are mostly idle for small n.
int choose_variant(jsim_ctx* ctx, u64 n, u64 W)
{
    (void)W;
    if (n <= 96 || !product_tc_supported(ctx->opt.device)) return JSIM_VARIANT_POPC;
    return n <= 160 ? JSIM_VARIANT_TC : JSIM_VARIANT_TC2;
}

// The semiring product C += X X^T with the chosen variant; err is the device
// error word the kernels raise (the context's when null).
int run_product(jsim_ctx* ctx, int variant, const u64* X, u64 stride, u64 n, u64 W, void* C, u32* err = nullptr)
{
    ProductArgs a{};
    a.X = X; a.stride = stride; a.n = n; a.W = W; a.C = C; a.ldc = n;
    a.count_bits = ctx->opt.count_bits; a.word_bits = ctx->opt.word_bits; a.sms = ctx->sms;
    a.timeout_ms = ctx->opt.timeout_ms > 0 ? ctx->opt.timeout_ms : 2000;
    a.err = err ? err : ctx->d_err;
    cudaError_t e = cudaSuccess;
    switch (variant) {
    case JSIM_VARIANT_TC:
        if (!product_tc_supported(ctx->opt.device)) return JSIM_ERR_UNSUPPORTED;
        e = product_tc(a, ctx->stream);
        break;
    case JSIM_VARIANT_TC2:
        if (!product_tc_supported(ctx->opt.device)) return JSIM_ERR_UNSUPPORTED;
        e = product_tc_pair(a, ctx->stream);
        break;
    case JSIM_VARIANT_POPC: e = product_popc(a, ctx->stream); break;
    case JSIM_VARIANT_B1:
    case JSIM_VARIANT_I8:
    case JSIM_VARIANT_F8: e = product_mma(a, variant, ctx->stream); break;
    default: return JSIM_ERR_UNSUPPORTED;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "product");
    ctx->stats.product_launches += a.launches;
    ctx->stats.launches += a.launches;
    ctx->stats.variant = variant;
    return JSIM_OK;
}

// first position in [lo, hi) of a sorted array with value >= v
u64 lower_bound_host(const uint64_t* a, u64 lo, u64 hi, u64 v)
{
    while (lo < hi) {
        u64 mid = lo + (hi - lo) / 2;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The same search started at lo, galloping (steps 1, 2, 4, ...) before
// bisecting: the cut a value boundary makes in a sample lies shortly after
// the previous boundary's cut, so this touches a few cache lines near it
// instead of bisecting the whole sample.  Like any bisection it leaves q with
// a[q-1] < v (or q = lo) and a[q] >= v (or q = hi), probed.
u64 gallop_host(const uint64_t* a, u64 lo, u64 hi, u64 v)
{
    u64 step = 1, base = lo;
    while (base + step <= hi && base + step - 1 < hi && a[base + step - 1] < v) {
        base += step;
        step *= 2;
    }
    return lower_bound_host(a, base, std::min(hi, base + step - 1), v);
}

// Working buffers of the batch loop.
struct BatchBufs {
    DevBuf bitmap, seen, dir, bsum, boff, R, X, plan_buf, bsizes;  // bitmap: the rows kept
    Plan plan{};
    u64 X_bytes = 0;
};

// One row batch [lo, lo+width): plan, filter, rank directory, zero + pack.
// On return bb.X holds n_pad rows of `stride` words and *R the nonzero rows.
// With beg_bound/end_bound, sample i's values are searched only in
// [beg_bound[i], end_bound[i]) (the slice of it already on the device).
int build_batch(jsim_ctx* ctx, const Staged& st, BatchBufs& bb, u64 lo, u64 width, u64& R, u64& stride,
                u64* batch_sizes, bool* has_next = nullptr, u64* next = nullptr, const u64* beg_bound = nullptr,
                const u64* end_bound = nullptr)
{
    const u64 n = st.n;
    const u64 nwords = width / 64;
    const u64 nb = std::max<u64>((nwords + kScanBlockWords - 1) / kScanBlockWords, 1);
    ALLOC(bb.plan_buf, plan_words(n) * sizeof(u64));
    bb.plan = carve_plan(bb.plan_buf, n);
    ALLOC(bb.bitmap, nwords * sizeof(u64));
    ALLOC(bb.dir, nwords * sizeof(u32));
    ALLOC(bb.bsum, nb * sizeof(u64));
    ALLOC(bb.boff, nb * sizeof(u64));
    ALLOC(bb.R, sizeof(u64));
    const u64 hi = lo + width;  // 0 on wrap-around = unbounded
    {
        StageTimer t(ctx, &ctx->stats.ms_filter);
        CK(launch_plan(beg_bound ? beg_bound : st.d_off, st.d_ids, n, lo, hi, false, bb.plan, ctx->stream, nullptr,
                       end_bound));
        CK(cudaMemsetAsync(bb.bitmap.p, 0, nwords * sizeof(u64), ctx->stream));
        if (ctx->opt.filter_min == 2) {
            // f of every row (seen) and the kept rows of two or more samples
            ALLOC(bb.seen, nwords * sizeof(u64));
            CK(cudaMemsetAsync(bb.seen.p, 0, nwords * sizeof(u64), ctx->stream));
            CK(launch_filter(st.d_ids, n, bb.plan, st.max_chunks, lo, width, bb.seen.as<u32>(), ctx->sms,
                             ctx->stream, bb.bitmap.as<u32>()));
        } else {
            CK(launch_filter(st.d_ids, n, bb.plan, st.max_chunks, lo, width, bb.bitmap.as<u32>(), ctx->sms,
                             ctx->stream));
        }
        ctx->stats.launches += 2;
    }
    {
        StageTimer t(ctx, &ctx->stats.ms_scan);
        CK(launch_scan(bb.bitmap.as<u64>(), nwords, bb.dir.as<u32>(), bb.bsum.as<u64>(), bb.boff.as<u64>(),
                       bb.R.as<u64>(), ctx->stream));
        ctx->stats.launches += 2;
    }
    CK(cudaMemcpyAsync(ctx->h_scalars, bb.R.p, sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_scalars + 1, bb.plan.totals + 2, 2 * sizeof(u64), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_scalars + 3, bb.plan.totals, sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    R = ctx->h_scalars[0];
    if (next) *next = ctx->h_scalars[1];
    if (has_next) *has_next = ctx->h_scalars[2] != 0;
    const u64 W = (R + 63) / 64;
    stride = row_stride_words(W);
    const u64 n_pad = round_up(std::max<u64>(n, 1), kRowPad);
    ctx->stats.pack_bytes += 8 * ctx->h_scalars[3] + 8 * n_pad * W;
    const u64 need = n_pad * stride * sizeof(u64);
    ALLOC(bb.X, need);
    {
        StageTimer t(ctx, &ctx->stats.ms_pack);
        if (batch_sizes) {
            // the step-level entry point: zero-filled rows (the caller sees the
            // padding words too) and per-sample counts of the batch
            CK(launch_zero_rows(bb.X.as<u64>(), n_pad, stride, stride, ctx->sms, ctx->stream));
            CK(cudaMemsetAsync(batch_sizes, 0, n * sizeof(u64), ctx->stream));
            CK(launch_pack(st.d_ids, n, bb.plan, st.max_chunks, lo, width, bb.bitmap.as<u64>(), bb.dir.as<u32>(),
                           bb.boff.as<u64>(), bb.X.as<u64>(), stride, batch_sizes, ctx->sms, ctx->stream));
        } else {
            CK(launch_zero_rows(bb.X.as<u64>(), n_pad, stride, stride, ctx->sms, ctx->stream));
            CK(launch_pack_full(st.d_ids, n, bb.plan, st.max_chunks, lo, width, bb.bitmap.as<u64>(),
                                bb.dir.as<u32>(), bb.boff.as<u64>(), bb.X.as<u64>(), stride, bb.R.as<u64>(), ctx->sms,
                                ctx->stream));
        }
        ctx->stats.launches += 2;
    }
    return JSIM_OK;
}


}  // namespace
