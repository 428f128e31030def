// C-ABI of the jsim library: argument checks, memory, batch planning and the
// order of the kernel launches (Listing 1 of the paper: per row batch
// filter -> prefix sum -> bitmask -> partial scores -> accumulate; then the
// final similarity scores).
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <vector>
#include <algorithm>
#include <mutex>
#include "common.cuh"

using namespace jsim;

struct jsim_ctx {
    jsim_options opt;
    cudaStream_t stream;
    bool own_stream;
    int sms;
    int cc_major, cc_minor;
    jsim_stats stats;
    char cuda_err[256];
    // small pinned host scratch for device -> host scalars
    unsigned long long* h_scalars;
    // device error word of kernels with bounded waits
    unsigned int* d_err;
    // stage timing (profile = 1): events recorded on the stream, resolved at
    // the end of each call, so timing adds no host synchronisation
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    struct Pending { cudaEvent_t a, b; double* acc; };
    std::vector<Pending> pending;
};

namespace {

void* default_alloc(size_t bytes, void* stream, void*)
{
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, (cudaStream_t)stream) != cudaSuccess) {
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
    StageTimer(jsim_ctx* c, double* target) : ctx(c), acc(target)
    {
        if (ctx->opt.profile) {
            a = take_event(ctx);
            if (a) cudaEventRecord(a, ctx->stream);
        }
    }
    void stop()
    {
        if (a) {
            cudaEvent_t b = take_event(ctx);
            if (b) {
                cudaEventRecord(b, ctx->stream);
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

// Copy (if needed) and validate a collection: sorted segments, value range,
// distinct counts per sample.  On success st.sizes holds |X_i|.
int stage_and_validate(jsim_ctx* ctx, const jsim_sets* s, Staged& st, const std::vector<u64>& hoff)
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
            if (st.N)
                CK(cudaMemcpyAsync(st.ids_buf.p, s->ids, st.N * sizeof(u64), cudaMemcpyHostToDevice, ctx->stream));
            st.d_off = st.off_buf.as<u64>();
            st.d_ids = st.ids_buf.as<u64>();
        } else {
            st.d_off = (const u64*)s->offsets;
            st.d_ids = (const u64*)s->ids;
        }
    }
    ALLOC(st.sizes, std::max<u64>(st.n, 1) * sizeof(u64));
    ALLOC(st.plan_buf, (3 * st.n + 5) * sizeof(u64));
    st.plan = carve_plan(st.plan_buf, st.n);
    DevBuf flags;  // err (u32 in a u64), max value, min value
    ALLOC(flags, 3 * sizeof(u64));
    st.max_chunks = st.N / kChunk + st.n + 1;
    {
        StageTimer t(ctx, &ctx->stats.ms_validate);
        CK(cudaMemsetAsync(st.sizes.p, 0, st.n * sizeof(u64), ctx->stream));
        CK(cudaMemsetAsync(flags.p, 0, 2 * sizeof(u64), ctx->stream));
        CK(cudaMemsetAsync(flags.as<u64>() + 2, 0xff, sizeof(u64), ctx->stream));
        CK(launch_plan(st.d_off, st.d_ids, st.n, 0, 0, true, st.plan, ctx->stream));
        CK(launch_validate(st.d_off, st.d_ids, st.n, st.plan, st.max_chunks, ctx->opt.id_bits, st.sizes.as<u64>(),
                           flags.as<u32>(), flags.as<u64>() + 1, flags.as<u64>() + 2, ctx->sms, ctx->stream));
        ctx->stats.launches += 2;
    }
    std::vector<u64> hs(st.n);
    CK(cudaMemcpyAsync(ctx->h_scalars, flags.p, 3 * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
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

// Working buffers of the batch loop.
struct BatchBufs {
    DevBuf bitmap, dir, bsum, boff, R, X, plan_buf, bsizes;
    Plan plan{};
    u64 X_bytes = 0;
};

// Largest power-of-two batch whose filter bitmap and rank directory stay in
// L2 (64 MiB bitmap + 32 MiB directory at 2^29), or the whole value range
// when it is smaller.
u64 auto_batch_rows(u64 domain)
{
    const u64 cap = 1ull << 28;
    u64 m = 64;
    while (m < domain && m < cap) m <<= 1;
    return m;
}

// Variant choice (measured on GB300: for 1024 samples the CUDA-core
// AND+popcount kernel runs ~128 Tbit-ops/s, the legacy mma.sync e4m3/s8/b1
// kernels at or below that, the tcgen05 FP8 kernel ~700; for 64 samples the
// CUDA-core kernel wins, 0.33 ms against 0.88 ms per all-pairs call, because
// one 128 x 256 tensor tile is mostly idle).
int choose_variant(jsim_ctx* ctx, u64 n, u64 W)
{
    (void)W;
    if (n >= 256 && product_tc_supported(ctx->opt.device)) return JSIM_VARIANT_TC;
    return JSIM_VARIANT_POPC;
}

int run_product(jsim_ctx* ctx, int variant, const u64* X, u64 stride, u64 n, u64 W, void* C)
{
    ProductArgs a{};
    a.X = X; a.stride = stride; a.n = n; a.W = W; a.C = C; a.ldc = n;
    a.count_bits = ctx->opt.count_bits; a.word_bits = ctx->opt.word_bits; a.sms = ctx->sms;
    a.timeout_ms = ctx->opt.timeout_ms > 0 ? ctx->opt.timeout_ms : 2000;
    a.err = ctx->d_err;
    cudaError_t e = cudaSuccess;
    switch (variant) {
    case JSIM_VARIANT_TC:
        if (!product_tc_supported(ctx->opt.device)) return JSIM_ERR_UNSUPPORTED;
        e = product_tc(a, ctx->stream);
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

// One row batch [lo, lo+width): plan, filter, rank directory, zero + pack.
// On return bb.X holds n_pad rows of `stride` words and *R the nonzero rows.
int build_batch(jsim_ctx* ctx, const Staged& st, BatchBufs& bb, u64 lo, u64 width, u64& R, u64& stride,
                u64* batch_sizes, bool* has_next = nullptr, u64* next = nullptr)
{
    const u64 n = st.n;
    const u64 nwords = width / 64;
    const u64 nb = std::max<u64>((nwords + kScanBlockWords - 1) / kScanBlockWords, 1);
    ALLOC(bb.plan_buf, (3 * n + 5) * sizeof(u64));
    bb.plan = carve_plan(bb.plan_buf, n);
    ALLOC(bb.bitmap, nwords * sizeof(u64));
    ALLOC(bb.dir, nwords * sizeof(u32));
    ALLOC(bb.bsum, nb * sizeof(u64));
    ALLOC(bb.boff, nb * sizeof(u64));
    ALLOC(bb.R, sizeof(u64));
    const u64 hi = lo + width;  // 0 on wrap-around = unbounded
    {
        StageTimer t(ctx, &ctx->stats.ms_filter);
        CK(launch_plan(st.d_off, st.d_ids, n, lo, hi, false, bb.plan, ctx->stream));
        CK(cudaMemsetAsync(bb.bitmap.p, 0, nwords * sizeof(u64), ctx->stream));
        CK(launch_filter(st.d_ids, n, bb.plan, st.max_chunks, lo, width, bb.bitmap.as<u32>(), ctx->sms,
                         ctx->stream));
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
    CK(cudaStreamSynchronize(ctx->stream));
    R = ctx->h_scalars[0];
    if (next) *next = ctx->h_scalars[1];
    if (has_next) *has_next = ctx->h_scalars[2] != 0;
    const u64 W = (R + 63) / 64;
    stride = round_up(std::max<u64>(W, 1), kWordPad);
    const u64 n_pad = round_up(std::max<u64>(n, 1), kRowPad);
    const u64 need = n_pad * stride * sizeof(u64);
    ALLOC(bb.X, need);
    {
        StageTimer t(ctx, &ctx->stats.ms_pack);
        CK(launch_zero_rows(bb.X.as<u64>(), n_pad, stride, stride, ctx->sms, ctx->stream));
        if (batch_sizes) CK(cudaMemsetAsync(batch_sizes, 0, n * sizeof(u64), ctx->stream));
        CK(launch_pack(st.d_ids, n, bb.plan, st.max_chunks, lo, width, bb.bitmap.as<u64>(), bb.dir.as<u32>(),
                       bb.boff.as<u64>(), bb.X.as<u64>(), stride, batch_sizes, ctx->sms, ctx->stream));
        ctx->stats.launches += 2;
    }
    return JSIM_OK;
}

}  // namespace

extern "C" {

void jsim_default_options(jsim_options* opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof *opt);
    opt->batch_rows = 0;
    opt->word_bits = 64;
    opt->variant = JSIM_VARIANT_AUTO;
    opt->count_bits = 32;
    opt->id_bits = 64;
    opt->device = 0;
    opt->timeout_ms = 2000;
}

int jsim_create(jsim_ctx** out, const jsim_options* opt)
{
    if (!out) return JSIM_ERR_ARG;
    *out = nullptr;
    jsim_options o;
    if (opt) o = *opt; else jsim_default_options(&o);
    if (o.word_bits != 32 && o.word_bits != 64) return JSIM_ERR_ARG;
    if (o.count_bits != 32 && o.count_bits != 64) return JSIM_ERR_ARG;
    if (o.id_bits < 1 || o.id_bits > 64) return JSIM_ERR_ARG;
    if (o.variant < 0 || o.variant >= JSIM_VARIANT_COUNT) return JSIM_ERR_ARG;
    if (o.batch_rows % 64 != 0) return JSIM_ERR_ARG;
    if ((o.alloc == nullptr) != (o.free == nullptr)) return JSIM_ERR_ARG;
    if (!o.alloc) { o.alloc = default_alloc; o.free = default_free; }
    jsim_ctx* c = new jsim_ctx();
    memset(&c->stats, 0, sizeof c->stats);
    c->opt = o;
    c->cuda_err[0] = 0;
    cudaError_t e = cudaSetDevice(o.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, o.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->cc_major, cudaDevAttrComputeCapabilityMajor, o.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->cc_minor, cudaDevAttrComputeCapabilityMinor, o.device);
    if (e == cudaSuccess) {
        if (o.stream) {
            c->stream = (cudaStream_t)o.stream;
            c->own_stream = false;
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = true;
        }
    }
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_scalars, 64 * sizeof(u64));
    if (e == cudaSuccess) {
        c->d_err = (unsigned int*)o.alloc(256, (void*)c->stream, o.alloc_user);
        if (!c->d_err) e = cudaErrorMemoryAllocation;
        else e = cudaMemsetAsync(c->d_err, 0, 256, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return JSIM_ERR_CUDA;
    }
    *out = c;
    return JSIM_OK;
}

void jsim_destroy(jsim_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->opt.device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->d_err) ctx->opt.free(ctx->d_err, 256, (void*)ctx->stream, ctx->opt.alloc_user);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->h_scalars) cudaFreeHost(ctx->h_scalars);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int jsim_all_pairs(jsim_ctx* ctx, const jsim_sets* sets, void* C, uint64_t* sizes, double* J, int out_mem)
{
    if (!ctx) return JSIM_ERR_ARG;
    int rc = check_sets(sets);
    if (rc) return rc;
    if (out_mem != JSIM_MEM_HOST && out_mem != JSIM_MEM_DEVICE) return JSIM_ERR_ARG;
    CK(cudaSetDevice(ctx->opt.device));
    CallScope scope(ctx);
    StageTimer total(ctx, &ctx->stats.ms_total);
    const u64 n = sets->n;
    if (n == 0) return JSIM_OK;
    if (n > (1ull << 20)) return JSIM_ERR_ARG;  // n*n outputs must stay addressable
    std::vector<u64> hoff;
    rc = load_offsets(ctx, sets, hoff);
    if (rc) return rc;

    Staged st;
    rc = stage_and_validate(ctx, sets, st, hoff);
    if (rc) return rc;

    const size_t cb = ctx->opt.count_bits == 64 ? 8 : 4;
    DevBuf Cacc;
    ALLOC(Cacc, n * n * cb);
    CK(cudaMemsetAsync(Cacc.p, 0, n * n * cb, ctx->stream));

    // values lie in [minid, maxid]; batches are aligned to multiples of m~ and
    // empty stretches of the value range are skipped
    const u64 span = st.N ? st.maxid - st.minid : 0;
    u64 mt = ctx->opt.batch_rows ? ctx->opt.batch_rows : auto_batch_rows(span + 1 ? span + 1 : ~0ull);
    ctx->stats.batch_rows = mt;
    int variant = ctx->opt.variant;
    if (st.N) {
        BatchBufs bb;
        u64 lo = st.minid / mt * mt;
        for (;;) {
            u64 R = 0, stride = 0, next = 0;
            bool has_next = false;
            rc = build_batch(ctx, st, bb, lo, mt, R, stride, nullptr, &has_next, &next);
            if (rc) return rc;
            if (R) {
                const u64 W = (R + 63) / 64;
                int v = variant == JSIM_VARIANT_AUTO ? choose_variant(ctx, n, W) : variant;
                StageTimer t(ctx, &ctx->stats.ms_product);
                rc = run_product(ctx, v, bb.X.as<u64>(), stride, n, W, Cacc.p);
                if (rc) return rc;
                ctx->stats.batches += 1;
                ctx->stats.rows_nonzero += R;
                ctx->stats.words += W;
                ctx->stats.bitops_dense += 64.0 * (double)W * (double)n * (double)(n + 1) / 2.0;
            }
            if (!has_next) break;
            lo = next / mt * mt;
        }
    }

    // epilogue into the outputs (device) or staging buffers (host)
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
            CK(launch_epilogue(Cacc.p, n, ctx->opt.count_bits, st.sizes.as<u64>(), Cdst, Jdst, ctx->stream));
            ctx->stats.launches += 1;
        }
    }
    {
        StageTimer t(ctx, &ctx->stats.ms_d2h);
        cudaMemcpyKind k = out_mem == JSIM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        if (out_mem == JSIM_MEM_HOST) {
            if (C) CK(cudaMemcpyAsync(C, Cst.p, n * n * cb, k, ctx->stream));
            if (J) CK(cudaMemcpyAsync(J, Jst.p, n * n * sizeof(double), k, ctx->stream));
        }
        if (sizes) CK(cudaMemcpyAsync(sizes, st.sizes.p, n * sizeof(u64), k, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return JSIM_OK;
}

int jsim_pack(jsim_ctx* ctx, const jsim_sets* sets, uint64_t lo, uint64_t width, uint64_t* filter,
              uint64_t* words, uint64_t stride, uint64_t* R_out, uint64_t* sizes, int out_mem)
{
    if (!ctx) return JSIM_ERR_ARG;
    int rc = check_sets(sets);
    if (rc) return rc;
    if (out_mem != JSIM_MEM_HOST && out_mem != JSIM_MEM_DEVICE) return JSIM_ERR_ARG;
    if (width == 0 || width % 64) return JSIM_ERR_ARG;
    CK(cudaSetDevice(ctx->opt.device));
    CallScope scope(ctx);
    const u64 n = sets->n;
    std::vector<u64> hoff;
    rc = load_offsets(ctx, sets, hoff);
    if (rc) return rc;
    Staged st;
    rc = stage_and_validate(ctx, sets, st, hoff);
    if (rc) return rc;
    BatchBufs bb;
    DevBuf bs;
    if (sizes) ALLOC(bs, std::max<u64>(n, 1) * sizeof(u64));
    u64 R = 0, xs = 0;
    rc = build_batch(ctx, st, bb, lo, width, R, xs, sizes ? bs.as<u64>() : nullptr);
    if (rc) return rc;
    if (R_out) *R_out = R;
    const u64 W = (R + 63) / 64;
    if (words && stride < W) return JSIM_ERR_ARG;
    cudaMemcpyKind k = out_mem == JSIM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (filter) CK(cudaMemcpyAsync(filter, bb.bitmap.p, width / 8, k, ctx->stream));
    if (words && n) {
        if (out_mem == JSIM_MEM_DEVICE) CK(cudaMemsetAsync(words, 0, n * stride * sizeof(u64), ctx->stream));
        else memset(words, 0, n * stride * sizeof(u64));
        if (W) CK(cudaMemcpy2DAsync(words, stride * sizeof(u64), bb.X.p, xs * sizeof(u64), W * sizeof(u64), n, k,
                                    ctx->stream));
    }
    if (sizes && n) CK(cudaMemcpyAsync(sizes, bs.p, n * sizeof(u64), k, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return JSIM_OK;
}

int jsim_product(jsim_ctx* ctx, const uint64_t* words, uint64_t n, uint64_t W, uint64_t stride, void* C,
                 int variant)
{
    if (!ctx || !C) return JSIM_ERR_ARG;
    if (n && !words && W) return JSIM_ERR_ARG;
    if (stride < W) return JSIM_ERR_ARG;
    if (variant < 0 || variant >= JSIM_VARIANT_COUNT) return JSIM_ERR_ARG;
    if (n > (1ull << 20)) return JSIM_ERR_ARG;
    CK(cudaSetDevice(ctx->opt.device));
    CallScope scope(ctx);
    if (n == 0) return JSIM_OK;
    const size_t cb = ctx->opt.count_bits == 64 ? 8 : 4;
    DevBuf Cacc;
    ALLOC(Cacc, n * n * cb);
    CK(cudaMemsetAsync(Cacc.p, 0, n * n * cb, ctx->stream));
    int v = variant == JSIM_VARIANT_AUTO ? choose_variant(ctx, n, W) : variant;
    if (W) {
        StageTimer t(ctx, &ctx->stats.ms_product);
        int rc = run_product(ctx, v, (const u64*)words, stride, n, W, Cacc.p);
        if (rc) return rc;
    }
    ctx->stats.words = W;
    ctx->stats.bitops_dense = 64.0 * (double)W * (double)n * (double)(n + 1) / 2.0;
    CK(launch_epilogue(Cacc.p, n, ctx->opt.count_bits, nullptr, C, nullptr, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return JSIM_OK;
}

int jsim_get_stats(const jsim_ctx* ctx, jsim_stats* out)
{
    if (!ctx || !out) return JSIM_ERR_ARG;
    *out = ctx->stats;
    return JSIM_OK;
}

const char* jsim_strerror(int code)
{
    switch (code) {
    case JSIM_OK: return "ok";
    case JSIM_ERR_ARG: return "invalid argument";
    case JSIM_ERR_UNSORTED: return "a sample's values are not sorted ascending";
    case JSIM_ERR_OVERFLOW: return "a set size does not fit the count width";
    case JSIM_ERR_ID_RANGE: return "a value is outside [0, 2^id_bits)";
    case JSIM_ERR_OOM: return "device memory allocation failed";
    case JSIM_ERR_CUDA: return "CUDA runtime error";
    case JSIM_ERR_TIMEOUT: return "a bounded device wait timed out";
    case JSIM_ERR_CANCELLED: return "request cancelled";
    case JSIM_ERR_UNSUPPORTED: return "variant or mode not supported";
    default: return "unknown error";
    }
}

const char* jsim_last_cuda_error(const jsim_ctx* ctx)
{
    return ctx ? ctx->cuda_err : "";
}

const char* jsim_version(void)
{
    return "jsim 0.1";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free product.
//
// Some callers cannot let the library allocate device memory while a call
// runs: an application that sizes and owns every byte of the GPU up front,
// an allocation-free steady-state loop (a server that must not stall on
// cudaMalloc or fragment a pool mid-request), or a host that plugs its own
// allocator into everything else but cannot hand one to this library.  For
// them jsim_product_noalloc keeps its only scratch - the upper-triangle count
// accumulator and a device error word - in one fixed array of device memory
// that belongs to the library module itself.  Every GPU that loads the
// library holds that array until the process exits, and every call on a
// device uses the same array, so calls that overlap on the GPU race.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocCountBytes = 4u << 20;      // 4 MiB of counts: n <= 1024 (32-bit), 724 (64-bit)
constexpr size_t kNoAllocBytes = kNoAllocCountBytes + 256;  // + error word
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices];

// Device address of the scratch array on `device` (current), looked up once.
void* noalloc_scratch(int device, cudaError_t& err)
{
    err = cudaSuccess;
    if (device < 0 || device >= kMaxDevices) {
        err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess) return nullptr;
        g_noalloc_ptr[device] = p;
    }
    return g_noalloc_ptr[device];
}

}  // namespace

extern "C" int jsim_product_noalloc(jsim_ctx* ctx, const uint64_t* words, uint64_t n, uint64_t W,
                                    uint64_t stride, void* C, int variant)
{
    if (!ctx || !C) return JSIM_ERR_ARG;
    if (n && !words && W) return JSIM_ERR_ARG;
    if (stride < W) return JSIM_ERR_ARG;
    if (variant < 0 || variant >= JSIM_VARIANT_COUNT) return JSIM_ERR_ARG;
    const size_t cb = ctx->opt.count_bits == 64 ? 8 : 4;
    if (n > (1u << 16) || (size_t)(n * n) * cb > kNoAllocCountBytes) return JSIM_ERR_ARG;
    CK(cudaSetDevice(ctx->opt.device));
    if (n == 0) return JSIM_OK;
    cudaError_t e;
    unsigned char* scratch = (unsigned char*)noalloc_scratch(ctx->opt.device, e);
    if (!scratch) return cuda_fail(ctx, e, "cudaGetSymbolAddress(scratch)");
    u32* err = (u32*)(scratch + kNoAllocCountBytes);
    CK(cudaMemsetAsync(scratch, 0, (size_t)(n * n) * cb, ctx->stream));
    CK(cudaMemsetAsync(err, 0, sizeof(u32), ctx->stream));
    int v = variant == JSIM_VARIANT_AUTO ? choose_variant(ctx, n, W) : variant;
    if (W) {
        ProductArgs a{};
        a.X = (const u64*)words; a.stride = stride; a.n = n; a.W = W; a.C = scratch; a.ldc = n;
        a.count_bits = ctx->opt.count_bits; a.word_bits = ctx->opt.word_bits; a.sms = ctx->sms;
        a.timeout_ms = ctx->opt.timeout_ms > 0 ? ctx->opt.timeout_ms : 2000;
        a.err = err;
        switch (v) {
        case JSIM_VARIANT_TC:
            if (!product_tc_supported(ctx->opt.device)) return JSIM_ERR_UNSUPPORTED;
            e = product_tc(a, ctx->stream);
            break;
        case JSIM_VARIANT_POPC: e = product_popc(a, ctx->stream); break;
        case JSIM_VARIANT_B1:
        case JSIM_VARIANT_I8:
        case JSIM_VARIANT_F8: e = product_mma(a, v, ctx->stream); break;
        default: return JSIM_ERR_UNSUPPORTED;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "product");
    }
    CK(launch_epilogue(scratch, n, ctx->opt.count_bits, nullptr, C, nullptr, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_scalars, err, sizeof(u32), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if ((u32)ctx->h_scalars[0] != 0) return JSIM_ERR_TIMEOUT;
    return JSIM_OK;
}
