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
#include <memory>
#include "common.cuh"

using namespace jsim;

#include "ctx.cuh"
#include "feed.cuh"
#include "sparse.cuh"

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
    opt->filter_min = 1;
    opt->distance = 0;
    opt->count_useful = 0;
    opt->tile_n = 0;
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
    if (o.filter_min != 1 && o.filter_min != 2) return JSIM_ERR_ARG;
    if (o.distance != 0 && o.distance != 1) return JSIM_ERR_ARG;
    if (o.count_useful != 0 && o.count_useful != 1) return JSIM_ERR_ARG;
    if (o.tile_n != 0 && o.tile_n != 128 && o.tile_n != 256) return JSIM_ERR_ARG;
    if ((o.alloc == nullptr) != (o.free == nullptr)) return JSIM_ERR_ARG;
    const bool own_pool = !o.alloc;
    jsim_ctx* c = new jsim_ctx();
    memset(&c->stats, 0, sizeof c->stats);
    c->cuda_err[0] = 0;
    cudaError_t e = cudaSetDevice(o.device);
    if (e == cudaSuccess && own_pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = o.device;
        e = cudaMemPoolCreate(&c->pool, &props);
        if (e == cudaSuccess) {
            unsigned long long keep = ~0ull;  // keep freed memory for the context's later calls
            e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        o.alloc = default_alloc;
        o.free = default_free;
        o.alloc_user = c->pool;
    }
    c->opt = o;
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
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_scalars, 256 * sizeof(u64));
    bool oom = false;
    if (e == cudaSuccess) {
        c->d_err = (unsigned int*)o.alloc(256, (void*)c->stream, o.alloc_user);
        if (!c->d_err) { e = cudaErrorMemoryAllocation; oom = true; }
        else e = cudaMemsetAsync(c->d_err, 0, 256, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c->d_err) o.free(c->d_err, 256, (void*)c->stream, o.alloc_user);
        if (c->h_scalars) cudaFreeHost(c->h_scalars);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        if (c->pool) cudaMemPoolDestroy(c->pool);
        delete c;
        return oom ? JSIM_ERR_OOM : JSIM_ERR_CUDA;
    }
    *out = c;
    return JSIM_OK;
}

void jsim_destroy(jsim_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->opt.device);
    cudaStreamSynchronize(ctx->stream);
    jsim_batched_release(ctx);
    jsim_streamed_release(ctx);
    for (cudaStream_t s : ctx->lanes) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    if (ctx->class_stream) { cudaStreamSynchronize(ctx->class_stream); cudaStreamDestroy(ctx->class_stream); }
    for (cudaEvent_t e : ctx->lane_join) cudaEventDestroy(e);
    if (ctx->lane_fork) cudaEventDestroy(ctx->lane_fork);
    if (ctx->d_err) ctx->opt.free(ctx->d_err, 256, (void*)ctx->stream, ctx->opt.alloc_user);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->h_scalars) cudaFreeHost(ctx->h_scalars);
    if (ctx->h_sketch) cudaFreeHost(ctx->h_sketch);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);  // released once nothing from it is outstanding
    delete ctx;
}

// Host input above kHostStreamMin bytes of values goes through the streamed
// call (super-batches of kHostStreamBytes, copies overlapping the device's
// work) instead of one copy before the batch loop.  Measured on 1024 clade
// samples (10.5 GB of pinned host values): one copy then the batch loop 256
// ms per call; streamed through 256 MiB / 512 MiB / 1 GiB / 2 GiB staging
// 276 / 238 / 228 / 261 ms; the device-resident call 207 ms.  For 2048
// samples of 1.6 GB the streamed call was slower (260 against 189 ms with a
// fresh context: the pinned staging is allocated on first use).
constexpr u64 kHostStreamBytes = 1ull << 30;
constexpr u64 kHostStreamMin = 4ull << 30;

namespace {

// Whether host input above kHostStreamMin should rather be brought to the
// device whole for the block-sparse path (asked for, or AUTO in its range of
// sample counts) than streamed through the dense path: the values, the
// block-sparse path's class matrices (sparse_matrix_budget) and 4 GiB for
// its other buffers must fit in the free device memory.  The block-sparse
// call is three times faster on the device than the dense one for clade
// collections, more than bringing the input over costs (1024 samples,
// 10.5 GB: 71 ms end to end; the streamed dense call 216 ms).
bool sparse_may_apply(jsim_ctx* ctx, const jsim_sets* sets)
{
    const int v = ctx->opt.variant;
    const u64 n = sets->n;
    if (v != JSIM_VARIANT_SPARSE &&
        !(v == JSIM_VARIANT_AUTO && n >= 256 && n <= 2048 && !ctx->opt.count_useful &&
          (ctx->opt.batch_rows == 0 || ctx->opt.batch_rows % (1ull << 18) == 0)))
        return false;
    if (cudaSetDevice(ctx->opt.device) != cudaSuccess || !product_tc_supported(ctx->opt.device)) {
        cudaGetLastError();
        return false;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const u64 bytes = (sets->offsets[n] - sets->offsets[0]) * sizeof(u64);
    return bytes + sparse_matrix_budget(total_b) + (4ull << 30) < (u64)free_b;
}

// Does the plain call copy its host input piece by piece under the
// block-sparse batch loop (feed.cuh)?  For page-locked input of at least
// kFeedMinBytes that the device can read (hv: its device-mapped address);
// minid and maxid from every sample's first and last value
// (JSIM_ERR_UNSORTED later if the input is not sorted after all).
bool feed_applies(jsim_ctx* ctx, const jsim_sets* sets, const std::vector<u64>& hoff, u64& minid, u64& maxid,
                  const u64*& hv)
{
    (void)ctx;
    const u64 n = sets->n, N = hoff[n];
    if (sets->mem != JSIM_MEM_HOST || N * sizeof(u64) < kFeedMinBytes) return false;
    cudaPointerAttributes pa{};
    const bool mapped = cudaPointerGetAttributes(&pa, sets->ids) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
                        pa.devicePointer != nullptr;
    cudaGetLastError();
    if (!mapped) return false;
    hv = (const u64*)pa.devicePointer;
    minid = ~0ull;
    maxid = 0;
    for (u64 i = 0; i < n; ++i)
        if (hoff[i + 1] > hoff[i]) {
            minid = std::min<u64>(minid, sets->ids[hoff[i]]);
            maxid = std::max<u64>(maxid, sets->ids[hoff[i + 1] - 1]);
        }
    return minid <= maxid;
}

// Row batches of part `part` of `parts` (the split contraction of
// jsim_all_pairs_part): the batch size mt (batch_rows, or the automatic size
// for the value span [minid, maxid]), and the batches [b_beg, b_end) (batch b
// = values [b mt, (b+1) mt)) of this part: the nb batches between the first
// and the last value cut into `parts` contiguous runs.
void partition_rows(u64 minid, u64 maxid, u64 batch_rows, u64 part, u64 parts, u64& b_beg, u64& b_end, u64& mt)
{
    const u64 span = maxid - minid;
    mt = batch_rows ? batch_rows : auto_batch_rows(span + 1 ? span + 1 : ~0ull);
    const u64 b_first = minid / mt, nb = maxid / mt - b_first + 1;
    b_beg = b_first + (u64)((unsigned __int128)nb * part / parts);
    b_end = b_first + (u64)((unsigned __int128)nb * (part + 1) / parts);
}

}  // namespace

// The plain call over the row batches [b_first + nb * part / parts,
// b_first + nb * (part + 1) / parts) of the nb batches between the first and
// the last value (parts = 1: all of them).  counts_only: C gets the part's
// counts (both triangles, the diagonal from the part's rows only) and J is
// not formed.
int all_pairs_impl(jsim_ctx* ctx, const jsim_sets* sets, void* C, uint64_t* sizes, double* J, int out_mem,
                   u64 part, u64 parts, bool counts_only, bool own_scope)
{
    int rc = 0;
    CK(cudaSetDevice(ctx->opt.device));
    // a call of its own resets and resolves the statistics; one collection
    // of a batched call adds to the batched call's
    std::unique_ptr<CallScope> scope;
    std::unique_ptr<StageTimer> total;
    if (own_scope) {
        scope.reset(new CallScope(ctx));
        total.reset(new StageTimer(ctx, &ctx->stats.ms_total));
    }
    const u64 n = sets->n;
    if (n == 0) return JSIM_OK;
    if (n > (1ull << 20)) return JSIM_ERR_ARG;  // n*n outputs must stay addressable
    std::vector<u64> hoff;
    rc = load_offsets(ctx, sets, hoff);
    if (rc) return rc;

    // the block-sparse path: asked for, or (AUTO) where a sketch shows that
    // ordering the samples empties enough tensor-core blocks
    const int want = ctx->opt.variant;
    const bool sparse = want == JSIM_VARIANT_SPARSE ||
                        (want == JSIM_VARIANT_AUTO && parts == 1 && !counts_only && n >= 256 && n <= 2048 &&
                         !ctx->opt.count_useful && product_tc_supported(ctx->opt.device) &&
                         (ctx->opt.batch_rows == 0 || ctx->opt.batch_rows % (1ull << 18) == 0));
    if (sparse && (parts != 1 || counts_only || ctx->opt.count_useful)) return JSIM_ERR_UNSUPPORTED;

    Staged st;
    std::unique_ptr<InputFeed> feed;  // after st: its copies end before st's buffers are released
    std::unique_ptr<SideValidation> sv;
    u64 feed_mt = 0, fminid = 0, fmaxid = 0;
    const u64* hv = nullptr;
    if (sparse && feed_applies(ctx, sets, hoff, fminid, fmaxid, hv) &&
        (feed_mt = sparse_batch_rows(ctx, n, fmaxid - fminid)) != 0 && fmaxid / feed_mt - fminid / feed_mt >= 3) {
        // page-locked host input: copied piece by piece under the batch loop
        rc = stage_input(ctx, sets, st, hoff, false);
        if (rc) return rc;
        st.minid = fminid;
        st.maxid = fmaxid;
        feed.reset(new InputFeed());
        rc = feed->start(ctx, st, hv, feed_mt, fminid, fmaxid);
        if (rc) return rc;
    } else if (sparse) {
        // the input is validated beside the sketch and the batch loop
        rc = stage_input(ctx, sets, st, hoff, true);
        if (rc) return rc;
        rc = first_last_values(ctx, st);
        if (rc) return rc;
        sv.reset(new SideValidation());  // started once the sketch is enqueued
    } else {
        rc = stage_and_validate(ctx, sets, st, hoff);
        if (rc) return rc;
    }
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(u32), ctx->stream));

    if (sparse) {
        bool declined = false;
        rc = all_pairs_sparse(ctx, st, C, sizes, J, out_mem, want == JSIM_VARIANT_AUTO, declined, feed.get(),
                              sv.get());
        if (rc || !declined) return rc;
        // the dense path reads the whole input: all of it in and valid
        rc = feed ? feed->finish(st) : sv->finish(ctx, st);
        if (rc) return rc;
    }
    const size_t cb = ctx->opt.count_bits == 64 ? 8 : 4;
    DevBuf Cacc, useful;
    ALLOC(Cacc, n * n * cb);
    CK(cudaMemsetAsync(Cacc.p, 0, n * n * cb, ctx->stream));
    if (ctx->opt.count_useful) {
        ALLOC(useful, sizeof(u64));
        CK(cudaMemsetAsync(useful.p, 0, sizeof(u64), ctx->stream));
    }

    // values lie in [minid, maxid]; batches are aligned to multiples of m~ and
    // empty stretches of the value range are skipped
    u64 mt = 0, b_beg = 0, b_end = 0;
    partition_rows(st.N ? st.minid : 0, st.N ? st.maxid : 0, ctx->opt.batch_rows, part, parts, b_beg, b_end, mt);
    ctx->stats.batch_rows = mt;
    int variant = ctx->opt.variant;
    if (st.N && b_beg < b_end) {
        BatchBufs bb;
        u64 lo = b_beg * mt;
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
                if (ctx->opt.count_useful)
                    CK(launch_useful(bb.X.as<u64>(), n, stride, W, useful.as<u64>(), ctx->sms, ctx->stream));
                ctx->stats.batches += 1;
                ctx->stats.rows_nonzero += R;
                ctx->stats.words += W;
                ctx->stats.bitops_dense += 64.0 * (double)W * (double)n * (double)(n + 1) / 2.0;
                ctx->stats.bitops_done += 64.0 * (double)W * (double)n * (double)(n + 1) / 2.0;
            }
            if (!has_next || next / mt >= b_end) break;
            lo = next / mt * mt;
        }
    }

    // nothing is written when a bounded device wait ran out
    rc = check_device_waits(ctx, ctx->d_err);
    if (rc) return rc;
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
        if (counts_only) Jdst = nullptr;
        if (Cdst || Jdst) {
            CK(launch_epilogue(Cacc.p, n, ctx->opt.count_bits, st.sizes.as<u64>(), Cdst, Jdst, ctx->stream,
                               !counts_only && ctx->opt.filter_min == 2, ctx->opt.distance));
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
    CK(cudaMemcpyAsync(ctx->h_scalars, ctx->d_err, sizeof(u32), cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->opt.count_useful)
        CK(cudaMemcpyAsync(ctx->h_scalars + 1, useful.p, sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->opt.count_useful) ctx->stats.bitops_useful = 64.0 * (double)ctx->h_scalars[1];
    if ((u32)ctx->h_scalars[0] != 0) return JSIM_ERR_TIMEOUT;
    return JSIM_OK;
}


int jsim_all_pairs(jsim_ctx* ctx, const jsim_sets* sets, void* C, uint64_t* sizes, double* J, int out_mem)
{
    if (!ctx) return JSIM_ERR_ARG;
    int rc = check_sets(sets);
    if (rc) return rc;
    if (out_mem != JSIM_MEM_HOST && out_mem != JSIM_MEM_DEVICE) return JSIM_ERR_ARG;
    if (sets->mem == JSIM_MEM_HOST && sets->n > 0 && sets->offsets[sets->n] >= sets->offsets[0] &&
        (sets->offsets[sets->n] - sets->offsets[0]) * sizeof(u64) > kHostStreamMin &&
        !sparse_may_apply(ctx, sets))
        return jsim_all_pairs_streamed(ctx, sets, C, sizes, J, out_mem, kHostStreamBytes);
    return all_pairs_impl(ctx, sets, C, sizes, J, out_mem, 0, 1, false, true);
}

int jsim_all_pairs_part(jsim_ctx* ctx, const jsim_sets* sets, uint32_t part, uint32_t parts, void* C,
                        uint64_t* sizes, int out_mem)
{
    if (!ctx || !C) return JSIM_ERR_ARG;
    if (parts == 0 || part >= parts) return JSIM_ERR_ARG;
    int rc = check_sets(sets);
    if (rc) return rc;
    if (out_mem != JSIM_MEM_HOST && out_mem != JSIM_MEM_DEVICE) return JSIM_ERR_ARG;
    return all_pairs_impl(ctx, sets, C, sizes, nullptr, out_mem, part, parts, true, true);
}

int jsim_partition_batches(uint64_t minid, uint64_t maxid, uint64_t batch_rows, uint32_t part, uint32_t parts,
                           uint64_t* b_begin, uint64_t* b_end, uint64_t* batch_rows_used)
{
    if (parts == 0 || part >= parts || maxid < minid || (batch_rows && batch_rows % 64)) return JSIM_ERR_ARG;
    u64 b0 = 0, b1 = 0, mt = 0;
    partition_rows(minid, maxid, batch_rows, part, parts, b0, b1, mt);
    if (b_begin) *b_begin = b0;
    if (b_end) *b_end = b1;
    if (batch_rows_used) *batch_rows_used = mt;
    return JSIM_OK;
}

int jsim_finish(jsim_ctx* ctx, uint64_t n, const void* C, const uint64_t* sizes, void* Cout, double* J, int mem)
{
    if (!ctx || !C || !sizes) return JSIM_ERR_ARG;
    if (mem != JSIM_MEM_HOST && mem != JSIM_MEM_DEVICE) return JSIM_ERR_ARG;
    if (n > (1ull << 20)) return JSIM_ERR_ARG;
    if (n == 0 || (!Cout && !J)) return JSIM_OK;
    CK(cudaSetDevice(ctx->opt.device));
    CallScope scope(ctx);
    StageTimer total(ctx, &ctx->stats.ms_total);
    const size_t cb = ctx->opt.count_bits == 64 ? 8 : 4;
    cudaStream_t s = ctx->stream;
    DevBuf Cd, Sd, Co, Jd;
    const void* Cp = C;
    const u64* Sp = (const u64*)sizes;
    void* Cop = Cout;
    double* Jp = J;
    if (mem == JSIM_MEM_HOST) {
        ALLOC(Cd, n * n * cb);
        ALLOC(Sd, n * sizeof(u64));
        CK(cudaMemcpyAsync(Cd.p, C, n * n * cb, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(Sd.p, sizes, n * sizeof(u64), cudaMemcpyHostToDevice, s));
        Cp = Cd.p;
        Sp = Sd.as<u64>();
        if (Cout) { ALLOC(Co, n * n * cb); Cop = Co.p; }
        if (J) { ALLOC(Jd, n * n * sizeof(double)); Jp = Jd.as<double>(); }
    }
    {
        StageTimer t(ctx, &ctx->stats.ms_epilogue);
        // the diagonal is |X_i| (a part's own rows may miss some of it)
        CK(launch_epilogue(Cp, n, ctx->opt.count_bits, Sp, Cop, Jp, s, 1, ctx->opt.distance));
        ctx->stats.launches += 1;
    }
    if (mem == JSIM_MEM_HOST) {
        if (Cout) CK(cudaMemcpyAsync(Cout, Cop, n * n * cb, cudaMemcpyDeviceToHost, s));
        if (J) CK(cudaMemcpyAsync(J, Jp, n * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
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
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(u32), ctx->stream));
    DevBuf useful;
    if (W) {
        StageTimer t(ctx, &ctx->stats.ms_product);
        int rc = run_product(ctx, v, (const u64*)words, stride, n, W, Cacc.p);
        if (rc) return rc;
    }
    if (W && ctx->opt.count_useful) {
        ALLOC(useful, sizeof(u64));
        CK(cudaMemsetAsync(useful.p, 0, sizeof(u64), ctx->stream));
        CK(launch_useful((const u64*)words, n, stride, W, useful.as<u64>(), ctx->sms, ctx->stream));
        CK(cudaMemcpyAsync(ctx->h_scalars + 1, useful.p, sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->stats.bitops_useful = 64.0 * (double)ctx->h_scalars[1];
    }
    ctx->stats.words = W;
    ctx->stats.bitops_dense = 64.0 * (double)W * (double)n * (double)(n + 1) / 2.0;
    int rc = check_device_waits(ctx, ctx->d_err);
    if (rc) return rc;
    CK(launch_epilogue(Cacc.p, n, ctx->opt.count_bits, nullptr, C, nullptr, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return JSIM_OK;
}

int jsim_get_stats(const jsim_ctx* ctx, jsim_stats* out)
{
    if (!ctx || !out) return JSIM_ERR_ARG;
    *out = ctx->stats;
    if (out->bitops_done == 0) out->bitops_done = out->bitops_dense;  // the dense products do all of it
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
    case JSIM_ERR_INCOMPLETE: return "stopped early as asked; the checkpoint holds the progress";
    case JSIM_ERR_CHECKPOINT: return "checkpoint file unreadable, corrupt or from another call";
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
    CallScope scope(ctx);
    if (n == 0) return JSIM_OK;
    cudaError_t e;
    unsigned char* scratch = (unsigned char*)noalloc_scratch(ctx->opt.device, e);
    if (!scratch) return cuda_fail(ctx, e, "cudaGetSymbolAddress(scratch)");
    u32* err = (u32*)(scratch + kNoAllocCountBytes);
    CK(cudaMemsetAsync(scratch, 0, (size_t)(n * n) * cb, ctx->stream));
    CK(cudaMemsetAsync(err, 0, sizeof(u32), ctx->stream));
    const int v = variant == JSIM_VARIANT_AUTO ? choose_variant(ctx, n, W) : variant;
    if (W) {
        int rc = run_product(ctx, v, (const u64*)words, stride, n, W, scratch, err);
        if (rc) return rc;
    }
    ctx->stats.words = W;
    ctx->stats.bitops_dense = 64.0 * (double)W * (double)n * (double)(n + 1) / 2.0;
    int rc = check_device_waits(ctx, err);
    if (rc) return rc;
    CK(launch_epilogue(scratch, n, ctx->opt.count_bits, nullptr, C, nullptr, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return JSIM_OK;
}
