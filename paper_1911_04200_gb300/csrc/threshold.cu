// Threshold output from a similarity matrix: the pairs i < j whose J is at
// least tau (or, for a distance matrix, at most tau), in row-major order -
// the sparse form of the all-pairs result that large collections keep in
// place of n x n values.
//
// Three launches: a CTA per row counts its pairs, one CTA scans the counts
// into row offsets (and the total), a CTA per row writes its pairs at its
// offset with an order-preserving block compaction (ballot within warps,
// warp totals through shared memory), so the output order does not depend on
// scheduling.  Pairs past the caller's capacity are counted, not written.
#include <algorithm>
#include "ctx.cuh"
#include "ingest_dev.cuh"

namespace jsim {
namespace {

constexpr int kThThreads = 256;
constexpr int kThWarps = kThThreads / 32;

__device__ __forceinline__ bool keep(double v, double tau, int below)
{
    return below ? v <= tau : v >= tau;
}

__global__ void __launch_bounds__(kThThreads)
k_thr_count(const double* __restrict__ J, u64 n, double tau, int below, u64* __restrict__ cnt)
{
    __shared__ u64 red[kThWarps];
    for (u64 i = blockIdx.x; i < n; i += gridDim.x) {
        const double* row = J + i * n;
        u64 c = 0;
        for (u64 j = i + 1 + threadIdx.x; j < n; j += kThThreads) c += keep(row[j], tau, below);
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            u64 t = 0;
            for (int w = 0; w < kThWarps; ++w) t += red[w];
            cnt[i] = t;
        }
        __syncthreads();
    }
}

// off[i] = sum of cnt[0..i), off[n] = total (one CTA)
__global__ void __launch_bounds__(kPlanThreads) k_thr_scan(const u64* __restrict__ cnt, u64 n, u64* __restrict__ off)
{
    __shared__ u64 sm[kPlanThreads / 32];
    u64 carry = 0;
    for (u64 base = 0; base < n; base += kPlanThreads) {
        const u64 i = base + threadIdx.x;
        const u64 v = i < n ? cnt[i] : 0;
        u64 ex;
        const u64 tot = block_exclusive_scan<kPlanThreads>(v, ex, sm);
        if (i < n) off[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) off[n] = carry;
}

__global__ void __launch_bounds__(kThThreads)
k_thr_write(const double* __restrict__ J, u64 n, double tau, int below, const u64* __restrict__ off, u64 cap,
            u64* __restrict__ pi, u64* __restrict__ pj, double* __restrict__ val)
{
    __shared__ u32 wsum[kThWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (u64 i = blockIdx.x; i < n; i += gridDim.x) {
        u64 at = off[i];
        if (at >= cap) continue;  // uniform across the block
        const double* row = J + i * n;
        for (u64 j0 = i + 1; j0 < n && at < cap; j0 += kThThreads) {
            const u64 j = j0 + threadIdx.x;
            double v = 0.0;
            bool k = false;
            if (j < n) {
                v = row[j];
                k = keep(v, tau, below);
            }
            const unsigned m = __ballot_sync(0xffffffffu, k);
            if (lane == 0) wsum[warp] = (u32)__popc(m);
            __syncthreads();
            u64 before = 0, total = 0;
            #pragma unroll
            for (int w = 0; w < kThWarps; ++w) {
                const u64 c = wsum[w];
                before += w < warp ? c : 0;
                total += c;
            }
            const u64 pos = at + before + (u64)__popc(m & ((1u << lane) - 1u));
            if (k && pos < cap) {
                pi[pos] = i;
                pj[pos] = j;
                if (val) val[pos] = v;
            }
            at += total;
            __syncthreads();  // wsum is rewritten by the next step
        }
    }
}

}  // namespace
}  // namespace jsim

extern "C" int jsim_threshold(jsim_ctx* ctx, const double* J, uint64_t n, double tau, int below, uint64_t cap,
                              uint64_t* pi, uint64_t* pj, double* val, uint64_t* count, int mem)
{
    if (!ctx || !J || !count) return JSIM_ERR_ARG;
    if (mem != JSIM_MEM_HOST && mem != JSIM_MEM_DEVICE) return JSIM_ERR_ARG;
    if (below != 0 && below != 1) return JSIM_ERR_ARG;
    if (!(tau == tau)) return JSIM_ERR_ARG;  // NaN
    if (cap && (!pi || !pj)) return JSIM_ERR_ARG;
    if (n > 0xffffffffull) return JSIM_ERR_ARG;
    *count = 0;
    if (n < 2) return JSIM_OK;
    CK(cudaSetDevice(ctx->opt.device));
    CallScope scope(ctx);
    StageTimer total(ctx, &ctx->stats.ms_total);
    cudaStream_t st = ctx->stream;
    DevBuf Jd, cnt, off, pid, pjd, vd;
    const double* Jp = J;
    u64* ip = (u64*)pi;
    u64* jp = (u64*)pj;
    double* vp = val;
    if (mem == JSIM_MEM_HOST) {
        ALLOC(Jd, n * n * sizeof(double));
        CK(cudaMemcpyAsync(Jd.p, J, n * n * sizeof(double), cudaMemcpyHostToDevice, st));
        Jp = Jd.as<double>();
        if (cap) {
            ALLOC(pid, cap * sizeof(u64));
            ALLOC(pjd, cap * sizeof(u64));
            ip = pid.as<u64>();
            jp = pjd.as<u64>();
            if (val) {
                ALLOC(vd, cap * sizeof(double));
                vp = vd.as<double>();
            }
        }
    }
    ALLOC(cnt, n * sizeof(u64));
    ALLOC(off, (n + 1) * sizeof(u64));
    const unsigned grid = (unsigned)std::min<u64>(n, (u64)ctx->sms * 8);
    {
        StageTimer t(ctx, &ctx->stats.ms_epilogue);
        jsim::k_thr_count<<<grid, kThThreads, 0, st>>>(Jp, n, tau, below, cnt.as<u64>());
        CK(cudaGetLastError());
        jsim::k_thr_scan<<<1, kPlanThreads, 0, st>>>(cnt.as<u64>(), n, off.as<u64>());
        CK(cudaGetLastError());
        ctx->stats.launches += 2;
        if (cap) {
            jsim::k_thr_write<<<grid, kThThreads, 0, st>>>(Jp, n, tau, below, off.as<u64>(), cap, ip, jp, vp);
            CK(cudaGetLastError());
            ctx->stats.launches += 1;
        }
    }
    CK(cudaMemcpyAsync(ctx->h_scalars, off.as<u64>() + n, sizeof(u64), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const u64 found = ctx->h_scalars[0];
    *count = found;
    if (mem == JSIM_MEM_HOST && cap) {
        const u64 w = std::min<u64>(found, cap);
        if (w) {
            CK(cudaMemcpyAsync(pi, ip, w * sizeof(u64), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(pj, jp, w * sizeof(u64), cudaMemcpyDeviceToHost, st));
            if (val) CK(cudaMemcpyAsync(val, vp, w * sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
    }
    return JSIM_OK;
}
