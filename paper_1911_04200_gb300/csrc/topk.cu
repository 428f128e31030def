// Nearest neighbours from a similarity matrix: for every sample the k others
// with the largest J (the sparsified output that large collections need in
// place of an n x n matrix).  Ties in J go to the smaller index, so the
// result is unique.
//
// A CTA per row.  Candidates are ordered by (bits of J descending, index
// ascending) - non-negative doubles order like their bit patterns, and the
// index makes every candidate distinct.  Pass t takes the best candidate
// strictly after the pick of pass t-1 with a block-wide reduction, so k
// passes give the k best without marking anything; the row is staged in
// shared memory when it fits.
#include <algorithm>
#include "ctx.cuh"

namespace {

constexpr int kTkThreads = 256;
constexpr u64 kTkSmemRows = 16384;  // rows up to this length are staged in shared memory

__global__ void __launch_bounds__(kTkThreads)
k_topk(const double* __restrict__ J, u64 n, u32 k, u64* __restrict__ idx, double* __restrict__ val)
{
    extern __shared__ double row_s[];
    __shared__ u64 red_b[kTkThreads / 32];
    __shared__ u64 red_j[kTkThreads / 32];
    const u64 i = blockIdx.x;
    const double* row = J + i * n;
    const bool staged = n <= kTkSmemRows;
    if (staged)
        for (u64 j = threadIdx.x; j < n; j += kTkThreads) row_s[j] = row[j];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // previous pick (bits of J, index): the next pick is the best strictly after it
    u64 pb = ~0ull, pj = 0;
    bool first = true;
    for (u32 t = 0; t < k; ++t) {
        u64 bb = 0, bj = ~0ull;
        bool have = false;
        for (u64 j = threadIdx.x; j < n; j += kTkThreads) {
            if (j == i) continue;
            const u64 b = (u64)__double_as_longlong(staged ? row_s[j] : row[j]);
            // strictly after (pb, pj) in (bits desc, index asc)
            const bool after = first || b < pb || (b == pb && j > pj);
            if (!after) continue;
            // better than the current best (bb, bj)?
            if (!have || b > bb || (b == bb && j < bj)) { bb = b; bj = j; have = true; }
        }
        if (!have) { bb = 0; bj = ~0ull; }
        // block-wide best: larger bits, then smaller index; "none" is (0, ~0)
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const u64 ob = __shfl_xor_sync(0xffffffffu, bb, o), oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ob > bb || (ob == bb && oj < bj)) { bb = ob; bj = oj; }
        }
        if (lane == 0) { red_b[warp] = bb; red_j[warp] = bj; }
        __syncthreads();
        if (warp == 0) {
            bb = lane < kTkThreads / 32 ? red_b[lane] : 0ull;
            bj = lane < kTkThreads / 32 ? red_j[lane] : ~0ull;
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const u64 ob = __shfl_xor_sync(0xffffffffu, bb, o), oj = __shfl_xor_sync(0xffffffffu, bj, o);
                if (ob > bb || (ob == bb && oj < bj)) { bb = ob; bj = oj; }
            }
            if (lane == 0) { red_b[0] = bb; red_j[0] = bj; }
        }
        __syncthreads();
        pb = red_b[0];
        pj = red_j[0];
        first = false;
        if (threadIdx.x == 0) {
            idx[i * k + t] = pj;
            if (val) val[i * k + t] = __longlong_as_double((long long)pb);
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" int jsim_topk(jsim_ctx* ctx, const double* J, uint64_t n, uint32_t k, uint64_t* idx, double* val, int mem)
{
    if (!ctx || !J || !idx) return JSIM_ERR_ARG;
    if (mem != JSIM_MEM_HOST && mem != JSIM_MEM_DEVICE) return JSIM_ERR_ARG;
    if (k == 0 || k > 64 || n < 2 || k > n - 1 || n > 0xffffffffull) return JSIM_ERR_ARG;
    CK(cudaSetDevice(ctx->opt.device));
    CallScope scope(ctx);
    StageTimer total(ctx, &ctx->stats.ms_total);
    cudaStream_t st = ctx->stream;
    DevBuf Jd, id, vd;
    const double* Jp = J;
    u64* ip = (u64*)idx;
    double* vp = val;
    if (mem == JSIM_MEM_HOST) {
        ALLOC(Jd, n * n * sizeof(double));
        CK(cudaMemcpyAsync(Jd.p, J, n * n * sizeof(double), cudaMemcpyHostToDevice, st));
        Jp = Jd.as<double>();
        ALLOC(id, n * k * sizeof(u64));
        ip = id.as<u64>();
        if (val) {
            ALLOC(vd, n * k * sizeof(double));
            vp = vd.as<double>();
        }
    }
    const size_t smem = n <= kTkSmemRows ? n * sizeof(double) : 0;
    CK(cudaFuncSetAttribute(k_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kTkSmemRows * 8)));
    {
        StageTimer t(ctx, &ctx->stats.ms_epilogue);
        k_topk<<<(unsigned)n, kTkThreads, smem, st>>>(Jp, n, k, ip, vp);
        CK(cudaGetLastError());
        ctx->stats.launches += 1;
    }
    if (mem == JSIM_MEM_HOST) {
        CK(cudaMemcpyAsync(idx, ip, n * k * sizeof(u64), cudaMemcpyDeviceToHost, st));
        if (val) CK(cudaMemcpyAsync(val, vp, n * k * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    return JSIM_OK;
}
