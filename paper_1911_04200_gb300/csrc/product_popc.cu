// Semiring product on CUDA cores: C += X X^T over (AND, popcount, +) (Eq. 7).
//
// X holds one packed row per sample (word w of row i = 64 consecutive
// nonzero rows of the indicator matrix restricted to sample i).  A CTA owns a
// 64 x 64 tile of C on or above the diagonal and a slice of the word range;
// 256 threads each keep a 4 x 4 register tile of 32-bit partial counts.
// Operand tiles of 64 rows x 32 words are double-buffered in shared memory
// with cp.async (8-byte copies, zero-fill past row n and word W), row stride
// 33 words so that the 16 rows a warp reads at one word index fall in
// distinct banks.  Partial counts are added into C with atomics, so slices
// of the word range may run in any order.
#include "common.cuh"

namespace jsim {

namespace {

constexpr int kT = 64;          // tile edge (samples)
constexpr int kK = 32;          // words per stage
constexpr int kLd = kK + 1;     // padded row stride in shared memory (words)
constexpr int kThreads = 256;
constexpr int kStageWords = kT * kLd;
constexpr size_t kSmemBytes = 2ull * 2 * kStageWords * sizeof(u64);

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    int sz = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" :: "r"(s), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" :: "n"(N)); }

__device__ __forceinline__ void tile_coords(u64 t, u64 T, u64& ti, u64& tj)
{
    // upper-triangle tile t -> (ti, tj), ti <= tj, row-major over ti
    u64 r = 0, rem = t;
    while (rem >= T - r) { rem -= T - r; ++r; }
    ti = r; tj = r + rem;
}

template <typename CT, bool W32>
__global__ void __launch_bounds__(kThreads, 2)
k_prod_popc(const u64* __restrict__ X, u64 stride, u64 n, u64 W, const u64* Wdev, u64 T, u32 ksplit,
            CT* __restrict__ C, u64 ldc)
{
    if (Wdev) W = min(W, *Wdev);  // the launch was sized for the bound W
    extern __shared__ u64 smem[];
    u64* As = smem;                    // [2][kT][kLd]
    u64* Bs = smem + 2 * kStageWords;  // [2][kT][kLd]

    u64 ti, tj;
    tile_coords(blockIdx.x, T, ti, tj);
    const u64 r0 = ti * kT, c0 = tj * kT;
    const u64 nst = (W + kK - 1) / kK;
    const u64 s_begin = nst * blockIdx.y / ksplit, s_end = nst * (blockIdx.y + 1) / ksplit;
    if (s_begin >= s_end) return;

    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;

    auto load_stage = [&](u64 s, int buf) {
        const u64 k0 = s * kK;
        #pragma unroll
        for (int e = 0; e < (kT * kK) / kThreads; ++e) {
            int idx = tid + e * kThreads;
            int row = idx / kK, k = idx % kK;
            u64 gk = k0 + k;
            u64 ga = r0 + row, gb = c0 + row;
            bool va = ga < n && gk < W, vb = gb < n && gk < W;
            const u64* pa = va ? X + ga * stride + gk : X;
            const u64* pb = vb ? X + gb * stride + gk : X;
            cp_async8(As + buf * kStageWords + row * kLd + k, pa, va);
            cp_async8(Bs + buf * kStageWords + row * kLd + k, pb, vb);
        }
        cp_async_commit();
    };

    u32 acc[4][4];
    #pragma unroll
    for (int r = 0; r < 4; ++r)
        #pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0;

    load_stage(s_begin, 0);
    for (u64 s = s_begin; s < s_end; ++s) {
        const int buf = (int)((s - s_begin) & 1);
        if (s + 1 < s_end) {
            load_stage(s + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const u64* a_s = As + buf * kStageWords;
        const u64* b_s = Bs + buf * kStageWords;
        #pragma unroll 8
        for (int k = 0; k < kK; ++k) {
            u64 a[4], b[4];
            #pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = a_s[(ty + 16 * r) * kLd + k];
            #pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = b_s[(tx + 16 * c) * kLd + k];
            #pragma unroll
            for (int r = 0; r < 4; ++r)
                #pragma unroll
                for (int c = 0; c < 4; ++c) {
                    u64 x = a[r] & b[c];
                    if (W32) acc[r][c] += __popc((u32)x) + __popc((u32)(x >> 32));
                    else acc[r][c] += (u32)__popcll(x);
                }
        }
        __syncthreads();
    }

    #pragma unroll
    for (int r = 0; r < 4; ++r) {
        u64 i = r0 + ty + 16 * r;
        if (i >= n) continue;
        #pragma unroll
        for (int c = 0; c < 4; ++c) {
            u64 j = c0 + tx + 16 * c;
            if (j >= n || acc[r][c] == 0) continue;
            atomicAdd(C + i * ldc + j, (CT)acc[r][c]);
        }
    }
}

template <typename CT, bool W32>
cudaError_t run(ProductArgs& a, cudaStream_t st)
{
    const u64 T = (a.n + kT - 1) / kT;
    const u64 tiles = T * (T + 1) / 2;
    const u64 nst = (a.W + kK - 1) / kK;
    if (tiles == 0 || nst == 0) return cudaSuccess;
    // enough CTAs for ~4 waves of 2 CTAs per SM, each slice >= 4 stages
    u64 want = (u64)a.sms * 8;
    u64 ks = (want + tiles - 1) / tiles;
    u64 maxks = (nst + 3) / 4;
    if (ks > maxks) ks = maxks;
    if (ks < 1) ks = 1;
    if (ks > 65535) ks = 65535;
    cudaError_t e = cudaFuncSetAttribute(k_prod_popc<CT, W32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    if (tiles > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)tiles, (unsigned)ks);
    k_prod_popc<CT, W32><<<grid, kThreads, kSmemBytes, st>>>(a.X, a.stride, a.n, a.W, a.Wdev, T, (u32)ks,
                                                             (CT*)a.C, a.ldc);
    a.launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t product_popc(ProductArgs& a, cudaStream_t st)
{
    if (a.count_bits == 64) {
        return a.word_bits == 32 ? run<u64, true>(a, st) : run<u64, false>(a, st);
    }
    return a.word_bits == 32 ? run<u32, true>(a, st) : run<u32, false>(a, st);
}

}  // namespace jsim
