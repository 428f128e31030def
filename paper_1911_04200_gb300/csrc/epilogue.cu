// Epilogue: mirror the upper-triangle counts into a full C and form
// J = C / (|X_i| + |X_j| - C) (Sec. III-A: union by inclusion-exclusion,
// Eq. 2: s_ij = b_ij / c_ij), with J = 1 for two empty sets (Sec. II-A);
// or, with `distance`, the Jaccard distance D = 1 - J (Sec. II-A) as the
// binary64 subtraction 1.0 - J (D = 0 for two empty sets).
//
// The quotient is one IEEE binary64 division, round-to-nearest (__ddiv_rn),
// of two integers below 2^53 converted exactly, so it is correctly rounded
// and bit-identical to any other correctly rounded evaluation.  32 x 32
// tiles are staged through shared memory so both the read of the mirrored
// half and the writes stay coalesced.
#include <algorithm>
#include "common.cuh"

namespace jsim {

namespace {

constexpr int kE = 32;

template <typename CT>
__global__ void __launch_bounds__(kE * 8)
k_epilogue(const CT* __restrict__ Cacc, u64 n, const u64* __restrict__ sizes,
           CT* __restrict__ Cout, double* __restrict__ J, int diag_sizes, int distance, const u32* skip_if)
{
    // a raised error word (a bounded wait of the product ran out): write nothing
    if (skip_if && *(volatile const u32*)skip_if) return;
    __shared__ CT tile[kE][kE + 1];
    const u64 bi = blockIdx.y, bj = blockIdx.x;
    const u64 i0 = bi * kE, j0 = bj * kE;
    const bool lower = bi > bj;
    // source tile: (i0, j0) itself if on/above diagonal, else the transposed
    // tile (j0, i0) of the upper triangle
    const u64 si0 = lower ? j0 : i0, sj0 = lower ? i0 : j0;
    for (int r = threadIdx.y; r < kE; r += 8) {
        u64 si = si0 + r, sj = sj0 + threadIdx.x;
        CT v = 0;
        if (si < n && sj < n) v = Cacc[si * n + sj];
        tile[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < kE; r += 8) {
        u64 i = i0 + r, j = j0 + threadIdx.x;
        if (i >= n || j >= n) continue;
        // element (i, j): on/above the diagonal tile it is tile[r][x];
        // below it is the transposed element; inside a diagonal tile the
        // lower half mirrors the upper half
        CT c;
        if (lower) c = tile[threadIdx.x][r];
        else if (bi == bj && i > j) c = tile[threadIdx.x][r];
        else c = tile[r][threadIdx.x];
        if (diag_sizes && i == j) c = (CT)sizes[i];
        if (Cout) Cout[i * n + j] = c;
        if (J) {
            const u64 u = sizes[i] + sizes[j] - (u64)c;
            const double s = u ? __ddiv_rn(__ull2double_rn((u64)c), __ull2double_rn(u)) : 1.0;
            J[i * n + j] = distance ? __dsub_rn(1.0, s) : s;
        }
    }
}

// Useful work of a packed batch: for every word column w, nnz_w = rows whose
// word w is nonzero; adds sum_w nnz_w (nnz_w + 1) / 2 (the pairs i <= j of
// nonzero words) to *acc.  Consecutive threads take consecutive columns, so
// every row read is coalesced.
__global__ void k_useful(const u64* __restrict__ X, u64 n, u64 stride, u64 W, unsigned long long* acc)
{
    u64 local = 0;
    for (u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x; w < W; w += (u64)gridDim.x * blockDim.x) {
        u64 c = 0;
        for (u64 i = 0; i < n; ++i) c += X[i * stride + w] != 0ull;
        local += c * (c + 1) / 2;
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(acc, (unsigned long long)local);
}

}  // namespace

cudaError_t launch_useful(const u64* X, u64 n, u64 stride, u64 W, u64* acc, int sms, cudaStream_t st)
{
    if (W == 0 || n == 0) return cudaSuccess;
    const u64 blocks = std::min<u64>((W + 255) / 256, (u64)sms * 8);
    k_useful<<<(unsigned)blocks, 256, 0, st>>>(X, n, stride, W, (unsigned long long*)acc);
    return cudaGetLastError();
}

cudaError_t launch_epilogue(const void* Cacc, u64 n, int count_bits, const u64* sizes,
                            void* Cout, double* J, cudaStream_t st, int diag_sizes, int distance, const u32* skip_if)
{
    if (n == 0) return cudaSuccess;
    u64 nb = (n + kE - 1) / kE;
    if (nb > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)nb, (unsigned)nb), block(kE, 8);
    if (count_bits == 64)
        k_epilogue<u64><<<grid, block, 0, st>>>((const u64*)Cacc, n, sizes, (u64*)Cout, J, diag_sizes, distance,
                                                 skip_if);
    else
        k_epilogue<u32><<<grid, block, 0, st>>>((const u32*)Cacc, n, sizes, (u32*)Cout, J, diag_sizes, distance,
                                                 skip_if);
    return cudaGetLastError();
}

}  // namespace jsim
