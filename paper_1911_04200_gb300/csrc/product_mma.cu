// Semiring product on the legacy warp-level tensor-core path (mma.sync),
// C += X X^T over (AND, popcount, +) (Eq. 7), three exact variants:
//
//   B1  mma.m16n8k256 .b1 with .and.popc: the packed words are the operands
//       as they are; s32 accumulators.
//   I8  mma.m16n8k32 .s8: every bit becomes a byte 0 or 1; s32 accumulators.
//   F8  mma.m16n8k32 .e4m3: every bit becomes 0.0 or 1.0 (0x00 / 0x38);
//       f32 accumulators.  All partial sums are integers below 2^24, which
//       binary32 holds exactly, and a CTA's slice of the word range is capped
//       so that no accumulator can reach 2^24.
//
// A CTA owns a 128 x 128 tile of C on or above the diagonal and a slice of
// the word range; 4 warps (2 x 2) each hold a 64 x 64 register tile.  One
// stage covers 256 bit-rows (I8, F8: unpacked to 256 bytes per sample row) or
// 2048 bit-rows (B1: 256 packed bytes per row).  Shared memory holds the
// stage as two 128-byte-wide column blocks per operand, each 16-byte chunk at
// position chunk ^ (row % 8), so the 8 rows one ldmatrix phase reads fall in
// distinct banks.  The next stage's packed words are prefetched into
// registers while the tensor cores work on the current one.
#include "common.cuh"

namespace jsim {

namespace {

constexpr int kBM = 128;                      // tile edge (samples)
constexpr int kThreads = 128;                 // 4 warps
constexpr int kRowBytes = 256;                // bytes of one row per stage
constexpr int kOpBytes = kBM * kRowBytes;     // 32 KiB per operand per stage
constexpr int kSmem = 2 * kOpBytes;           // A and B
constexpr int kStageBytes = 2 * 2 * 128 * 4 * 8;  // packed staging of the unpacked variants
constexpr u64 kMaxSliceBits = 1ull << 22;     // per-CTA K cap (f32 exactness margin)

__device__ __forceinline__ u32 smem_addr(const void* p) { return (u32)__cvta_generic_to_shared(p); }

// byte offset of 16-byte chunk c (0..15) of row r inside one operand stage
__device__ __forceinline__ u32 swz(int r, int c)
{
    return (u32)((c >> 3) * (kBM * 128) + r * 128 + (((c & 7) ^ (r & 7)) << 4));
}

__device__ __forceinline__ void ldsm_x4(u32 addr, u32& d0, u32& d1, u32& d2, u32& d3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3) : "r"(addr));
}

template <int V> struct Mma;

template <> struct Mma<JSIM_VARIANT_F8> {
    typedef float acc_t;
    static constexpr int kBitsPerStage = 256;
    static constexpr u32 kOne = 0x38u;  // e4m3 1.0
    static __device__ __forceinline__ void run(acc_t* d, const u32* a, const u32* b)
    {
        asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};\n"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
};
template <> struct Mma<JSIM_VARIANT_I8> {
    typedef int acc_t;
    static constexpr int kBitsPerStage = 256;
    static constexpr u32 kOne = 0x01u;
    static __device__ __forceinline__ void run(acc_t* d, const u32* a, const u32* b)
    {
        asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};\n"
                     : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
};
template <> struct Mma<JSIM_VARIANT_B1> {
    typedef int acc_t;
    static constexpr int kBitsPerStage = 2048;
    static constexpr u32 kOne = 0u;
    static __device__ __forceinline__ void run(acc_t* d, const u32* a, const u32* b)
    {
        asm volatile("mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                     "{%8,%9}, {%0,%1,%2,%3};\n"
                     : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
};

// 4 bits -> 4 bytes, each 0 or `one` (bit i -> byte i)
__device__ __forceinline__ u32 expand4(u32 nib, u32 one)
{
    return ((nib * 0x00204081u) & 0x01010101u) * one;
}

template <int V, typename CT>
__global__ void __launch_bounds__(kThreads, 2)
k_prod_mma(const u64* __restrict__ X, u64 stride, u64 n, u64 W, u64 T, u32 ksplit, CT* __restrict__ C, u64 ldc)
{
    typedef Mma<V> M;
    typedef typename M::acc_t acc_t;
    constexpr int kStageWords = M::kBitsPerStage / 64;  // 4 (unpacked) or 32 (b1)
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + kOpBytes;

    // tile (ti, tj), ti <= tj
    u64 ti = 0, rem = blockIdx.x;
    while (rem >= T - ti) { rem -= T - ti; ++ti; }
    const u64 tj = ti + rem;
    const u64 r0 = ti * kBM, c0 = tj * kBM;
    const u64 nst = (W + kStageWords - 1) / kStageWords;
    const u64 s_begin = nst * blockIdx.y / ksplit, s_end = nst * (blockIdx.y + 1) / ksplit;
    if (s_begin >= s_end) return;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;

    acc_t acc[4][8][4];
    #pragma unroll
    for (int i = 0; i < 4; ++i)
        #pragma unroll
        for (int j = 0; j < 8; ++j)
            #pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0;

    // ---- stage loaders -------------------------------------------------------
    // unpacked variants: the packed stage (2 operands x 128 rows x 4 words)
    // goes to a double-buffered staging area with 8-byte cp.async, then every
    // bit is expanded into the swizzled byte tiles
    u64* stage_buf = (u64*)(smem + kSmem);  // [2][2][128][4]
    auto fetch = [&](u64 s) {
        const u64 k0 = s * kStageWords;
        u64* dst = stage_buf + (s & 1) * 1024;
        #pragma unroll
        for (int e = 0; e < 8; ++e) {
            int idx = tid + kThreads * e;
            int op = idx >> 9, r = (idx >> 2) & 127, w = idx & 3;
            u64 grow = (op ? c0 : r0) + r, gk = k0 + w;
            bool ok = grow < n && gk < W;
            const u64* g = ok ? X + grow * stride + gk : X;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n"
                         :: "r"(smem_addr(dst + idx)), "l"(g), "r"(ok ? 8 : 0));
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };
    auto unpack_store = [&](u64 s) {
        const u64* src = stage_buf + (s & 1) * 1024;
        #pragma unroll 2
        for (int e = 0; e < 8; ++e) {
            int idx = tid + kThreads * e;
            int op = idx >> 9, r = (idx >> 2) & 127, w = idx & 3;
            unsigned char* base = op ? sB : sA;
            u64 x = src[idx];
            #pragma unroll
            for (int q = 0; q < 4; ++q) {  // 16 bits -> one 16-byte chunk
                u32 h = (u32)(x >> (16 * q));
                uint4 v;
                v.x = expand4(h & 15u, M::kOne);
                v.y = expand4((h >> 4) & 15u, M::kOne);
                v.z = expand4((h >> 8) & 15u, M::kOne);
                v.w = expand4((h >> 12) & 15u, M::kOne);
                *(uint4*)(base + swz(r, w * 4 + q)) = v;
            }
        }
    };
    // b1: 2 operands x 128 rows x 32 words, 8-byte cp.async (any row stride), 64/thread
    auto copy_b1 = [&](u64 s) {
        const u64 k0 = s * kStageWords;
        #pragma unroll 8
        for (int e = 0; e < 64; ++e) {
            int idx = tid + kThreads * e;
            int op = idx >> 12, r = (idx >> 5) & 127, w = idx & 31;
            u64 grow = (op ? c0 : r0) + r, gk = k0 + w;
            bool ok = grow < n && gk < W;
            const u64* g = ok ? X + grow * stride + gk : X;
            u32 sa = smem_addr((op ? sB : sA) + swz(r, w >> 1) + 8 * (w & 1));
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" :: "r"(sa), "l"(g), "r"(ok ? 8 : 0));
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };

    if (V == JSIM_VARIANT_B1) copy_b1(s_begin); else fetch(s_begin);

    const u32 a_base = smem_addr(sA), b_base = smem_addr(sB);
    const int q = lane >> 3, r8 = lane & 7;

    for (u64 s = s_begin; s < s_end; ++s) {
        if (V == JSIM_VARIANT_B1) {
            asm volatile("cp.async.wait_group 0;\n" ::);
        } else {
            if (s + 1 < s_end) {
                fetch(s + 1);
                asm volatile("cp.async.wait_group 1;\n" ::);
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::);
            }
            __syncthreads();
            unpack_store(s);
        }
        __syncthreads();
        #pragma unroll 1
        for (int kk = 0; kk < 8; ++kk) {
            u32 a[4][4], b[8][2];
            #pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                int row = wm * 64 + mi * 16 + (q & 1) * 8 + r8;
                int ch = kk * 2 + (q >> 1);
                ldsm_x4(a_base + swz(row, ch), a[mi][0], a[mi][1], a[mi][2], a[mi][3]);
            }
            #pragma unroll
            for (int nj = 0; nj < 8; nj += 2) {
                int row = wn * 64 + (nj + (q >> 1)) * 8 + r8;
                int ch = kk * 2 + (q & 1);
                ldsm_x4(b_base + swz(row, ch), b[nj][0], b[nj][1], b[nj + 1][0], b[nj + 1][1]);
            }
            #pragma unroll
            for (int mi = 0; mi < 4; ++mi)
                #pragma unroll
                for (int nj = 0; nj < 8; ++nj) M::run(acc[mi][nj], a[mi], b[nj]);
        }
        __syncthreads();
        if (V == JSIM_VARIANT_B1 && s + 1 < s_end) copy_b1(s + 1);
    }

    // ---- accumulate the tile into C ------------------------------------------
    const int g = lane >> 2, t4 = lane & 3;
    #pragma unroll
    for (int mi = 0; mi < 4; ++mi)
        #pragma unroll
        for (int nj = 0; nj < 8; ++nj)
            #pragma unroll
            for (int e = 0; e < 4; ++e) {
                u64 i = r0 + wm * 64 + mi * 16 + g + (e >> 1) * 8;
                u64 j = c0 + wn * 64 + nj * 8 + t4 * 2 + (e & 1);
                u32 v = (u32)acc[mi][nj][e];
                if (i < n && j < n && v) atomicAdd(C + i * ldc + j, (CT)v);
            }
}

template <int V, typename CT>
cudaError_t run(ProductArgs& a, cudaStream_t st)
{
    constexpr int kStageWords = Mma<V>::kBitsPerStage / 64;
    const u64 T = (a.n + kBM - 1) / kBM;
    const u64 tiles = T * (T + 1) / 2;
    const u64 nst = (a.W + kStageWords - 1) / kStageWords;
    if (tiles == 0 || nst == 0) return cudaSuccess;
    u64 want = (u64)a.sms * 4;
    u64 ks = (want + tiles - 1) / tiles;
    // f32 exactness: each CTA's slice below kMaxSliceBits
    u64 min_ks = (nst * (u64)Mma<V>::kBitsPerStage + kMaxSliceBits - 1) / kMaxSliceBits;
    if (ks < min_ks) ks = min_ks;
    u64 maxks = (nst + 1) / 2;
    if (ks > maxks && maxks >= min_ks) ks = maxks;
    if (ks < 1) ks = 1;
    if (ks > 65535 || tiles > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    const int smem = kSmem + (V == JSIM_VARIANT_B1 ? 0 : kStageBytes);
    cudaError_t e = cudaFuncSetAttribute(k_prod_mma<V, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)tiles, (unsigned)ks);
    k_prod_mma<V, CT><<<grid, kThreads, smem, st>>>(a.X, a.stride, a.n, a.W, T, (u32)ks, (CT*)a.C, a.ldc);
    a.launches += 1;
    return cudaGetLastError();
}

template <int V>
cudaError_t run_v(ProductArgs& a, cudaStream_t st)
{
    return a.count_bits == 64 ? run<V, u64>(a, st) : run<V, u32>(a, st);
}

}  // namespace

cudaError_t product_mma(ProductArgs& a, int variant, cudaStream_t st)
{
    switch (variant) {
    case JSIM_VARIANT_F8: return run_v<JSIM_VARIANT_F8>(a, st);
    case JSIM_VARIANT_I8: return run_v<JSIM_VARIANT_I8>(a, st);
    case JSIM_VARIANT_B1: return run_v<JSIM_VARIANT_B1>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace jsim
