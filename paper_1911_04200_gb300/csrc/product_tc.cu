// Semiring product on the 5th-generation tensor cores (tcgen05, sm_103a):
// C += X X^T over (AND, popcount, +) (Eq. 7), computed exactly as an FP8
// matrix product of 0/1 values.
//
// Every bit of a packed word becomes one e4m3 byte, 0x00 (0.0) or 0x38
// (1.0); a product of two such values is 0 or 1, and the tensor core sums
// them into FP32 accumulators held in tensor memory (TMEM).  A CTA's slice of
// the word range is capped at 2^22 bit-rows, so every accumulator is an
// integer below 2^24 and FP32 holds it exactly.  The epilogue converts to
// integers and adds them into C.
//
// A CTA owns a 128 x 256 tile of C (128 rows of the A side, 256 of the B
// side, both taken from X) that touches the upper triangle, and a slice of the
// word range.  One stage covers 256 bit-rows: the packed words are loaded
// with plain 8-byte loads (prefetched two stages ahead in registers), expanded
// to bytes by all 256 threads and stored into shared memory in the canonical
// K-major 128-byte-swizzle layout (8-row x 128-byte atoms, 16-byte chunk c of
// row r at c ^ (r % 8)), two 128-byte column blocks per operand.  After a
// proxy fence and a CTA barrier one thread issues 8 tcgen05.mma
// (M=128, N=256, K=32 each) and commits them to the stage buffer's mbarrier;
// the buffer is refilled once that barrier reports the tensor core done with
// it.  Two stage buffers of 96 KiB alternate.  Every mbarrier wait is bounded
// (clock64 budget); on time-out the CTA raises an error flag, waits (bounded)
// for its committed MMAs, frees its TMEM and leaves.
#include <algorithm>
#include "common.cuh"

namespace jsim {

namespace {

constexpr int kThreads = 256;
constexpr int kM = 128;                 // A-side rows per tile
constexpr int kN = 256;                 // B-side rows per tile
constexpr int kStageBits = 256;         // bit-rows per stage
constexpr int kStageWords = kStageBits / 64;
constexpr int kBlkBytes = 128;          // one swizzle atom row
// one byte per bit-row after unpacking
constexpr int kABytes = kM * kStageBits;       // 32 KiB (two 16 KiB column blocks)
constexpr int kBBytes = kN * kStageBits;       // 64 KiB (two 32 KiB column blocks)
constexpr int kStageBytes = kABytes + kBBytes; // 96 KiB
static_assert(kABytes == (kStageBits / 128) * kM * kBlkBytes, "A stage = column blocks x rows x 128 B");
static_assert(kBBytes == (kStageBits / 128) * kN * kBlkBytes, "B stage = column blocks x rows x 128 B");
constexpr int kStages = 2;
constexpr int kSmemBytes = kStages * kStageBytes + 1024;  // + alignment slack
static_assert(kSmemBytes <= 232448, "fits the per-CTA shared-memory limit");
constexpr int kTmemCols = 256;
constexpr u64 kMaxSliceBits = 1ull << 22;
constexpr u32 kErrTimeout = 4u;

// instruction descriptor: kind::f8f6f4, D = F32, A = B = E4M3, both K-major,
// N = 256 (bits 17..22 hold N/8), M = 128 (bits 24..28 hold M/16)
constexpr u32 kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((u32)(kN >> 3) << 17) | ((u32)(kM >> 4) << 24);

__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, K-major, 128-byte swizzle: start address,
// leading byte offset 16 (unused by swizzled K-major), stride byte offset
// 1024 (next 8-row group), descriptor version 1, layout SWIZZLE_128B (2)
__device__ __forceinline__ u64 sw128_desc(u32 saddr)
{
    return (u64)((saddr & 0x3FFFFu) >> 4) | ((u64)1 << 16) | ((u64)(1024 >> 4) << 32) | ((u64)1 << 46) |
           ((u64)2 << 61);
}

__device__ __forceinline__ void mbar_init(u64* bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity)
{
    u32 ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// bounded wait: true when the phase completed, false on time-out
__device__ __forceinline__ bool mbar_wait(u64* bar, u32 parity, long long budget)
{
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

__device__ __forceinline__ u32 expand4(u32 nib)
{
    return ((nib * 0x00204081u) & 0x01010101u) * 0x38u;
}

__device__ __forceinline__ void tmem_ld32(u32 taddr, u32 (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// tile t -> (ti, tj) over 128 x 256 tiles with rows [128 ti, +128) and
// columns [256 tj, +256) that hold at least one pair i <= j (ti <= 2 tj + 1)
__device__ __forceinline__ void tc_tile(u64 t, u64 TM, u64& ti, u64& tj)
{
    u64 j = 0;
    for (;;) {
        u64 cnt = min(TM, 2 * j + 2);
        if (t < cnt) break;
        t -= cnt;
        ++j;
    }
    ti = t;
    tj = j;
}

template <typename CT>
__global__ void __launch_bounds__(kThreads, 1)
k_prod_tc(const u64* __restrict__ X, u64 stride, u64 n, u64 W, u64 TM, u32 ksplit, CT* __restrict__ C, u64 ldc,
          u32* err, long long budget)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) u64 bars[kStages];
    __shared__ u32 tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    u64 ti, tj;
    tc_tile(blockIdx.x, TM, ti, tj);
    const u64 r0 = ti * kM, c0 = tj * kN;
    const u64 nst = (W + kStageWords - 1) / kStageWords;
    const u64 s_begin = nst * blockIdx.y / ksplit, s_end = nst * (blockIdx.y + 1) / ksplit;
    if (s_begin >= s_end) return;  // uniform per CTA, before any TMEM or barrier use

    // 1024-aligned operand area
    const u32 raw = smem_u32(smem_raw);
    const u32 base = (raw + 1023u) & ~1023u;
    unsigned char* sm = smem_raw + (base - raw);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     :: "r"(smem_u32(&tmem_slot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const u32 tmem = tmem_slot;

    // this thread's three (row, 128-bit block) items of every stage, loaded
    // two stages ahead
    u64 cur[3][2], nxt[3][2], nxt2[3][2];
    auto load = [&](u64 s, u64 (&v)[3][2]) {
        const u64 k0 = s * kStageWords;
        #pragma unroll
        for (int e = 0; e < 3; ++e) {
            int idx = tid + kThreads * e;
            int ra = idx >> 1, blk = idx & 1;
            u64 grow = ra < kM ? r0 + ra : c0 + (ra - kM);
            u64 gk = k0 + 2 * blk;
            const u64* p = X + grow * stride + gk;
            bool rowok = grow < n;
            v[e][0] = (rowok && gk < W) ? __ldg(p) : 0ull;
            v[e][1] = (rowok && gk + 1 < W) ? __ldg(p + 1) : 0ull;
        }
    };
    auto unpack = [&](int b, const u64 (&v)[3][2]) {
        unsigned char* sbuf = sm + b * kStageBytes;
        #pragma unroll
        for (int e = 0; e < 3; ++e) {
            int idx = tid + kThreads * e;
            int ra = idx >> 1, blk = idx & 1;
            unsigned char* opbase;
            int row;
            if (ra < kM) { opbase = sbuf + blk * (kM * kBlkBytes); row = ra; }
            else { opbase = sbuf + kABytes + blk * (kN * kBlkBytes); row = ra - kM; }
            unsigned char* rowp = opbase + row * kBlkBytes;
            #pragma unroll
            for (int c = 0; c < 8; ++c) {
                u32 h = (u32)(v[e][c >> 2] >> (16 * (c & 3)));
                uint4 o;
                o.x = expand4(h & 15u);
                o.y = expand4((h >> 4) & 15u);
                o.z = expand4((h >> 8) & 15u);
                o.w = expand4((h >> 12) & 15u);
                *(uint4*)(rowp + ((c ^ (row & 7)) << 4)) = o;
            }
        }
    };

    bool ok = true;
    load(s_begin, cur);
    if (s_begin + 1 < s_end) load(s_begin + 1, nxt);
    for (u64 s = s_begin; s < s_end; ++s) {
        const int b = (int)((s - s_begin) & 1);
        if (s + 2 < s_end) load(s + 2, nxt2);
        // buffer b was last read by the MMAs of stage s - 2
        if (s - s_begin >= 2) {
            u32 parity = (u32)(((s - s_begin) / 2 - 1) & 1);
            if (!mbar_wait(&bars[b], parity, budget)) ok = false;
        }
        if (__syncthreads_and(ok) == 0) { ok = false; break; }
        unpack(b, cur);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const u32 abase = base + b * kStageBytes, bbase = abase + kABytes;
            #pragma unroll
            for (int k = 0; k < kStageBits / 32; ++k) {
                const int blk = k >> 2, off = (k & 3) * 32;
                u64 da = sw128_desc(abase + blk * (kM * kBlkBytes) + off);
                u64 db = sw128_desc(bbase + blk * (kN * kBlkBytes) + off);
                u32 acc = (s > s_begin || k > 0) ? 1u : 0u;
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
                             :: "r"(tmem), "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         :: "r"(smem_u32(&bars[b])) : "memory");
        }
        #pragma unroll
        for (int e = 0; e < 3; ++e) {
            cur[e][0] = nxt[e][0]; cur[e][1] = nxt[e][1];
            nxt[e][0] = nxt2[e][0]; nxt[e][1] = nxt2[e][1];
        }
    }

    // wait for every committed stage (the last commit on each buffer)
    const u64 ns = s_end - s_begin;
    for (int b = 0; b < kStages; ++b) {
        if ((u64)b >= ns) continue;
        // the last stage that used buffer b is its (last / 2)-th commit; the
        // barrier has completed either last / 2 or last / 2 + 1 phases, so
        // the parity of that phase tells which
        u64 last = ((ns - 1 - b) / 2) * 2 + b;
        u32 parity = (u32)((last / 2) & 1);
        if (!mbar_wait(&bars[b], parity, budget)) ok = false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const bool all_ok = __syncthreads_and(ok) != 0;

    if (all_ok && warp < 4) {
        // TMEM lane = tile row, column = tile column
        const u64 i = r0 + warp * 32 + lane;
        #pragma unroll 1
        for (int cb = 0; cb < kN / 32; ++cb) {
            u32 r[32];
            tmem_ld32(tmem + ((u32)(warp * 32) << 16) + (u32)(cb * 32), r);
            if (i < n) {
                #pragma unroll
                for (int x = 0; x < 32; ++x) {
                    u64 j = c0 + cb * 32 + x;
                    u32 v = (u32)__uint_as_float(r[x]);
                    if (j < n && i <= j && v) atomicAdd(C + i * ldc + j, (CT)v);
                }
            }
        }
    }
    if (!all_ok && tid == 0) atomicOr(err, kErrTimeout);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(kTmemCols));
    }
}

template <typename CT>
cudaError_t run(ProductArgs& a, cudaStream_t st)
{
    const u64 TM = (a.n + kM - 1) / kM, TN = (a.n + kN - 1) / kN;
    u64 tiles = 0;
    for (u64 j = 0; j < TN; ++j) tiles += std::min<u64>(TM, 2 * j + 2);
    const u64 nst = (a.W + kStageWords - 1) / kStageWords;
    if (tiles == 0 || nst == 0) return cudaSuccess;
    u64 want = (u64)a.sms;  // one wave of one CTA per SM
    u64 ks = (want + tiles - 1) / tiles;
    u64 min_ks = (nst * (u64)kStageBits + kMaxSliceBits - 1) / kMaxSliceBits;
    if (ks < min_ks) ks = min_ks;
    u64 maxks = (nst + 3) / 4;  // at least 4 stages per CTA
    if (ks > maxks && maxks >= min_ks) ks = maxks;
    if (ks < 1) ks = 1;
    if (ks > 65535 || tiles > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_prod_tc<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    long long budget = (long long)(clk_khz > 0 ? clk_khz : 2000000) * 1000LL * (long long)a.timeout_ms / 1000LL;
    dim3 grid((unsigned)tiles, (unsigned)ks);
    k_prod_tc<CT><<<grid, kThreads, kSmemBytes, st>>>(a.X, a.stride, a.n, a.W, TM, (u32)ks, (CT*)a.C, a.ldc,
                                                      a.err, budget);
    a.launches += 1;
    return cudaGetLastError();
}

}  // namespace

bool product_tc_supported(int device)
{
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) return false;
    return major == 10 && minor == 3;
}

cudaError_t product_tc(ProductArgs& a, cudaStream_t st)
{
    return a.count_bits == 64 ? run<u64>(a, st) : run<u32>(a, st);
}

}  // namespace jsim
