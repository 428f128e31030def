/*
 * jsim: exact all-pairs Jaccard similarity on one GB300 GPU (sm_103a).
 *
 * Method: "Communication-Efficient Jaccard Similarity for High-Performance
 * Distributed Genome Comparisons" (arXiv 1911.04200).  Each sample i is a
 * set X_i of unsigned 64-bit values (k-mer IDs in genomics).  The samples are
 * the columns of a boolean indicator matrix A (a_ki = 1 iff k in X_i,
 * Sec. III-A).  The library computes, for every pair of samples,
 *
 *   C[i][j] = |X_i ∩ X_j|            the intersection matrix A^T A (the paper
 *                                    calls it B, Sec. III-A)
 *   sizes[i] = |X_i|                 column sums of A (the paper's a-hat)
 *   J[i][j] = C / (|X_i|+|X_j|-C)    in IEEE binary64, round-to-nearest;
 *                                    1.0 when both sets are empty (Sec. II-A)
 *
 * by the paper's method (Sec. III-B): rows of A are cut into batches of
 * `batch_rows` consecutive values (Eq. 3); in each batch the all-zero rows are
 * dropped through a filter vector and its prefix sum (Eq. 5, Eq. 6); every 64
 * consecutive surviving rows of a sample become one bitmask word (b = 64);
 * and C accumulates sum_w popcount(word_wi AND word_wj) over all batches
 * (Eq. 7, Eq. 4).  All of it runs in this library's CUDA kernels.
 *
 * Results are exact: C and sizes are integers, and J is the correctly rounded
 * binary64 quotient of two integers below 2^53.
 *
 * Conventions for every call:
 *  - Return value: JSIM_OK (0) or one of the JSIM_ERR_* codes below;
 *    jsim_strerror() gives a message.  On an error no output buffer is
 *    written, except where a call says otherwise.
 *  - Ownership: the caller owns every buffer it passes.  The library reads
 *    inputs during the call only, never keeps or frees caller pointers, and
 *    frees whatever it allocated before it returns (handles excepted, which
 *    their destroy calls free).
 *  - Pointers are host or device pointers as the `mem` field or argument says.
 *    Device pointers must be on the context's device.  Host pointers may be
 *    pageable; pinned host memory makes the copies faster.
 *  - Calls on one context are not thread-safe; use one context per thread.
 *  - All device work is ordered on the context's stream; every call returns
 *    after its work has finished (it synchronises that stream).
 */
#ifndef JSIM_H
#define JSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define JSIM_API __attribute__((visibility("default")))
#else
#define JSIM_API
#endif

/* ---- error codes --------------------------------------------------------- */
#define JSIM_OK               0
#define JSIM_ERR_ARG          1  /* invalid argument (NULL pointer, bad size or option) */
#define JSIM_ERR_UNSORTED     2  /* a sample's values are not in ascending order */
#define JSIM_ERR_OVERFLOW     3  /* a set size does not fit count_bits */
#define JSIM_ERR_ID_RANGE     4  /* a value is >= 2^id_bits */
#define JSIM_ERR_OOM          5  /* the allocator returned NULL */
#define JSIM_ERR_CUDA         6  /* a CUDA runtime call failed (see jsim_last_cuda_error) */
#define JSIM_ERR_TIMEOUT      7  /* a bounded device wait ran out */
#define JSIM_ERR_CANCELLED    8  /* a request was cancelled */
#define JSIM_ERR_UNSUPPORTED  9  /* the requested variant or mode is not available */
#define JSIM_ERR_INCOMPLETE  10  /* the call stopped early as asked; its checkpoint holds the progress */
#define JSIM_ERR_CHECKPOINT  11  /* a checkpoint file is unreadable, corrupt or from another call */

/* ---- memory kinds ---------------------------------------------------------- */
#define JSIM_MEM_HOST   0
#define JSIM_MEM_DEVICE 1

/* ---- product variants (the semiring product of Eq. 7) --------------------- */
#define JSIM_VARIANT_AUTO 0  /* choose by size and density (measured table) */
#define JSIM_VARIANT_POPC 1  /* CUDA cores: AND + population count, register tiles */
#define JSIM_VARIANT_B1   2  /* legacy tensor mma.sync .b1 with .and.popc */
#define JSIM_VARIANT_I8   3  /* legacy tensor mma.sync .s8, bits unpacked to 0/1 bytes, s32 accumulate */
#define JSIM_VARIANT_F8   4  /* legacy tensor mma.sync .e4m3, bits unpacked to 0/1.0, f32 accumulate in exact ranges */
#define JSIM_VARIANT_TC   5  /* tcgen05.mma kind::f8f6f4 with TMEM accumulators, 0/1.0 e4m3 operands */
#define JSIM_VARIANT_TC2  6  /* as TC, on pairs of SMs (cta_group::2, 256 x 256 tiles) */
#define JSIM_VARIANT_SPARSE 7 /* block-sparse (jsim_all_pairs only, 1..2048 samples, tensor cores):
                                samples ordered by a sketch of their similarity into tiles of
                                128, rows held by one tile multiplied within that tile's
                                diagonal block only (Sec. III-B/III-C: sparsity and row/column
                                permutations); bit-identical results */
#define JSIM_VARIANT_COUNT 8

/*
 * A collection of n samples in compressed-row form: sample i is
 * ids[offsets[i] .. offsets[i+1]), sorted ascending.  Equal adjacent values
 * are one set element (set semantics).  offsets has n+1 entries and
 * offsets[0] must be 0.  n = 0 is allowed.  ids may be NULL when
 * offsets[n] = 0.  mem says where offsets and ids live.
 */
typedef struct {
    uint64_t n;
    const uint64_t* offsets;
    const uint64_t* ids;
    int mem;
} jsim_sets;

/* Device memory hooks.  alloc returns a device pointer of at least `bytes`
 * bytes, usable in stream order on `stream`, or NULL; free releases it. */
typedef void* (*jsim_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*jsim_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

typedef struct {
    uint64_t batch_rows;  /* m~ of Eq. 3: values per row batch, a multiple of 64;
                             0 = automatic (largest batch whose filter state stays
                             in L2 and whose packed block fits memory) */
    int word_bits;        /* b of the bitmask words: 64 (default) or 32 */
    int variant;          /* JSIM_VARIANT_* for the product */
    int count_bits;       /* width of C: 32 (default) or 64 */
    int id_bits;          /* values must be < 2^id_bits; 1..64 (default 64) */
    jsim_alloc_fn alloc;  /* NULL: cudaMallocAsync on the stream */
    jsim_free_fn free;    /* NULL: cudaFreeAsync on the stream */
    void* alloc_user;     /* passed to alloc/free */
    void* stream;         /* cudaStream_t; NULL = a stream the context creates */
    int device;           /* CUDA device ordinal */
    int timeout_ms;       /* bound on device-side waits (persistent kernels, serving) */
    int profile;          /* 1: record per-stage CUDA-event times into jsim_stats */
    int filter_min;       /* rows kept by the filter of a batch: 1 (default) keeps every
                             row some sample holds (Eq. 5); 2 keeps rows held by two or
                             more samples - a row only sample i holds adds 1 to C_ii alone,
                             and C_ii = |X_i| is known, so C and J are unchanged while the
                             product runs over fewer words.  Serving ignores it. */
    int distance;         /* 0 (default): the J output holds the similarity J = C / U (Eq. 2);
                             1: it holds the Jaccard distance D = 1 - J (Sec. II-A), the
                             binary64 subtraction 1.0 - J of the correctly rounded J
                             (D = 0 for two empty sets).  Applies to every call that writes
                             J (plain, streamed, batched, serving indexes built on the
                             context). */
    int count_useful;     /* 1: also count the useful work of the plain and streamed calls and
                             of jsim_product into jsim_stats.bitops_useful (one more read of
                             every packed batch; a resumed streamed call counts the
                             super-batches it ran); 0 (default): not counted */
    int tile_n;           /* tensor-core tiles of a batched call's job-table product: 128 x 256
                             (256) or 128 x 128 (128); 0 (default): the tuner times both */
} jsim_options;

typedef struct jsim_ctx jsim_ctx;

/* Statistics of the last jsim_all_pairs / jsim_product call on a context. */
typedef struct {
    uint64_t batches;          /* row batches processed (non-empty ones) */
    uint64_t rows_nonzero;     /* sum over batches of R_l = |f^(l)| (Eq. 5; rows of two or more
                                  samples with filter_min 2) */
    uint64_t words;            /* sum over batches of W_l = ceil(R_l / 64) */
    uint64_t batch_rows;       /* m~ actually used */
    int variant;               /* product variant actually used */
    int product_launches;      /* product kernel launches */
    int launches;              /* all kernel launches of the call */
    double ms_total;           /* wall time of the call's device work (profile=1) */
    double ms_h2d, ms_validate, ms_filter, ms_scan, ms_pack, ms_product, ms_epilogue, ms_d2h;
    double bitops_dense;       /* 64 * sum_l W_l * n(n+1)/2: dense AND+popcount bit-operations */
    double bitops_useful;      /* with count_useful: 64 * sum over word columns of
                                  nnz(nnz+1)/2, nnz the rows whose word is nonzero - the pairs of
                                  nonzero words, the work a sparse product needs (the operation
                                  count depends on the sparsity structure, Sec. IV); else 0 */
    double bitops_done;        /* bit-operations the product kernels carried out (64 per word pair of
                                  the upper triangle they multiplied): bitops_dense, except for the
                                  block-sparse variant, which skips the blocks no row reaches */
    uint64_t tile_n;           /* a batched call's tensor-core tiles: 128 x tile_n (256 or 128, as
                                  tuned); 0 when its product ran on CUDA cores */
    uint64_t pack_bytes;       /* bytes the pack kernels read and wrote by algorithm: 8 per value
                                  packed plus 8 per word of the packed matrices they fill (zero
                                  words included) */
    uint64_t h2d_copies;       /* host -> device DMA copies the call issued for its input */
    uint64_t h2d_bytes;        /* bytes of its input brought to the device (copies and pieces) */
    uint64_t h2d_pieces;       /* page-locked host input read by the device in this many value-range
                                  pieces while the batch loop ran (0: not fed in pieces) */
    uint64_t windows;          /* row windows the block-sparse variant's windowed ingest classified and
                                  packed (0: its per-value ingest ran, or another variant) */
} jsim_stats;

/* Fill *opt with the defaults described above. */
JSIM_API void jsim_default_options(jsim_options* opt);

/* Create a context on opt->device.  Returns JSIM_ERR_ARG for bad options. */
JSIM_API int jsim_create(jsim_ctx** out, const jsim_options* opt);

/* Destroy a context (waits for its stream).  NULL is ignored. */
JSIM_API void jsim_destroy(jsim_ctx* ctx);

/*
 * All-pairs similarity of one collection (Sec. III, Listing 1): C, sizes and
 * J as defined at the top of this file.
 *   C     n*n row-major, uint32 (count_bits 32) or uint64 (count_bits 64), or NULL
 *   sizes n entries, or NULL
 *   J     n*n row-major binary64, or NULL
 *   out_mem: JSIM_MEM_HOST or JSIM_MEM_DEVICE for all three outputs.
 * Host input of more than 4 GiB of values runs as jsim_all_pairs_streamed
 * with 1 GiB staging (copies overlap the device's work; same results, the
 * statistics count super-batches).
 * Errors: JSIM_ERR_ARG, JSIM_ERR_UNSORTED, JSIM_ERR_ID_RANGE, JSIM_ERR_OVERFLOW
 * (a size >= 2^count_bits), JSIM_ERR_OOM, JSIM_ERR_CUDA, JSIM_ERR_UNSUPPORTED.
 */
JSIM_API int jsim_all_pairs(jsim_ctx* ctx, const jsim_sets* sets,
                   void* C, uint64_t* sizes, double* J, int out_mem);

/*
 * One part of an all-pairs call split over several devices or processes
 * (the batches of Eq. 3 are independent and C is their sum, Eq. 4; the
 * paper's layered grid reduces the partial counts in the same way).  The
 * nb row batches between the collection's first and last value are cut into
 * `parts` contiguous runs; part p takes batches [nb*p/parts, nb*(p+1)/parts)
 * (by value range, so hashed values balance).
 *   part, parts   0 <= part < parts
 *   C             n*n counts of this part's rows (uint32 or uint64 as
 *                 count_bits), both triangles; required
 *   sizes         n distinct counts |X_i| of the whole samples (every part
 *                 gives the same), or NULL
 * Summing C over all parts (any order; each sum fits count_bits) and calling
 * jsim_finish gives jsim_all_pairs's C and J, bit for bit.  The input is
 * validated whole by every part.  Errors: as jsim_all_pairs.
 */
JSIM_API int jsim_all_pairs_part(jsim_ctx* ctx, const jsim_sets* sets, uint32_t part, uint32_t parts, void* C,
                                 uint64_t* sizes, int out_mem);

/*
 * C and J from summed counts: Cout = C with the diagonal set to sizes (a
 * part's rows may miss rows only one sample holds, with filter_min 2), J as
 * in jsim_all_pairs (or the distance, per the context's options).
 *   n       samples; C n*n counts (count_bits), sizes n
 *   Cout, J outputs (either may be NULL); mem: JSIM_MEM_HOST or JSIM_MEM_DEVICE for all
 * Errors: JSIM_ERR_ARG, JSIM_ERR_OOM, JSIM_ERR_CUDA.
 */
JSIM_API int jsim_finish(jsim_ctx* ctx, uint64_t n, const void* C, const uint64_t* sizes, void* Cout, double* J,
                         int mem);

/*
 * The partition rule of jsim_all_pairs_part, on the host (no device, no
 * context): the row batches of Eq. 3 that part `part` of `parts` counts, for
 * a collection whose values lie in [minid, maxid].
 *   batch_rows       m~ (a multiple of 64), or 0 for the automatic choice
 *                    (the one jsim_all_pairs makes for this value span)
 *   b_begin, b_end   batches [b_begin, b_end) of this part: batch b holds the
 *                    values [b m~, (b+1) m~); may be NULL
 *   batch_rows_used  the m~ used; may be NULL
 * Parts 0..parts-1 tile the batches from minid's to maxid's in order.  Lets
 * the ranks of a split contraction agree on the split before any device
 * work.  Errors: JSIM_ERR_ARG (parts 0, part >= parts, maxid < minid, or
 * batch_rows not a multiple of 64).
 */
JSIM_API int jsim_partition_batches(uint64_t minid, uint64_t maxid, uint64_t batch_rows, uint32_t part,
                                    uint32_t parts, uint64_t* b_begin, uint64_t* b_end, uint64_t* batch_rows_used);

/*
 * All-pairs similarity of k independent collections in one call (the
 * batched pattern).  Every collection is processed exactly as by
 * jsim_all_pairs (its own row batches, filter, prefix sum, words and product;
 * Sec. III-B, Eq. 3-7) and gets its own outputs:
 *   cols      k collections (host or device, each with its own mem)
 *   C, sizes, J   arrays of k pointers (or NULL for none); C[c] is n_c*n_c
 *             uint32/uint64, sizes[c] n_c, J[c] n_c*n_c binary64; an entry may
 *             be NULL.  out_mem applies to all of them.
 * Execution: one validation synchronisation for the whole call; the batches
 * of every collection are appended along the word axis on the device; the
 * products of all collections run as one persistent tensor-core launch (up to
 * 256 collections per launch) or, when the tuner measures it faster, one
 * CUDA-core launch per collection.  With variant AUTO and device-resident
 * inputs, collections of 256 to 2048 samples are instead validated first and
 * then run as jsim_all_pairs does (the block-sparse product where it pays;
 * their statistics add to the call's).  With variant AUTO the first call for a
 * collection shape times the candidate products and remembers the fastest for
 * the context.  When every input and output is in device memory the launch
 * sequence is captured into a CUDA graph and later calls with the same
 * collections (same pointers and offsets) replay it after re-validating.
 * Errors: as jsim_all_pairs, plus JSIM_ERR_UNSUPPORTED when a collection's
 * value span needs more than 4096 row batches.
 */
JSIM_API int jsim_all_pairs_batched(jsim_ctx* ctx, const jsim_sets* cols, uint64_t k, void* const* C,
                                    uint64_t* const* sizes, double* const* J, int out_mem);

/*
 * All-pairs similarity of one collection held in host memory, streamed to
 * the device in pieces (the batch loop of Sec. III-B, Eq. 3 and Eq. 4, for
 * inputs that do not fit in device memory).  Results are those of
 * jsim_all_pairs, bit for bit.
 *   sets          host memory only (JSIM_ERR_ARG otherwise); caller-owned,
 *                 read (never written) during the call
 *   C, sizes, J, out_mem   as jsim_all_pairs
 *   staging_bytes size of each of two pinned host staging buffers (>= 1 MiB);
 *                 the device holds two value buffers of at most this size,
 *                 filter bitmaps of at most twice it, and the packed matrix
 *                 of one super-batch
 * Execution: the value range is cut into super-batches of whole row batches
 * (m~ = batch_rows, or the automatic choice) whose values fit the staging;
 * each super-batch is filtered, ranked and packed as one batch (C is additive
 * over any partition of the rows, Eq. 4), so m~ only sets where super-batches
 * may begin and end.  While the device multiplies super-batch g, the host
 * gathers super-batch g+1 into the other pinned buffer and a second stream
 * copies it, so host->device traffic overlaps the product.  The pinned
 * buffers are kept by the context for later calls (freed by jsim_destroy).
 * Errors: as jsim_all_pairs, plus JSIM_ERR_OOM when a single row batch holds
 * more values than the staging (lower batch_rows or raise staging_bytes).
 */
JSIM_API int jsim_all_pairs_streamed(jsim_ctx* ctx, const jsim_sets* sets, void* C, uint64_t* sizes, double* J,
                                     int out_mem, uint64_t staging_bytes);

/* Checkpoint/resume of a streamed call (progress is kept after whole
 * super-batches: the counts C accumulated so far - a sum over batches, Eq. 4,
 * so the remaining super-batches can be added later - the sizes, the
 * input-error flags and the statistics). */
typedef struct {
    const char* path;     /* checkpoint file; written as path + ".tmp", then renamed */
    uint32_t every;       /* write it after every `every` super-batches (0: only when stopping) */
    uint32_t max_supers;  /* process at most this many super-batches in this call (0: all); if work
                             remains, write the checkpoint and return JSIM_ERR_INCOMPLETE */
    int resume;           /* 1: when `path` exists, continue after the super-batches it holds */
} jsim_checkpoint;

/*
 * jsim_all_pairs_streamed with checkpoints (ck may be NULL: no checkpoint).
 * A resumed call must be the same call: the same collection (checked by a
 * fingerprint of the offsets, every sample's first and last value and 4096
 * evenly spaced values), options and staging_bytes; otherwise, or when the
 * file is corrupt (checksum), it returns JSIM_ERR_CHECKPOINT and writes
 * nothing.  The file stays in place after a complete call.  The results of a
 * call resumed any number of times are those of one uninterrupted call, bit
 * for bit.  The file holds host-endian binary (header, sizes, C, checksum).
 * Errors: as jsim_all_pairs_streamed, plus JSIM_ERR_INCOMPLETE (max_supers
 * reached with work left) and JSIM_ERR_CHECKPOINT (file I/O, mismatch,
 * corruption; max_supers without a path).
 */
JSIM_API int jsim_all_pairs_streamed_ckpt(jsim_ctx* ctx, const jsim_sets* sets, void* C, uint64_t* sizes,
                                          double* J, int out_mem, uint64_t staging_bytes,
                                          const jsim_checkpoint* ck);

/*
 * One row batch of the method, for inspection and step-level testing
 * (Eq. 5, Eq. 6 and the bitmask compression before Eq. 7): the values of
 * each sample in [lo, lo + width) become packed words.
 *   width     a multiple of 64, > 0
 *   filter    width/64 uint64 words of f^(l) (bit k of word w = row 64w+k), or NULL
 *   words     n rows of `stride` uint64 words, word r/64 bit r%64 set iff the
 *             sample holds the value of rank r (rank = p^(l), LSB first);
 *             words beyond W = ceil(R/64) in a row are zero.  Or NULL.
 *   stride    row stride of `words` in uint64 units, >= ceil(width/64) or >= W
 *   R_out     number of nonzero rows R_l (may be NULL)
 *   sizes     per-sample count of distinct values in the batch (Eq. 4's a-hat^(l)), or NULL
 * If stride < W, returns JSIM_ERR_ARG with *R_out set, so a caller may ask for
 * R first with words = NULL.
 */
JSIM_API int jsim_pack(jsim_ctx* ctx, const jsim_sets* sets, uint64_t lo, uint64_t width,
              uint64_t* filter, uint64_t* words, uint64_t stride, uint64_t* R_out,
              uint64_t* sizes, int out_mem);

/*
 * The semiring product alone (Eq. 7) on packed words already in device
 * memory: C[i][j] = sum_{w<W} popcount(words[i][w] AND words[j][w]) for all
 * i, j (computed on the upper triangle and mirrored).
 *   words   device, n rows of `stride` uint64 words (stride >= W)
 *   C       device, n*n uint32 (count_bits 32) or uint64, overwritten
 *   variant JSIM_VARIANT_*
 * Errors: JSIM_ERR_ARG, JSIM_ERR_UNSUPPORTED, JSIM_ERR_OOM, JSIM_ERR_CUDA.
 */
JSIM_API int jsim_product(jsim_ctx* ctx, const uint64_t* words, uint64_t n, uint64_t W, uint64_t stride,
                 void* C, int variant);

/*
 * Allocation-free variant of jsim_product, for callers that cannot let the
 * library allocate device memory during a call - for example an application
 * that owns a fixed memory budget for the whole GPU, or a steady-state loop
 * that must not stall on an allocation.  The paper has no counterpart: it is
 * an interface of this library only.
 *
 * Same arguments, result and errors as jsim_product; the caller still passes
 * the packed words and C.  Instead of allocating, the call keeps its scratch
 * (the count accumulator and a device error word) in one fixed array of
 * 4 MiB + 256 bytes of device memory owned by the library module, so n*n
 * counts must fit in 4 MiB: n <= 1024 with count_bits 32, n <= 724 with
 * count_bits 64; larger n returns JSIM_ERR_ARG.  Every GPU that loads the
 * library holds the array until the process exits.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with the context's device current); make that first call before
 * any stream capture.  The address is kept for the life of the process: a
 * device reset (cudaDeviceReset, or anything else that destroys the
 * device's primary context) invalidates it, and no call may follow one.  All calls on a device share the array and the call
 * clears what it needs before use, so calls that overlap on the GPU (two
 * streams, two threads, two contexts on one device) race: serialize them.
 */
JSIM_API int jsim_product_noalloc(jsim_ctx* ctx, const uint64_t* words, uint64_t n, uint64_t W,
                                  uint64_t stride, void* C, int variant);

/* ---- Serving: a resident reference index and continuous query batching ----
 *
 * The reference collection is packed once, as one batch of the method over
 * its whole value range (Sec. III-B: filter f, Eq. 5; rank directory, Eq. 6;
 * the kept rows of Abar, each an n_ref-bit vector of the reference samples
 * holding it), and stays in device memory.  A query sample Q is compared
 * with every reference sample S_j: C[q][j] = |Q cap S_j|, J as above, and
 * |Q| counts every distinct value of Q, also those the reference lacks.
 * Query values are ranked against the resident filter (a value absent from
 * f meets no reference sample), and C[q] is the sum of the rows of Q's
 * values (Eq. 7 with the query's 0/1 column): one row read per value.
 */
typedef struct jsim_index jsim_index;
typedef struct jsim_request jsim_request;

typedef struct {
    uint64_t max_batch_samples; /* query samples per device batch, 1..64 (default 64) */
    uint64_t max_batch_values;  /* query values per device batch, < 2^32 (default 2^27) */
    int slots;                  /* device batches in flight, 1..8 (default 3) */
} jsim_serve_options;

typedef struct {
    uint64_t requests_submitted, requests_done, samples_done, values_done;
    uint64_t batches;           /* device batches retired */
    uint64_t queued;            /* requests waiting for a slot now */
    uint64_t rows_read;         /* index rows read (query values the reference filter holds), summed */
    double ms_device;           /* device time of the batches (copy in to copy out), summed */
    double ms_product;          /* device time of the query x index kernels, summed */
    double index_bytes_read;    /* rows read x row bytes (ceil(n_ref / 64) x 8), summed */
    double bitops_dense;        /* rows read x n_ref (one AND+popcount bit per row and reference), summed */
} jsim_serve_stats;

JSIM_API void jsim_serve_default_options(jsim_serve_options* opt);

/*
 * Build the index of `ref` (host or device memory, n >= 1) on the context's
 * device and start its server thread.  The index allocates everything it will
 * use here (index, filter, per-slot buffers, pinned staging) through the
 * context's allocator; serving allocates nothing.  The context must outlive
 * the index and must not be used by another thread during this call.
 * Device memory: R x ceil(n / 64) x 8 bytes of index (R the reference's
 * distinct values), width/8 + width/16 bytes of filter and directory, and
 * per slot about max_batch_values x 8 + max_batch_samples x n x 16 bytes.
 * Errors: JSIM_ERR_ARG, JSIM_ERR_UNSORTED, JSIM_ERR_ID_RANGE, JSIM_ERR_OOM,
 * JSIM_ERR_CUDA, JSIM_ERR_UNSUPPORTED (reference value span >= 2^36, or
 * more than 8192 reference samples).
 */
JSIM_API int jsim_index_build(jsim_ctx* ctx, const jsim_sets* ref, const jsim_serve_options* opt,
                              jsim_index** out);

/* Stop the server (queued requests end with JSIM_ERR_CANCELLED, running
 * batches finish) and free the index.  Free every request first or after;
 * a request that was cancelled here stays valid until jsim_request_free. */
JSIM_API void jsim_index_destroy(jsim_index* ix);

/* n_ref, the index's rows R (the reference's distinct values), and the
 * reference sizes |S_j| (host, n_ref entries); any pointer may be NULL. */
JSIM_API int jsim_index_info(const jsim_index* ix, uint64_t* n_ref, uint64_t* words, uint64_t* ref_sizes);

/* Server counters since the index was built. */
JSIM_API int jsim_index_stats(jsim_index* ix, jsim_serve_stats* out);

/*
 * Queue a request of q->n query samples (host memory only).  Thread-safe.
 * The offsets are copied; the values are read by the server until the
 * request is done, so they must stay valid and unchanged until
 * jsim_request_wait has returned for it (or jsim_request_free).
 * Errors: JSIM_ERR_ARG (bad offsets, device memory, or more samples or values
 * than one batch holds), JSIM_ERR_CANCELLED (the index is stopping).
 */
JSIM_API int jsim_query_submit(jsim_index* ix, const jsim_sets* q, jsim_request** out);

/*
 * Wait up to timeout_ms (< 0: no limit) for a request and copy its results
 * (host memory; any may be NULL): C q x n_ref (uint32 or uint64 as the
 * context's count_bits), qsizes q, J q x n_ref binary64.
 * Errors: JSIM_ERR_TIMEOUT (not done yet; wait again), JSIM_ERR_UNSORTED or
 * JSIM_ERR_ID_RANGE (this request's input), JSIM_ERR_OVERFLOW,
 * JSIM_ERR_CANCELLED, JSIM_ERR_CUDA.
 */
JSIM_API int jsim_request_wait(jsim_request* r, void* C, uint64_t* qsizes, double* J, int timeout_ms);

/* Host-clock times of a finished request: submit to admission into a device
 * batch, and submit to results ready.  JSIM_ERR_TIMEOUT while not done. */
JSIM_API int jsim_request_latency(const jsim_request* r, double* queued_ms, double* total_ms);

/* Release a request: a queued one is withdrawn, a running one is waited for. */
JSIM_API void jsim_request_free(jsim_request* r);

/*
 * Nearest neighbours: for every sample i, the k samples j != i with the
 * largest J[i][j], best first; ties in J go to the smaller j, so the result is
 * unique.  The sparsified output for collections too large to keep n x n
 * (the paper's all-pairs matrix, Sec. II-A, feeds exactly such queries).
 *   J     n*n row-major binary64 as jsim_all_pairs writes it (values in [0, 1])
 *   k     1..64 and < n
 *   idx   n*k uint64 neighbour indices; val n*k binary64 of their J, or NULL
 *   mem   JSIM_MEM_HOST or JSIM_MEM_DEVICE for J, idx and val
 * Errors: JSIM_ERR_ARG, JSIM_ERR_OOM, JSIM_ERR_CUDA.
 */
JSIM_API int jsim_topk(jsim_ctx* ctx, const double* J, uint64_t n, uint32_t k, uint64_t* idx, double* val,
                       int mem);

/*
 * Threshold output: the pairs i < j with J[i][j] >= tau (below = 0), or with
 * J[i][j] <= tau (below = 1, for a distance matrix), in row-major order (i,
 * then j).  The sparse form of the all-pairs matrix (Sec. II-A) for
 * collections too large to keep n x n.
 *   J      n*n row-major binary64 as jsim_all_pairs writes it
 *   tau    threshold (not NaN)
 *   cap    capacity of pi, pj and val in pairs (0: count only)
 *   pi,pj  uint64 indices of the first min(count, cap) pairs (NULL when cap is 0)
 *   val    their J, or NULL
 *   count  total number of pairs that pass (also when above cap)
 *   mem    JSIM_MEM_HOST or JSIM_MEM_DEVICE for J, pi, pj and val (count: host)
 * Errors: JSIM_ERR_ARG, JSIM_ERR_OOM, JSIM_ERR_CUDA.
 */
JSIM_API int jsim_threshold(jsim_ctx* ctx, const double* J, uint64_t n, double tau, int below, uint64_t cap,
                            uint64_t* pi, uint64_t* pj, double* val, uint64_t* count, int mem);

/*
 * Self-check of the work schedule of the job-table tensor-core product (the
 * persistent launch of jsim_all_pairs_batched), on the host: no device, no
 * context.  The paper has no counterpart; the product it schedules is Eq. 7.
 * For a launch of `grid` persistent CTAs over `njobs` collections (job k: n[k]
 * samples, W[k] packed words per sample, rows of stride[k] words, rows[k] >=
 * n[k] rows allocated), it replays what every CTA does - each unpack
 * thread's loads (row, word, 16-byte alignment), the MMA thread's segments
 * and accumulator slots, the epilogue's TMEM columns and count writes - with
 * the same functions the kernel runs, and checks every address against its
 * buffer, that every (collection, tile, stage) unit is taken exactly once,
 * that every pair i <= j lies in exactly one tile, that no accumulator holds
 * more stages than the exact-count cap, and that every slot is drained as
 * often as it is committed.
 *   njobs       1..256; grid >= 1
 *   tile_n      the tile width: 256 (tiles of 128 x 256) or 128 (tiles of 128 x 128)
 *   stage_bits  bit-rows per stage: 256 (or 0), or 512 with tile_n 128 (the
 *               diagonal-only launch of the block-sparse path)
 *   msg         receives a description of the first failed check (cap bytes, may be NULL)
 * Returns 0 when every check passes, JSIM_ERR_ARG for bad arguments, and a
 * positive check number otherwise.
 */
JSIM_API int jsim_check_tc_schedule(uint32_t njobs, const uint64_t* n, const uint64_t* W, const uint64_t* stride,
                                    const uint64_t* rows, uint32_t grid, uint32_t tile_n, uint32_t stage_bits,
                                    char* msg, size_t cap);

/* Statistics of the last call on the context. */
JSIM_API int jsim_get_stats(const jsim_ctx* ctx, jsim_stats* out);

/* Message for an error code. */
JSIM_API const char* jsim_strerror(int code);

/* The CUDA error string behind the last JSIM_ERR_CUDA on this context. */
JSIM_API const char* jsim_last_cuda_error(const jsim_ctx* ctx);

/* Library version, e.g. "jsim 0.1". */
JSIM_API const char* jsim_version(void);

#ifdef __cplusplus
}
#endif
#endif /* JSIM_H */
