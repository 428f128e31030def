/*
 * Exact all-pairs Jaccard oracle: TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load this library.  The product path never calls it and shares no code
 * with it: no headers, no helpers, no constants.
 *
 * What it computes is the plain definition of the quantities (Sec. II-A and
 * Sec. III-A of "Communication-Efficient Jaccard Similarity for
 * High-Performance Distributed Genome Comparisons", arXiv 1911.04200):
 *
 *   |X_i|                 number of distinct values of sample i
 *   b_ij = |X_i ∩ X_j|    counted by a two-pointer merge of the two sorted
 *                         value lists (the intersection matrix, Sec. III-A;
 *                         called C in this library's interface)
 *   c_ij = |X_i| + |X_j| - b_ij           (union by inclusion-exclusion)
 *   s_ij = b_ij / c_ij    in IEEE binary64, round-to-nearest (Eq. 2);
 *                         s_ij = 1 when both sets are empty (Sec. II-A)
 *   d_ij = 1.0 - s_ij     the Jaccard distance (Sec. II-A), one binary64
 *                         subtraction
 *
 * Inputs are sample value lists sorted ascending (the paper's samples are
 * sorted numeric files, Sec. IV); equal adjacent values are one set element.
 * There is no blocking, no packing and no reordering: every pair is merged.
 *
 * For collections too large to merge pair by pair in memory, b_ij is also
 * given by its other plain reading, B = A^T A summed over the rows of the
 * indicator matrix (oracle_rows_range below), restricted to a value range so
 * that disjoint ranges add up (Eq. 4).
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

/* Number of distinct values in a sorted list (|X|, Sec. II-A). */
uint64_t oracle_distinct(const uint64_t* a, uint64_t na)
{
    uint64_t k = 0;
    for (uint64_t i = 0; i < na; ++i)
        if (i == 0 || a[i] != a[i - 1]) ++k;
    return k;
}

/* |X ∩ Y| for two sorted lists, by a two-pointer merge (Sec. II-A). */
uint64_t oracle_intersect(const uint64_t* a, uint64_t na,
                          const uint64_t* b, uint64_t nb)
{
    uint64_t i = 0, j = 0, k = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) {
            ++i;
        } else if (b[j] < a[i]) {
            ++j;
        } else {
            uint64_t v = a[i];
            ++k;
            while (i < na && a[i] == v) ++i;
            while (j < nb && b[j] == v) ++j;
        }
    }
    return k;
}

/* s = b / (|X|+|Y|-b) in binary64; 1 for two empty sets (Sec. II-A, Eq. 2). */
double oracle_jaccard(uint64_t inter, uint64_t size_x, uint64_t size_y)
{
    uint64_t uni = size_x + size_y - inter;
    if (uni == 0) return 1.0;
    return (double)inter / (double)uni;
}

/*
 * Jaccard distance 1 - J (Sec. II-A), as the binary64 subtraction 1.0 - J of
 * the correctly rounded J above (0 for two empty sets).
 */
double oracle_distance(uint64_t inter, uint64_t size_x, uint64_t size_y)
{
    return 1.0 - oracle_jaccard(inter, size_x, size_y);
}

/* J[r][c] = oracle_jaccard(C[r][c], srow[r], scol[c]) for an nr x nc matrix. */
void oracle_jaccard_matrix(uint64_t nr, uint64_t nc, const uint64_t* C, const uint64_t* srow,
                           const uint64_t* scol, double* J)
{
    for (uint64_t r = 0; r < nr; ++r)
        for (uint64_t c = 0; c < nc; ++c) J[r * nc + c] = oracle_jaccard(C[r * nc + c], srow[r], scol[c]);
}

/* D[r][c] = oracle_distance(C[r][c], srow[r], scol[c]) for an nr x nc matrix. */
void oracle_distance_matrix(uint64_t nr, uint64_t nc, const uint64_t* C, const uint64_t* srow,
                            const uint64_t* scol, double* D)
{
    for (uint64_t r = 0; r < nr; ++r)
        for (uint64_t c = 0; c < nc; ++c) D[r * nc + c] = oracle_distance(C[r * nc + c], srow[r], scol[c]);
}

/*
 * All pairs of one collection.  offsets has n+1 entries; sample i is
 * ids[offsets[i] .. offsets[i+1]).  C and J are n*n row-major (either may be
 * NULL), sizes has n entries (may be NULL).
 */
void oracle_all_pairs(uint64_t n, const uint64_t* offsets, const uint64_t* ids,
                      uint64_t* C, uint64_t* sizes, double* J, int threads)
{
    uint64_t* sz = sizes;
    /* sizes are needed for J; compute them first */
    #pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t d = oracle_distinct(ids + offsets[i], offsets[i + 1] - offsets[i]);
        if (sz) sz[i] = d;
    }
    #pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        const uint64_t* a = ids + offsets[i];
        uint64_t na = offsets[i + 1] - offsets[i];
        uint64_t si = sz ? sz[i] : oracle_distinct(a, na);
        for (uint64_t j = (uint64_t)i; j < n; ++j) {
            const uint64_t* b = ids + offsets[j];
            uint64_t nb = offsets[j + 1] - offsets[j];
            uint64_t inter = oracle_intersect(a, na, b, nb);
            if (C) { C[(uint64_t)i * n + j] = inter; C[j * n + (uint64_t)i] = inter; }
            if (J) {
                uint64_t sj = sz ? sz[j] : oracle_distinct(b, nb);
                double s = oracle_jaccard(inter, si, sj);
                J[(uint64_t)i * n + j] = s;
                J[j * n + (uint64_t)i] = s;
            }
        }
    }
}

/*
 * A sample of pairs (pi[t], pj[t]) of one collection, each merged on its own.
 * Used where the whole matrix is too large for this oracle.
 */
void oracle_pairs(uint64_t n, const uint64_t* offsets, const uint64_t* ids,
                  uint64_t npairs, const uint64_t* pi, const uint64_t* pj,
                  uint64_t* C_out, double* J_out, int threads)
{
    (void)n;
    #pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
    for (int64_t t = 0; t < (int64_t)npairs; ++t) {
        const uint64_t* a = ids + offsets[pi[t]];
        uint64_t na = offsets[pi[t] + 1] - offsets[pi[t]];
        const uint64_t* b = ids + offsets[pj[t]];
        uint64_t nb = offsets[pj[t] + 1] - offsets[pj[t]];
        uint64_t inter = oracle_intersect(a, na, b, nb);
        if (C_out) C_out[t] = inter;
        if (J_out) J_out[t] = oracle_jaccard(inter, oracle_distinct(a, na), oracle_distinct(b, nb));
    }
}

/*
 * Query collection against reference collection: C[q][r] = |Q_q ∩ R_r|,
 * J likewise (the same definitions with X from one collection and Y from the
 * other).  C and J are nq*nr row-major; qsizes has nq entries.
 */
void oracle_cross(uint64_t nq, const uint64_t* qoff, const uint64_t* qids,
                  uint64_t nr, const uint64_t* roff, const uint64_t* rids,
                  uint64_t* C, uint64_t* qsizes, double* J, int threads)
{
    #pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
    for (int64_t q = 0; q < (int64_t)nq; ++q) {
        const uint64_t* a = qids + qoff[q];
        uint64_t na = qoff[q + 1] - qoff[q];
        uint64_t sq = oracle_distinct(a, na);
        if (qsizes) qsizes[q] = sq;
        for (uint64_t r = 0; r < nr; ++r) {
            const uint64_t* b = rids + roff[r];
            uint64_t nb = roff[r + 1] - roff[r];
            uint64_t inter = oracle_intersect(a, na, b, nb);
            if (C) C[(uint64_t)q * nr + r] = inter;
            if (J) J[(uint64_t)q * nr + r] = oracle_jaccard(inter, sq, oracle_distinct(b, nb));
        }
    }
}

/*
 * Intersection counts by the rows of the indicator matrix, restricted to the
 * values of [lo, hi): the plain definition B = A^T A of Sec. III-A read row
 * by row, B = sum over values x of a_x a_x^T, where a_x is the 0/1 row of
 * value x (sample i holds x).  Every value x in [lo, hi) adds 1 to C[i][j]
 * for every pair i <= j of samples that both hold x (i = j included, so the
 * diagonal gains |X_i restricted to the range|).  C is additive over any
 * partition of the values into ranges (Eq. 4), so the counts of a
 * collection too large for memory are the sum of calls over disjoint ranges.
 *
 * C is n*n row-major uint64; only the upper triangle (i <= j) is added to.
 * The range is cut into `pieces` equal stretches of values, processed by
 * threads in any order (each stretch's counts go into a thread-private
 * matrix, added into C at the end).  For one stretch: every (value, sample)
 * membership is listed, the list is sorted by value then sample (qsort),
 * repeated memberships (duplicate values inside a sample) are one, and each
 * run of equal values is one row a_x whose pairs are counted.
 * Returns 0, or -1 when a thread-private matrix cannot be allocated.
 */
typedef struct { uint64_t v; uint64_t s; } oracle_member;

static int oracle_member_cmp(const void* pa, const void* pb)
{
    const oracle_member* a = (const oracle_member*)pa;
    const oracle_member* b = (const oracle_member*)pb;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    if (a->s != b->s) return a->s < b->s ? -1 : 1;
    return 0;
}

/* first index k of sorted a[0..na) with a[k] >= x */
static uint64_t oracle_lower_bound(const uint64_t* a, uint64_t na, uint64_t x)
{
    uint64_t lo = 0, hi = na;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

int oracle_rows_range(uint64_t n, const uint64_t* offsets, const uint64_t* ids,
                      uint64_t lo, uint64_t hi, uint64_t pieces, uint64_t* C, int threads)
{
    if (hi <= lo || n == 0) return 0;
    if (pieces == 0) pieces = 1;
    if (pieces > hi - lo) pieces = hi - lo;
    int nt = threads > 0 ? threads : 1;
    int failed = 0;
    #pragma omp parallel num_threads(nt)
    {
        uint64_t* Cp = (uint64_t*)calloc(n * n, sizeof(uint64_t));
        if (!Cp) {
            #pragma omp atomic write
            failed = 1;
        }
        #pragma omp for schedule(dynamic, 1)
        for (int64_t pc = 0; pc < (int64_t)pieces; ++pc) {
            if (!Cp) continue;
            /* stretch [a, b) of the values; the last one ends at hi */
            uint64_t width = hi - lo;
            uint64_t a = lo + (uint64_t)(((unsigned __int128)width * (uint64_t)pc) / pieces);
            uint64_t b = lo + (uint64_t)(((unsigned __int128)width * (uint64_t)(pc + 1)) / pieces);
            uint64_t total = 0;
            for (uint64_t i = 0; i < n; ++i) {
                const uint64_t* s = ids + offsets[i];
                uint64_t ns = offsets[i + 1] - offsets[i];
                total += oracle_lower_bound(s, ns, b) - oracle_lower_bound(s, ns, a);
            }
            if (total == 0) continue;
            oracle_member* m = (oracle_member*)malloc(total * sizeof(oracle_member));
            if (!m) {
                #pragma omp atomic write
                failed = 1;
                continue;
            }
            uint64_t k = 0;
            for (uint64_t i = 0; i < n; ++i) {
                const uint64_t* s = ids + offsets[i];
                uint64_t ns = offsets[i + 1] - offsets[i];
                uint64_t e = oracle_lower_bound(s, ns, b);
                for (uint64_t t = oracle_lower_bound(s, ns, a); t < e; ++t) {
                    m[k].v = s[t];
                    m[k].s = i;
                    ++k;
                }
            }
            qsort(m, total, sizeof(oracle_member), oracle_member_cmp);
            /* drop repeated (value, sample) memberships: a set holds a value once */
            uint64_t u = 0;
            for (uint64_t t = 0; t < total; ++t)
                if (u == 0 || m[t].v != m[u - 1].v || m[t].s != m[u - 1].s) m[u++] = m[t];
            /* every run of equal values is one row a_x; add a_x a_x^T (i <= j) */
            for (uint64_t r = 0; r < u;) {
                uint64_t e = r;
                while (e < u && m[e].v == m[r].v) ++e;
                for (uint64_t p = r; p < e; ++p) {
                    uint64_t* row = Cp + m[p].s * n;
                    for (uint64_t q = p; q < e; ++q) row[m[q].s] += 1;
                }
                r = e;
            }
            free(m);
        }
        if (Cp) {
            #pragma omp critical
            {
                for (uint64_t i = 0; i < n; ++i)
                    for (uint64_t j = i; j < n; ++j) C[i * n + j] += Cp[i * n + j];
            }
            free(Cp);
        }
    }
    return failed ? -1 : 0;
}
