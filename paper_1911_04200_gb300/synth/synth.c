/*
 * Seeded synthetic sample collections (sorted, distinct uint64 values per
 * sample).  This module holds none of the similarity method's arithmetic: it
 * only draws sets.  Both the CUDA path's tests and the CPU oracle's tests take
 * their inputs from here.
 *
 * Every random number is a counter-based hash (the splitmix64 finaliser of
 * Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) of (seed, stream tag, indices), so the output depends only on
 * the parameters, not on thread count or machine.  Floating point uses only
 * +, -, *, / and comparisons in binary64 (no libm), built with
 * -ffp-contract=off, so x86-64 and AArch64 draw identical sets.
 *
 * Two models:
 *
 *  ANCESTRAL (kind 0): A ancestors, each `anc_size` distinct uniform values in
 *    [0, 2^id_bits).  Sample i copies ancestor i mod A and replaces
 *    floor(u_i * anc_size) of its positions (u_i uniform in [0, u_max)) by
 *    fresh uniform values; then sort + dedupe.
 *
 *  CLADE (kind 1): a root stream rho(t); clade c's stream is rho(t) where a
 *    per-(c,t) draw is below `core` and a clade-private value otherwise.
 *    Sample i (clade i mod n_clades) takes the clade stream at t < s_i except
 *    where a per-(i,t) draw falls below u_i (u_i uniform in [0, u_max)), which
 *    gets a fresh value.  s_i is log-normal with median `median`, shape sigma,
 *    truncated to [lo, hi] by resampling.  Values are hash >> (64 - id_bits).
 *    Then sort + dedupe.  `sample_base` offsets the sample index so that query
 *    sets can be drawn from the same clades as a reference collection.
 *
 *  BERNOULLI (kind 2): every value t of [0, m) is in sample i independently
 *    with probability p (the synthetic indicator matrices of the paper's
 *    evaluation, Sec. V-A).  Drawn as geometric gaps: the next member after
 *    t is t + 1 + floor(log(U) / log(1 - p)), U uniform in (0, 1].  Sorted and
 *    distinct by construction.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t H3(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b)
{
    return mix64(mix64(mix64(seed ^ (tag * 0xD1B54A32D192ED03ull)) ^ a) + b);
}

/* uniform in [0,1) with 53 bits */
static inline double U01(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

static inline uint64_t to_domain(uint64_t h, int id_bits)
{
    return id_bits >= 64 ? h : (h >> (64 - id_bits));
}

enum { T_ANC = 1, T_U = 2, T_PERM = 3, T_NEW = 4, T_ROOT = 5, T_CORE = 6, T_CLADE = 7,
       T_SUB = 8, T_FRESH = 9, T_SIZE = 10, T_BERN = 11 };

/* exp(x) for |x| <= 40 from +,*,/ only: x = k*ln2/64 ... computed as
 * (1 + y + y^2/2 + ... ) ^ (2^s) with y = x / 2^s, |y| < 2^-10, 12 terms.
 * Deterministic; accurate to a few ulp, which is all a set-size draw needs. */
static double det_exp(double x)
{
    int s = 0;
    double y = x;
    while (y > 0.0009765625 || y < -0.0009765625) { y *= 0.5; ++s; }
    double term = 1.0, sum = 1.0;
    for (int k = 1; k <= 12; ++k) { term = term * y / (double)k; sum += term; }
    for (int k = 0; k < s; ++k) sum = sum * sum;
    return sum;
}

/* log(x) for x in (0, 1] from +,*,/ only: x = f * 2^-e with f in [0.5, 1),
 * log f = 2 atanh(z), z = (f - 1) / (f + 1) in [-1/3, 0), summed to z^41
 * (error below 3^-41).  Deterministic; a gap draw needs no more. */
static double det_log01(double x)
{
    int e = 0;
    while (x < 0.5) { x *= 2.0; ++e; }
    double z = (x - 1.0) / (x + 1.0), z2 = z * z, term = z, sum = 0.0;
    for (int k = 1; k <= 41; k += 2) { sum += term / (double)k; term *= z2; }
    return 2.0 * sum - (double)e * 0.6931471805599453;
}

/* standard normal deviate, Irwin-Hall sum of 12 uniforms minus 6 */
static double normal12(uint64_t seed, uint64_t a, uint64_t b)
{
    double z = -6.0;
    for (int k = 0; k < 12; ++k) z += U01(H3(seed, T_SIZE, a, b * 16 + (uint64_t)k));
    return z;
}

typedef struct {
    int kind;            /* 0 ancestral, 1 clade */
    int id_bits;         /* values in [0, 2^id_bits) */
    uint64_t seed;
    uint64_t n;          /* samples */
    uint64_t sample_base;/* offset of sample indices (clade model) */
    /* ancestral */
    uint64_t n_anc, anc_size;
    /* clade */
    uint64_t n_clades;
    double core, u_max;
    double median, sigma, lo, hi;
    /* bernoulli */
    uint64_t m;
    double p;
} synth_params;

static uint64_t sample_len(const synth_params* p, uint64_t i)
{
    if (p->kind == 0) return p->anc_size;
    if (p->kind == 2) {
        /* slot: mean + 12 standard deviations + 64 of Binomial(m, p); the
           draw stops at the slot's end (never reached in practice) */
        double mu = (double)p->m * p->p, var = mu * (1.0 - p->p), sd = 1.0;
        for (int k = 0; k < 60; ++k) sd = 0.5 * (sd + var / sd);  /* sqrt by Newton */
        double L = mu + 12.0 * sd + 64.0;
        return L > (double)p->m ? p->m : (uint64_t)L;
    }
    uint64_t gi = i + p->sample_base;
    double lm = p->median;
    for (uint64_t attempt = 0; attempt < 1000; ++attempt) {
        double z = normal12(p->seed, gi, attempt);
        double s = lm * det_exp(p->sigma * z);
        if (s >= p->lo && s <= p->hi) return (uint64_t)s;
    }
    return (uint64_t)lm;
}

/* pre-dedupe length of each sample */
void synth_lengths(const synth_params* p, uint64_t* len)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)p->n; ++i) len[i] = sample_len(p, (uint64_t)i);
}

/* LSD radix sort of v[0..n) on the low `bits` bits, 8 bits per pass */
static void radix_sort(uint64_t* v, uint64_t n, int bits, uint64_t* tmp)
{
    uint64_t* a = v; uint64_t* b = tmp;
    for (int sh = 0; sh < bits; sh += 8) {
        uint64_t cnt[256];
        memset(cnt, 0, sizeof cnt);
        for (uint64_t k = 0; k < n; ++k) cnt[(a[k] >> sh) & 255]++;
        uint64_t s = 0;
        for (int d = 0; d < 256; ++d) { uint64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (uint64_t k = 0; k < n; ++k) b[cnt[(a[k] >> sh) & 255]++] = a[k];
        uint64_t* t = a; a = b; b = t;
    }
    if (a != v) memcpy(v, a, n * sizeof(uint64_t));
}

static uint64_t sort_unique(uint64_t* v, uint64_t n, int bits, uint64_t* tmp)
{
    if (n == 0) return 0;
    radix_sort(v, n, bits, tmp);
    uint64_t k = 1;
    for (uint64_t t = 1; t < n; ++t) if (v[t] != v[k - 1]) v[k++] = v[t];
    return k;
}

/* ancestor a: anc_size distinct uniform values (drawn in order until distinct) */
static void make_ancestor(const synth_params* p, uint64_t a, uint64_t* out, uint64_t* tmp)
{
    uint64_t want = p->anc_size, have = 0, t = 0;
    /* draw, sort-unique, top up until exactly `want` distinct values exist;
       the final set is the first `want` distinct values in draw order */
    uint64_t* draw = (uint64_t*)malloc(sizeof(uint64_t) * (want * 2 + 64));
    uint64_t* srt = (uint64_t*)malloc(sizeof(uint64_t) * (want * 2 + 64));
    uint64_t* tt = (uint64_t*)malloc(sizeof(uint64_t) * (want * 2 + 64));
    uint64_t nd = 0;
    while (have < want && nd < want * 2 + 64) {
        draw[nd++] = to_domain(H3(p->seed, T_ANC, a, t++), p->id_bits);
        if (nd % 1024 == 0 || nd >= want) {
            memcpy(srt, draw, nd * sizeof(uint64_t));
            have = sort_unique(srt, nd, p->id_bits, tt);
        }
    }
    /* keep first `want` distinct in draw order */
    memcpy(srt, draw, nd * sizeof(uint64_t));
    (void)sort_unique(srt, nd, p->id_bits, tt);
    /* mark which draws are first occurrences: walk draws, binary-search the
       sorted distinct list and a seen-bitmap over it */
    uint8_t* seen = (uint8_t*)calloc(have ? have : 1, 1);
    uint64_t k = 0;
    for (uint64_t d = 0; d < nd && k < want; ++d) {
        uint64_t x = draw[d], lo = 0, hi = have;
        while (lo < hi) { uint64_t mid = (lo + hi) / 2; if (srt[mid] < x) lo = mid + 1; else hi = mid; }
        if (!seen[lo]) { seen[lo] = 1; out[k++] = x; }
    }
    while (k < want) out[k++] = 0; /* unreachable for sane parameters */
    free(seen); free(draw); free(srt); free(tt);
    (void)tmp;
}

/*
 * Draw sample i into v[0..L) (L = its pre-dedupe length from synth_lengths)
 * and return the number of distinct values, which are then the sorted prefix
 * of v.  tmp and perm hold L entries each; anc holds the ancestors (kind 0).
 */
static uint64_t draw_sample(const synth_params* p, const uint64_t* anc, uint64_t i, uint64_t L,
                            uint64_t* v, uint64_t* tmp, uint64_t* perm)
{
    if (p->kind == 2) {
        uint64_t k = 0;
        if (p->p >= 1.0) {
            for (; k < L; ++k) v[k] = k;
        } else if (p->p > 0.0) {
            const double lq = det_log01(1.0 - p->p);
            uint64_t t = 0;
            for (uint64_t d = 0; k < L; ++d) {
                const double u = 1.0 - U01(H3(p->seed, T_BERN, i + p->sample_base, d));
                const double g = det_log01(u) / lq;
                if (g >= (double)(p->m - t)) break;
                t += (uint64_t)g;
                if (t >= p->m) break;
                v[k++] = t++;
            }
        }
        return k;
    }
    if (p->kind == 0) {
        const uint64_t* A = anc + (i % p->n_anc) * p->anc_size;
        memcpy(v, A, L * sizeof(uint64_t));
        double u = p->u_max * U01(H3(p->seed, T_U, i, 0));
        uint64_t k = (uint64_t)(u * (double)L);
        /* partial Fisher-Yates over positions: the first k are replaced */
        for (uint64_t t = 0; t < L; ++t) perm[t] = t;
        for (uint64_t t = 0; t < k; ++t) {
            uint64_t r = t + H3(p->seed, T_PERM, i, t) % (L - t);
            uint64_t x = perm[t]; perm[t] = perm[r]; perm[r] = x;
        }
        for (uint64_t t = 0; t < k; ++t)
            v[perm[t]] = to_domain(H3(p->seed, T_NEW, i, perm[t]), p->id_bits);
    } else {
        uint64_t gi = i + p->sample_base;
        uint64_t c = gi % p->n_clades;
        double u = p->u_max * U01(H3(p->seed, T_U, gi, 0));
        for (uint64_t t = 0; t < L; ++t) {
            uint64_t h;
            if (U01(H3(p->seed, T_SUB, gi, t)) < u) {
                h = H3(p->seed, T_FRESH, gi, t);
            } else if (U01(H3(p->seed, T_CORE, c, t)) < p->core) {
                h = H3(p->seed, T_ROOT, 0, t);
            } else {
                h = H3(p->seed, T_CLADE, c, t);
            }
            v[t] = to_domain(h, p->id_bits);
        }
    }
    return sort_unique(v, L, p->id_bits, tmp);
}

static uint64_t* make_ancestors(const synth_params* p)
{
    if (p->kind != 0) return NULL;
    uint64_t* anc = (uint64_t*)malloc(sizeof(uint64_t) * p->n_anc * p->anc_size + 8);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < (int64_t)p->n_anc; ++a)
        make_ancestor(p, (uint64_t)a, anc + (uint64_t)a * p->anc_size, NULL);
    return anc;
}

/*
 * Fill sample slots.  slot[i] .. slot[i+1] is sample i's slot of length
 * len[i] (from synth_lengths).  On return the first distinct[i] entries of
 * the slot are the sample's sorted distinct values.
 */
void synth_fill(const synth_params* p, const uint64_t* slot, uint64_t* ids, uint64_t* distinct)
{
    uint64_t* anc = make_ancestors(p);
    #pragma omp parallel
    {
        uint64_t cap = 0;
        uint64_t* tmp = NULL;
        uint64_t* perm = NULL;
        #pragma omp for schedule(dynamic, 1)
        for (int64_t ii = 0; ii < (int64_t)p->n; ++ii) {
            uint64_t i = (uint64_t)ii;
            uint64_t L = slot[i + 1] - slot[i];
            if (L > cap) {
                free(tmp); free(perm);
                cap = L;
                tmp = (uint64_t*)malloc(sizeof(uint64_t) * cap);
                perm = (uint64_t*)malloc(sizeof(uint64_t) * cap);
            }
            distinct[i] = draw_sample(p, anc, i, L, ids + slot[i], tmp, perm);
        }
        free(tmp); free(perm);
    }
    free(anc);
}

static uint64_t first_at_least(const uint64_t* v, uint64_t n, uint64_t x)
{
    uint64_t a = 0, b = n;
    while (a < b) { uint64_t mid = a + (b - a) / 2; if (v[mid] < x) a = mid + 1; else b = mid; }
    return a;
}

/*
 * The same collection restricted to the values of [lo, hi): every sample is
 * drawn whole (as synth_fill draws it) and only its values inside the range
 * are kept, so the restrictions of a collection to disjoint ranges are
 * exactly the pieces of the whole.  With ids == NULL, counts[i] receives the
 * number of sample i's values inside the range; otherwise ids receives them,
 * sample i's at slot[i] (slot[i+1] - slot[i] = counts[i] from the first
 * call).  len[i] is the pre-dedupe length from synth_lengths.
 */
void synth_fill_range(const synth_params* p, const uint64_t* len, uint64_t lo, uint64_t hi,
                      uint64_t* counts, const uint64_t* slot, uint64_t* ids)
{
    uint64_t* anc = make_ancestors(p);
    #pragma omp parallel
    {
        uint64_t cap = 0;
        uint64_t* v = NULL;
        uint64_t* tmp = NULL;
        uint64_t* perm = NULL;
        #pragma omp for schedule(dynamic, 1)
        for (int64_t ii = 0; ii < (int64_t)p->n; ++ii) {
            uint64_t i = (uint64_t)ii;
            uint64_t L = len[i];
            if (L > cap) {
                free(v); free(tmp); free(perm);
                cap = L;
                v = (uint64_t*)malloc(sizeof(uint64_t) * cap);
                tmp = (uint64_t*)malloc(sizeof(uint64_t) * cap);
                perm = (uint64_t*)malloc(sizeof(uint64_t) * cap);
            }
            uint64_t d = draw_sample(p, anc, i, L, v, tmp, perm);
            uint64_t a = first_at_least(v, d, lo), b = hi > lo ? first_at_least(v, d, hi) : a;
            if (!ids) counts[i] = b - a;
            else memcpy(ids + slot[i], v + a, (b - a) * sizeof(uint64_t));
        }
        free(v); free(tmp); free(perm);
    }
    free(anc);
}

/*
 * Compact the sorted distinct prefixes of the slots to the front, in sample
 * order, and write the final offsets (n+1).  Returns the total value count.
 */
uint64_t synth_compact(uint64_t n, const uint64_t* slot, const uint64_t* distinct,
                       uint64_t* ids, uint64_t* offsets)
{
    uint64_t o = 0;
    for (uint64_t i = 0; i < n; ++i) {
        offsets[i] = o;
        if (o != slot[i]) memmove(ids + o, ids + slot[i], distinct[i] * sizeof(uint64_t));
        o += distinct[i];
    }
    offsets[n] = o;
    return o;
}

/*
 * Workload statistics (not part of any result): number of distinct values of
 * the whole collection inside each aligned range [r * 2^range_bits,
 * (r+1) * 2^range_bits) for r < nranges, written to counts[r].  Used only to
 * state how much dense packed work a batch plan implies.  Values must be
 * below nranges * 2^range_bits.  One bit per value of the domain is set in a
 * scratch bitmap (domain_bits <= 36), partitioned by range across threads.
 */
int synth_range_distinct(uint64_t n_values, const uint64_t* ids, int range_bits, uint64_t nranges,
                         uint64_t* counts)
{
    uint64_t domain = nranges << range_bits;
    if (range_bits < 6 || domain == 0 || domain > (1ull << 36)) return -1;
    uint64_t nw = domain / 64;
    uint64_t* bm = (uint64_t*)calloc(nw, sizeof(uint64_t));
    if (!bm) return -2;
    int bad = 0;
    #pragma omp parallel
    {
        /* every thread owns a contiguous stripe of the bitmap words */
        int nt = 1, t = 0;
#ifdef _OPENMP
        nt = omp_get_num_threads(); t = omp_get_thread_num();
#endif
        uint64_t w0 = nw * (uint64_t)t / (uint64_t)nt, w1 = nw * (uint64_t)(t + 1) / (uint64_t)nt;
        for (uint64_t k = 0; k < n_values; ++k) {
            uint64_t x = ids[k];
            if (x >= domain) { bad = 1; continue; }
            uint64_t w = x >> 6;
            if (w >= w0 && w < w1) bm[w] |= 1ull << (x & 63);
        }
    }
    uint64_t per = (1ull << range_bits) / 64;
    for (uint64_t r = 0; r < nranges; ++r) {
        uint64_t c = 0;
        for (uint64_t w = r * per; w < (r + 1) * per; ++w) c += (uint64_t)__builtin_popcountll(bm[w]);
        counts[r] = c;
    }
    free(bm);
    return bad ? -3 : 0;
}
