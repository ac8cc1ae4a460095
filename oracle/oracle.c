/*
 * oracle.c -- plain, slow, sequential CPU reference for the in-place
 * samplesort of Axtmann, Witt, Ferizovic and Sanders, "Engineering In-place
 * (Shared-memory) Sorting Algorithms" (IPS4o / IPS2Ra).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU library never
 * includes, links or calls it, and it shares no source with the GPU library.
 *
 * What it computes (each function below names the passage it follows):
 *   - oracle_classify: one classification level with given splitters.  The
 *     bucket of e is the i with s_{i-1} < e <= s_i (Sec. 2, "(Super Scalar)
 *     Samplesort"), found here by a plain binary search rather than the
 *     branchless tree.  With equality buckets the class is 2i + 1 - [e < s_i]
 *     on the splitter array padded to a power of two with its largest entry
 *     and the last splitter duplicated (Sec. 2, refined decision tree;
 *     Algorithm 1).
 *   - oracle_radix_classify: the IPS2Ra radix extractor, digit =
 *     (key >> shift) & (2^bits - 1) (Sec. 5, IPS2Ra paragraph).
 *   - oracle_partition: a stable out-of-place distribution by class, giving
 *     bucket boundaries (prefix sum of bucket sizes, Sec. 3.1.3).
 *   - oracle_sort: a recursive sequential samplesort following Sec. 3.1.1
 *     (sampling), Sec. 3.2 (base-case rule and adaptive k) and Sec. 5
 *     (parameters k = 256, alpha = 0.2 log2 n, n0 = 16, insertion-sort base
 *     case).  Because the sorted sequence of keys is unique, none of the
 *     sampling choices can change the resulting key sequence.
 *
 * Element types and their key order (Sec. 6, data types; Table of types):
 *   0 u32 (numeric), 1 u64 (numeric),
 *   2 f64: IEEE-754 bits b mapped to (b >> 63) ? ~b : b | 2^63 and compared
 *          as unsigned integers; on non-NaN values this is '<' refined so that
 *          -0.0 sorts before +0.0,
 *   3 pair: 16 bytes, key = first little-endian u64, value = second u64,
 *   4 rec100: 100 bytes, key = first 10 bytes compared lexicographically as
 *          unsigned bytes (the byte comparison of Sec. 6 with unsigned chars),
 *   5 quartet: 32 bytes, key = three little-endian u64 words (a, b, c)
 *          compared lexicographically: a first, b on a tie in a, c on a tie
 *          in both (the Quartet comparison of Sec. 6); value = fourth u64.
 *
 * Random sample positions come from splitmix64 (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014), written
 * here from its published definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { DT_U32 = 0, DT_U64 = 1, DT_F64 = 2, DT_PAIR = 3, DT_REC100 = 4, DT_QUARTET = 5 };

static size_t elem_size(int dt) {
    switch (dt) {
    case DT_U32: return 4;
    case DT_U64: return 8;
    case DT_F64: return 8;
    case DT_PAIR: return 16;
    case DT_REC100: return 100;
    case DT_QUARTET: return 32;
    default: return 0;
    }
}

int oracle_elem_size(int dt) { return (int)elem_size(dt); }

/* ---- key order --------------------------------------------------------- */

static uint64_t load_u64(const unsigned char *p) {
    uint64_t x;
    memcpy(&x, p, 8);
    return x;
}

static uint64_t f64_order_bits(uint64_t b) {
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

/* returns 1 if key(a) < key(b) */
static int key_less(int dt, const unsigned char *a, const unsigned char *b) {
    switch (dt) {
    case DT_U32: {
        uint32_t x, y;
        memcpy(&x, a, 4);
        memcpy(&y, b, 4);
        return x < y;
    }
    case DT_U64:
    case DT_PAIR:
        return load_u64(a) < load_u64(b);
    case DT_F64:
        return f64_order_bits(load_u64(a)) < f64_order_bits(load_u64(b));
    case DT_REC100:
        return memcmp(a, b, 10) < 0;
    case DT_QUARTET:
        for (int w = 0; w < 3; w++) {
            uint64_t x = load_u64(a + 8 * w), y = load_u64(b + 8 * w);
            if (x != y) return x < y;
        }
        return 0;
    }
    return 0;
}

/* unsigned integer key for the radix extractor (u32, u64, pair only) */
static uint64_t radix_key(int dt, const unsigned char *a) {
    if (dt == DT_U32) {
        uint32_t x;
        memcpy(&x, a, 4);
        return x;
    }
    return load_u64(a);
}

/* ---- splitmix64 -------------------------------------------------------- */

static uint64_t splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ---- one classification level ----------------------------------------- */

/* smallest power of two >= x (x >= 1) */
static uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

/*
 * Classify n elements against m sorted splitters (elements of the same type,
 * only their keys are read).  K = 2^ceil(log2(m+1)); the splitter array is
 * padded to K entries with the largest splitter, so s_{K-1} = s_{K-2} (Sec. 2).
 * Without equality buckets class(e) = i, the smallest i in [0, K-1) with
 * e <= s_i, or K-1 if e is larger than every splitter; with equality buckets
 * class(e) = 2i + 1 - [e < s_i] (Algorithm 1, final step).
 * Writes class ids to cls[n]; returns the number of classes B (K or 2K), or
 * 0 if m == 0.
 */
static uint32_t classify_impl(int dt, const unsigned char *a, uint64_t n,
                              const unsigned char *spl, uint32_t m, int eq,
                              uint32_t *cls) {
    size_t D = elem_size(dt);
    if (m == 0) return 0;
    uint64_t K = next_pow2((uint64_t)m + 1);
    /* padded[j] = s_min(j, m-1) for j in [0, K) */
    for (uint64_t e = 0; e < n; e++) {
        const unsigned char *x = a + e * D;
        /* binary search over s_0 .. s_{K-2}: number of splitters < x */
        uint64_t lo = 0, hi = K - 1;
        while (lo < hi) {
            uint64_t mid = (lo + hi) / 2;
            uint64_t j = mid < m ? mid : m - 1;
            if (key_less(dt, spl + j * D, x))
                lo = mid + 1;
            else
                hi = mid;
        }
        uint64_t i = lo;
        if (eq) {
            uint64_t j = i < m ? i : m - 1; /* padded s_i, incl. s_{K-1} */
            cls[e] = (uint32_t)(2 * i + 1 - (uint64_t)key_less(dt, x, spl + j * D));
        } else {
            cls[e] = (uint32_t)i;
        }
    }
    return (uint32_t)(eq ? 2 * K : K);
}

uint32_t oracle_classify(int dt, const void *a, uint64_t n, const void *spl,
                         uint32_t m, int eq, uint32_t *cls) {
    return classify_impl(dt, (const unsigned char *)a, n,
                         (const unsigned char *)spl, m, eq, cls);
}

/* IPS2Ra radix extractor (Sec. 5): class = (key >> shift) & (2^bits - 1). */
uint32_t oracle_radix_classify(int dt, const void *a, uint64_t n, uint32_t shift,
                               uint32_t bits, uint32_t *cls) {
    const unsigned char *p = (const unsigned char *)a;
    size_t D = elem_size(dt);
    uint64_t mask = (bits >= 64) ? ~0ULL : ((1ULL << bits) - 1);
    for (uint64_t e = 0; e < n; e++) {
        uint64_t k = radix_key(dt, p + e * D);
        cls[e] = (uint32_t)((shift >= 64 ? 0 : (k >> shift)) & mask);
    }
    return (uint32_t)(1ULL << bits);
}

/*
 * Stable out-of-place distribution of a[n] by cls[] into out[n];
 * bucket_begin[j] = number of elements with class < j, j = 0..B
 * (the prefix sum over bucket sizes of Sec. 3.1.3).
 */
void oracle_partition(int dt, const void *a, uint64_t n, const uint32_t *cls,
                      uint32_t B, void *out, uint64_t *bucket_begin) {
    size_t D = elem_size(dt);
    const unsigned char *src = (const unsigned char *)a;
    unsigned char *dst = (unsigned char *)out;
    for (uint32_t j = 0; j <= B; j++) bucket_begin[j] = 0;
    for (uint64_t e = 0; e < n; e++) bucket_begin[cls[e] + 1]++;
    for (uint32_t j = 0; j < B; j++) bucket_begin[j + 1] += bucket_begin[j];
    uint64_t *pos = (uint64_t *)malloc(sizeof(uint64_t) * (B ? B : 1));
    for (uint32_t j = 0; j < B; j++) pos[j] = bucket_begin[j];
    for (uint64_t e = 0; e < n; e++) memcpy(dst + (pos[cls[e]]++) * D, src + e * D, D);
    free(pos);
}

/* ---- sequential samplesort --------------------------------------------- */

typedef struct {
    int dt;
    size_t D;
    uint32_t k;          /* maximum number of buckets, 256 in Sec. 5 */
    uint32_t n0;         /* base-case size, 16 in Sec. 5 */
    double alpha_scale;  /* alpha = alpha_scale * log2(n'), 0.2 in Sec. 5 */
    uint64_t rng;        /* splitmix64 state */
    unsigned char *tmp;  /* n elements: distribution target */
    unsigned char *swap; /* one element */
} sort_ctx;

static void insertion_sort(sort_ctx *c, unsigned char *a, uint64_t n) {
    size_t D = c->D;
    for (uint64_t i = 1; i < n; i++) {
        memcpy(c->swap, a + i * D, D);
        uint64_t j = i;
        while (j > 0 && key_less(c->dt, c->swap, a + (j - 1) * D)) {
            memcpy(a + j * D, a + (j - 1) * D, D);
            j--;
        }
        memcpy(a + j * D, c->swap, D);
    }
}

/* number of buckets for a task of n elements: the adaptive rule of Sec. 3.2 */
static uint32_t buckets_for(const sort_ctx *c, uint64_t n) {
    double r = (double)n / (double)c->n0;
    if (n <= (uint64_t)c->k * c->n0) {           /* n0 < n' <= k n0 */
        uint32_t l = (uint32_t)ceil(log2(r));
        return 1u << (l < 1 ? 1 : l);
    }
    if ((double)n < (double)c->k * c->k * c->n0) { /* k n0 < n' < k^2 n0 */
        uint32_t l = (uint32_t)ceil((log2(r) + 1.0) / 2.0);
        uint32_t kk = 1u << l;
        return kk > c->k ? c->k : kk;
    }
    return c->k;
}

static void sort_task(sort_ctx *c, unsigned char *a, uint64_t n, uint64_t parent_n);

/* One sequential partitioning step (Sec. 3.1) on a[0..n), then recursion. */
static void partition_and_recurse(sort_ctx *c, unsigned char *a, uint64_t n) {
    size_t D = c->D;
    uint32_t k = buckets_for(c, n);

    /* Sec. 3.1.1 step 1: sample k*alpha elements (with replacement) */
    double alpha = c->alpha_scale * log2((double)n);
    if (alpha < 1.0) alpha = 1.0;
    uint64_t m = (uint64_t)(alpha * k);
    if (m < k - 1) m = k - 1;
    unsigned char *sample = (unsigned char *)malloc(m * D);
    for (uint64_t t = 0; t < m; t++) {
        uint64_t pos = splitmix64_next(&c->rng) % n;
        memcpy(sample + t * D, a + pos * D, D);
    }
    insertion_sort(c, sample, m);

    /* step 2: k-1 equidistant splitters from the sorted sample */
    unsigned char *spl = (unsigned char *)malloc((size_t)(k - 1) * D);
    for (uint32_t j = 0; j + 1 < k; j++)
        memcpy(spl + (size_t)j * D, sample + (((uint64_t)(j + 1) * m) / k - 1) * D, D);

    /* step 3: remove duplicate splitters; equality buckets iff any existed */
    uint32_t distinct = 0;
    for (uint32_t j = 0; j + 1 < k; j++) {
        if (distinct == 0 || key_less(c->dt, spl + (size_t)(distinct - 1) * D, spl + (size_t)j * D)) {
            if (distinct != j) memcpy(spl + (size_t)distinct * D, spl + (size_t)j * D, D);
            distinct++;
        }
    }
    int eq = distinct < k - 1;

    /* classification and distribution */
    uint32_t *cls = (uint32_t *)malloc(sizeof(uint32_t) * n);
    uint32_t B = classify_impl(c->dt, a, n, spl, distinct, eq, cls);
    uint64_t *bb = (uint64_t *)malloc(sizeof(uint64_t) * (B + 1));
    oracle_partition(c->dt, a, n, cls, B, c->tmp, bb);
    memcpy(a, c->tmp, n * D);
    free(cls);
    free(spl);
    free(sample);

    /* recursion; equality buckets 2i+1 (i < K-1) hold one key only and are
     * finished.  The last class 2K-1 is odd too but holds every element above
     * the largest splitter, so it is recursed like the others. */
    for (uint32_t j = 0; j < B; j++) {
        if (eq && (j & 1) && j + 1 < B) continue;
        sort_task(c, a + bb[j] * D, bb[j + 1] - bb[j], n);
    }
    free(bb);
}

static void sort_task(sort_ctx *c, unsigned char *a, uint64_t n, uint64_t parent_n) {
    /* base case rule of Sec. 3.2: at most 2 n0 elements, or a parent task
     * with at most k n0 elements */
    if (n <= 2ULL * c->n0 || parent_n <= (uint64_t)c->k * c->n0) {
        insertion_sort(c, a, n);
        return;
    }
    partition_and_recurse(c, a, n);
}

/*
 * Sort a[n] in place.  k, n0 and alpha_scale default to 256, 16 and 0.2
 * (Sec. 5) when passed as 0.  Returns 0 on success, -1 on bad arguments.
 */
int oracle_sort(int dt, void *a, uint64_t n, uint32_t k, uint32_t n0,
                double alpha_scale, uint64_t seed) {
    sort_ctx c;
    c.dt = dt;
    c.D = elem_size(dt);
    if (c.D == 0) return -1;
    c.k = k ? k : 256;
    c.n0 = n0 ? n0 : 16;
    c.alpha_scale = alpha_scale > 0 ? alpha_scale : 0.2;
    /* k >= 4 guarantees progress: with a single splitter and no equality
     * buckets every element could fall into one bucket */
    if (c.k < 4 || (c.k & (c.k - 1))) return -1;
    c.rng = seed;
    if (n < 2) return 0;
    c.tmp = (unsigned char *)malloc(n * c.D);
    c.swap = (unsigned char *)malloc(c.D);
    if (!c.tmp || !c.swap) {
        free(c.tmp);
        free(c.swap);
        return -1;
    }
    /* the top-level task has no parent: treat it as a large one */
    sort_task(&c, (unsigned char *)a, n, ~0ULL);
    free(c.tmp);
    free(c.swap);
    return 0;
}

/* Insertion sort alone, the base-case algorithm of Sec. 5 (used by the
 * brute-force pins). */
int oracle_insertion_sort(int dt, void *a, uint64_t n) {
    sort_ctx c;
    c.dt = dt;
    c.D = elem_size(dt);
    if (c.D == 0) return -1;
    c.swap = (unsigned char *)malloc(c.D);
    insertion_sort(&c, (unsigned char *)a, n);
    free(c.swap);
    return 0;
}

/* 1 if a[0..n) is non-decreasing in the key order */
int oracle_is_sorted(int dt, const void *a, uint64_t n) {
    size_t D = elem_size(dt);
    const unsigned char *p = (const unsigned char *)a;
    for (uint64_t i = 1; i < n; i++)
        if (key_less(dt, p + i * D, p + (i - 1) * D)) return 0;
    return 1;
}
