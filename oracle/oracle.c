/*
 * Plain CPU oracle for the small-set sorters of Bingmann, Marianczuk and
 * Sanders, "Engineering Faster Sorters for Small Sets of Items".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm load this library.  It shares no
 * code, header, table or helper with the CUDA library; it is deliberately
 * slow and written to be checked against the paper by eye.
 *
 * What it computes (all integer, exact):
 *   - fixed-size arrays sorted ascending in place: the definition of a sorting
 *     network's result (Sec. 2.1: "a permutation of the original input" in
 *     "non-decreasing order"), computed by the paper's textbook insertion sort
 *     baseline "IS Def" (Sec. 4.2);
 *   - CSR segments sorted ascending with ties kept in their original order
 *     (a stable sort), payloads permuted alongside.  Items carry a reference
 *     value (Sec. 2.2.1, SortableRef); ordering by (key, original position)
 *     is this library's reading for making key-value output unique;
 *   - network checks: comparator semantics of Sec. 2.1 (the lower channel
 *     receives the smaller value), 0-1 inputs (Knuth's 0-1 principle; not
 *     stated in the paper), all permutations, size and depth (Sec. 2.1);
 *   - the paper's probabilistic permutation check (Sec. 4.1,
 *     "Checking Results: Permutation Check").
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stddef.h>

/* ---- Sorting: insertion sort "IS Def" (Sec. 4.2, textbook, array indices) ---- */

/* Sort `count` contiguous arrays of `n` u32 keys each, ascending, in place. */
void oracle_sort_fixed_u32(uint32_t *keys, int n, uint64_t count)
{
    for (uint64_t a = 0; a < count; ++a) {
        uint32_t *A = keys + a * (uint64_t)n;
        for (int i = 1; i < n; ++i) {
            uint32_t x = A[i];
            int j = i - 1;
            while (j >= 0 && A[j] > x) {
                A[j + 1] = A[j];
                --j;
            }
            A[j + 1] = x;
        }
    }
}

void oracle_sort_fixed_u64(uint64_t *keys, int n, uint64_t count)
{
    for (uint64_t a = 0; a < count; ++a) {
        uint64_t *A = keys + a * (uint64_t)n;
        for (int i = 1; i < n; ++i) {
            uint64_t x = A[i];
            int j = i - 1;
            while (j >= 0 && A[j] > x) {
                A[j + 1] = A[j];
                --j;
            }
            A[j + 1] = x;
        }
    }
}

/*
 * The 16-byte items of the paper's experiments (Sec. 4.1: a 64-bit key and a
 * 64-bit reference), `count` arrays of n items stored as key, ref, key, ref,
 * ...  Each array is sorted by key with insertion sort; the reference moves
 * with its key and equal keys keep their input order.
 */
void oracle_sort_fixed_items(uint64_t *items, int n, uint64_t count)
{
    for (uint64_t a = 0; a < count; ++a) {
        uint64_t *A = items + 2 * a * (uint64_t)n;
        for (int i = 1; i < n; ++i) {
            uint64_t key = A[2 * i], ref = A[2 * i + 1];
            int j = i - 1;
            while (j >= 0 && A[2 * j] > key) {
                A[2 * (j + 1)] = A[2 * j];
                A[2 * (j + 1) + 1] = A[2 * j + 1];
                --j;
            }
            A[2 * (j + 1)] = key;
            A[2 * (j + 1) + 1] = ref;
        }
    }
}

/*
 * Segment i is keys[offsets[i] .. offsets[i+1]).  Each segment is sorted by
 * key; equal keys keep their input order because insertion sort only moves
 * an element past strictly greater ones.  If vals != NULL, vals[] is permuted
 * exactly like keys[].  Offsets are assumed valid (non-decreasing).
 */
void oracle_sort_segments_u32(uint32_t *keys, uint32_t *vals,
                              const uint32_t *offsets, uint64_t nseg)
{
    for (uint64_t s = 0; s < nseg; ++s) {
        uint32_t *A = keys + offsets[s];
        uint32_t *V = vals ? vals + offsets[s] : NULL;
        int64_t len = (int64_t)offsets[s + 1] - (int64_t)offsets[s];
        for (int64_t i = 1; i < len; ++i) {
            uint32_t x = A[i];
            uint32_t v = V ? V[i] : 0;
            int64_t j = i - 1;
            while (j >= 0 && A[j] > x) {
                A[j + 1] = A[j];
                if (V) V[j + 1] = V[j];
                --j;
            }
            A[j + 1] = x;
            if (V) V[j + 1] = v;
        }
    }
}

void oracle_sort_segments_u64(uint64_t *keys, uint32_t *vals,
                              const uint32_t *offsets, uint64_t nseg)
{
    for (uint64_t s = 0; s < nseg; ++s) {
        uint64_t *A = keys + offsets[s];
        uint32_t *V = vals ? vals + offsets[s] : NULL;
        int64_t len = (int64_t)offsets[s + 1] - (int64_t)offsets[s];
        for (int64_t i = 1; i < len; ++i) {
            uint64_t x = A[i];
            uint32_t v = V ? V[i] : 0;
            int64_t j = i - 1;
            while (j >= 0 && A[j] > x) {
                A[j + 1] = A[j];
                if (V) V[j + 1] = V[j];
                --j;
            }
            A[j + 1] = x;
            if (V) V[j + 1] = v;
        }
    }
}

/*
 * One array of n u32 keys sorted ascending by a bottom-up merge sort (runs of
 * width 1, 2, 4, ... merged pairwise into a second buffer).  `tmp` holds n
 * keys of scratch.  For the large-array sort, where insertion sort would take
 * too long.
 */
void oracle_sort_array_u32(uint32_t *keys, uint32_t *tmp, uint64_t n)
{
    uint32_t *src = keys, *dst = tmp;
    for (uint64_t w = 1; w < n; w *= 2) {
        for (uint64_t lo = 0; lo < n; lo += 2 * w) {
            uint64_t mid = lo + w < n ? lo + w : n;
            uint64_t hi = lo + 2 * w < n ? lo + 2 * w : n;
            uint64_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi) dst[o++] = (src[j] < src[i]) ? src[j++] : src[i++];
            while (i < mid) dst[o++] = src[i++];
            while (j < hi) dst[o++] = src[j++];
        }
        uint32_t *t = src;
        src = dst;
        dst = t;
    }
    if (src != keys)
        for (uint64_t i = 0; i < n; ++i) keys[i] = src[i];
}

/* ---- Floating-point keys: IEEE 754 totalOrder ---- */

/*
 * greater(a, b): a follows b in the totalOrder of IEEE 754 (Sec. 5.10 of the
 * standard), written case by case from its definition rather than from a
 * bit encoding:
 *   - numbers (and infinities) compare by value;
 *   - -0 precedes +0;
 *   - a NaN with the sign bit set precedes every non-NaN, one without it
 *     follows every non-NaN;
 *   - two NaNs of the same sign: for positive NaNs the smaller payload (the
 *     bits below the sign) comes first, for negative NaNs the larger.
 * Identical bit patterns are not greater than each other.
 */
static int nan_class(int isnan_, int neg)
{
    return isnan_ ? (neg ? -1 : 1) : 0;
}

static int greater_f64(double a, double b)
{
    int ca = nan_class(isnan(a), signbit(a) != 0), cb = nan_class(isnan(b), signbit(b) != 0);
    if (ca != cb) return ca > cb;
    if (ca == 0) {
        if (a != b) return a > b;
        return (signbit(a) == 0) && (signbit(b) != 0); /* +0 after -0 */
    }
    uint64_t pa, pb;
    memcpy(&pa, &a, 8);
    memcpy(&pb, &b, 8);
    pa &= 0x7FFFFFFFFFFFFFFFull;
    pb &= 0x7FFFFFFFFFFFFFFFull;
    return ca > 0 ? pa > pb : pa < pb;
}

static int greater_f32(float a, float b)
{
    int ca = nan_class(isnan(a), signbit(a) != 0), cb = nan_class(isnan(b), signbit(b) != 0);
    if (ca != cb) return ca > cb;
    if (ca == 0) {
        if (a != b) return a > b;
        return (signbit(a) == 0) && (signbit(b) != 0);
    }
    uint32_t pa, pb;
    memcpy(&pa, &a, 4);
    memcpy(&pb, &b, 4);
    pa &= 0x7FFFFFFFu;
    pb &= 0x7FFFFFFFu;
    return ca > 0 ? pa > pb : pa < pb;
}

/* Arrays of n keys, insertion sort by totalOrder (stable). */
void oracle_sort_fixed_f32(float *keys, int n, uint64_t count)
{
    for (uint64_t a = 0; a < count; ++a) {
        float *A = keys + a * (uint64_t)n;
        for (int i = 1; i < n; ++i) {
            float x = A[i];
            int j = i - 1;
            while (j >= 0 && greater_f32(A[j], x)) {
                A[j + 1] = A[j];
                --j;
            }
            A[j + 1] = x;
        }
    }
}

void oracle_sort_fixed_f64(double *keys, int n, uint64_t count)
{
    for (uint64_t a = 0; a < count; ++a) {
        double *A = keys + a * (uint64_t)n;
        for (int i = 1; i < n; ++i) {
            double x = A[i];
            int j = i - 1;
            while (j >= 0 && greater_f64(A[j], x)) {
                A[j + 1] = A[j];
                --j;
            }
            A[j + 1] = x;
        }
    }
}

/* CSR segments by totalOrder, stable, payload moved with its key. */
void oracle_sort_segments_f32(float *keys, uint32_t *vals, const uint32_t *offsets, uint64_t nseg)
{
    for (uint64_t s = 0; s < nseg; ++s) {
        float *A = keys + offsets[s];
        uint32_t *V = vals ? vals + offsets[s] : NULL;
        int64_t len = (int64_t)offsets[s + 1] - (int64_t)offsets[s];
        for (int64_t i = 1; i < len; ++i) {
            float x = A[i];
            uint32_t v = V ? V[i] : 0;
            int64_t j = i - 1;
            while (j >= 0 && greater_f32(A[j], x)) {
                A[j + 1] = A[j];
                if (V) V[j + 1] = V[j];
                --j;
            }
            A[j + 1] = x;
            if (V) V[j + 1] = v;
        }
    }
}

void oracle_sort_segments_f64(double *keys, uint32_t *vals, const uint32_t *offsets, uint64_t nseg)
{
    for (uint64_t s = 0; s < nseg; ++s) {
        double *A = keys + offsets[s];
        uint32_t *V = vals ? vals + offsets[s] : NULL;
        int64_t len = (int64_t)offsets[s + 1] - (int64_t)offsets[s];
        for (int64_t i = 1; i < len; ++i) {
            double x = A[i];
            uint32_t v = V ? V[i] : 0;
            int64_t j = i - 1;
            while (j >= 0 && greater_f64(A[j], x)) {
                A[j + 1] = A[j];
                if (V) V[j + 1] = V[j];
                --j;
            }
            A[j + 1] = x;
            if (V) V[j + 1] = v;
        }
    }
}

/* ---- Sorting networks (Sec. 2.1) ---- */

/*
 * Apply a comparator network to one vector x[0..n-1]: for each comparator
 * (lo[c], hi[c]) in order, if the lower-numbered channel holds a greater value
 * than the higher-numbered one, exchange them (Sec. 2.1).  Channels are 0-based.
 */
static void apply_network(int64_t *x, const int *lo, const int *hi, int m)
{
    for (int c = 0; c < m; ++c) {
        if (x[lo[c]] > x[hi[c]]) {
            int64_t t = x[lo[c]];
            x[lo[c]] = x[hi[c]];
            x[hi[c]] = t;
        }
    }
}

static int is_nondecreasing(const int64_t *x, int n)
{
    for (int i = 1; i < n; ++i)
        if (x[i - 1] > x[i]) return 0;
    return 1;
}

/* Returns -1 if any comparator is malformed (channel out of range or lo >= hi). */
static int check_pairs(int n, const int *lo, const int *hi, int m)
{
    for (int c = 0; c < m; ++c)
        if (lo[c] < 0 || hi[c] >= n || lo[c] >= hi[c]) return -1;
    return 0;
}

/*
 * Number of the 2^n vectors over {0,1} that the network leaves unsorted
 * (0 means: sorts every input, by the 0-1 principle).  n <= 24.
 */
int64_t oracle_network_failures_01(int n, const int *lo, const int *hi, int m)
{
    if (n < 1 || n > 24 || check_pairs(n, lo, hi, m)) return -1;
    int64_t x[64];
    int64_t failures = 0;
    for (uint64_t v = 0; v < (1ull << n); ++v) {
        for (int i = 0; i < n; ++i) x[i] = (int64_t)((v >> i) & 1u);
        apply_network(x, lo, hi, m);
        if (!is_nondecreasing(x, n)) ++failures;
    }
    return failures;
}

/*
 * Number of the n! permutations of 0..n-1 that the network leaves unsorted.
 * Permutations are enumerated in lexicographic order (next-permutation).
 * n <= 10.
 */
int64_t oracle_network_failures_perm(int n, const int *lo, const int *hi, int m)
{
    if (n < 1 || n > 10 || check_pairs(n, lo, hi, m)) return -1;
    int p[16];
    int64_t x[16];
    int64_t failures = 0;
    for (int i = 0; i < n; ++i) p[i] = i;
    for (;;) {
        for (int i = 0; i < n; ++i) x[i] = p[i];
        apply_network(x, lo, hi, m);
        if (!is_nondecreasing(x, n)) ++failures;
        /* next permutation */
        int i = n - 2;
        while (i >= 0 && p[i] > p[i + 1]) --i;
        if (i < 0) break;
        int j = n - 1;
        while (p[j] < p[i]) --j;
        int t = p[i]; p[i] = p[j]; p[j] = t;
        for (int a = i + 1, b = n - 1; a < b; ++a, --b) {
            t = p[a]; p[a] = p[b]; p[b] = t;
        }
    }
    return failures;
}

/*
 * Depth (Sec. 2.1): the minimal number of levels, a level being a set of
 * comparators that share no channel.  Each comparator is placed one level
 * after the latest level that used either of its channels.
 */
int oracle_network_depth(int n, const int *lo, const int *hi, int m)
{
    if (n < 1 || n > 64 || check_pairs(n, lo, hi, m)) return -1;
    int last[64];
    int depth = 0;
    for (int i = 0; i < n; ++i) last[i] = 0;
    for (int c = 0; c < m; ++c) {
        int l = last[lo[c]] > last[hi[c]] ? last[lo[c]] : last[hi[c]];
        l += 1;
        last[lo[c]] = l;
        last[hi[c]] = l;
        if (l > depth) depth = l;
    }
    return depth;
}

/*
 * 0-1 check for wide networks (n <= 32): the same test as
 * oracle_network_failures_01, evaluated 64 input vectors at a time.  Word w of
 * channel i holds bit i of the 64 vector indices 64*block + (0..63); a
 * comparator maps (a, b) to (a AND b, a OR b), which is min/max on bits.
 */
int64_t oracle_network_failures_01_wide(int n, const int *lo, const int *hi, int m)
{
    if (n < 7 || n > 32 || check_pairs(n, lo, hi, m)) return -1;
    static const uint64_t low_pattern[6] = {
        0xAAAAAAAAAAAAAAAAull, 0xCCCCCCCCCCCCCCCCull, 0xF0F0F0F0F0F0F0F0ull,
        0xFF00FF00FF00FF00ull, 0xFFFF0000FFFF0000ull, 0xFFFFFFFF00000000ull};
    uint64_t x[32];
    int64_t failures = 0;
    uint64_t nblocks = 1ull << (n - 6);
    for (uint64_t blk = 0; blk < nblocks; ++blk) {
        for (int i = 0; i < 6; ++i) x[i] = low_pattern[i];
        for (int i = 6; i < n; ++i) x[i] = ((blk >> (i - 6)) & 1u) ? ~0ull : 0ull;
        for (int c = 0; c < m; ++c) {
            uint64_t a = x[lo[c]], b = x[hi[c]];
            x[lo[c]] = a & b;
            x[hi[c]] = a | b;
        }
        uint64_t bad = 0;
        for (int i = 1; i < n; ++i) bad |= x[i - 1] & ~x[i];
        failures += __builtin_popcountll(bad);
    }
    return failures;
}

/* ---- The paper's permutation check (Sec. 4.1) ---- */

/* (a * b) mod p, exact through a 128-bit product (GCC's unsigned __int128). */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p)
{
    return (uint64_t)(((unsigned __int128)(a % p) * (unsigned __int128)(b % p)) % p);
}

/* v = prod_i (z - a_i) mod p, with the subtraction taken mod p; p < 2^63. */
uint64_t oracle_perm_product_u64(const uint64_t *a, uint64_t len, uint64_t z, uint64_t p)
{
    uint64_t v = 1 % p;
    uint64_t zr = z % p;
    for (uint64_t i = 0; i < len; ++i) {
        uint64_t ar = a[i] % p;
        uint64_t d = zr >= ar ? zr - ar : zr + (p - ar);
        v = mulmod(v, d, p);
    }
    return v;
}

uint64_t oracle_perm_product_u32(const uint32_t *a, uint64_t len, uint64_t z, uint64_t p)
{
    uint64_t v = 1 % p;
    uint64_t zr = z % p;
    for (uint64_t i = 0; i < len; ++i) {
        uint64_t ar = (uint64_t)a[i] % p;
        uint64_t d = zr >= ar ? zr - ar : zr + (p - ar);
        v = mulmod(v, d, p);
    }
    return v;
}

/* 1 if every array / segment is non-decreasing, else 0 (Sec. 4.1 sorted check). */
int oracle_is_sorted_segments_u64(const uint64_t *keys, const uint32_t *offsets, uint64_t nseg)
{
    for (uint64_t s = 0; s < nseg; ++s)
        for (uint64_t i = (uint64_t)offsets[s] + 1; i < offsets[s + 1]; ++i)
            if (keys[i - 1] > keys[i]) return 0;
    return 1;
}

int oracle_is_sorted_segments_u32(const uint32_t *keys, const uint32_t *offsets, uint64_t nseg)
{
    for (uint64_t s = 0; s < nseg; ++s)
        for (uint64_t i = (uint64_t)offsets[s] + 1; i < offsets[s + 1]; ++i)
            if (keys[i - 1] > keys[i]) return 0;
    return 1;
}
