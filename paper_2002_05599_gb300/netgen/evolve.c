/*
 * Evolutionary search for small sorting networks (build-time tool).
 *
 * Works on the set S of distinct 0-1 vectors a network can output (bit i =
 * channel i).  By the 0-1 principle a network on n channels sorts every input
 * once S holds only the n + 1 sorted vectors.  A comparator (i, j), i < j,
 * maps every v in S with v_i = 1, v_j = 0 to v with those two bits exchanged;
 * a comparator that maps no vector of its input set is redundant and dropped.
 *
 * A network is a fixed prefix (command line) followed by a suffix that the
 * search changes.  The search keeps one current suffix and repeats:
 *   1. copy it and change it at random (drop one or two comparators, replace
 *      one, swap two, or insert one);
 *   2. evaluate the copy on the prefix's output set, dropping comparators that
 *      move nothing;
 *   3. if the copy no longer sorts, append comparators until it does, each a
 *      pair with the largest reduction of |S| (ties at random, now and then a
 *      random pair among those that move something);
 *   4. keep the copy if it is no longer than the current suffix (equal length
 *      is kept too, so the search can drift across plateaus), and now and
 *      then one a comparator longer; after many steps without a new best the
 *      search goes back to the best network found.
 * Environment: EVOLVE_RANDOM (percent of completion steps that pick a random
 * useful pair, default 6), EVOLVE_WORSE (per mille of one-longer copies kept,
 * default 20), EVOLVE_RESTART (steps without a new best before going back,
 * default 2e6).
 * With the reflection flag every change is applied to a comparator and to its
 * mirror image (n-1-j, n-1-i) together, which keeps the network symmetric
 * under reversing the channels and complementing the bits; the search space
 * shrinks by about half.  The prefix must then be symmetric too.
 *
 * usage: evolve N TARGET SEED SECONDS SYM [i j]...   (prefix pairs, 0-based, i < j)
 * Prints every new best as "size K" followed by one "i j" line per comparator
 * (prefix included) and stops at TARGET or after SECONDS.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define MAXN 16
#define MAXC 160

static uint64_t rng_state;
static uint64_t rng_next(void)
{ /* SplitMix64 (Steele, Lea, Flood 2014) */
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static uint32_t rnd(uint32_t m) { return (uint32_t)(rng_next() % m); }

typedef struct {
    uint8_t i, j;
} Cmp;

static int n, sym;
static int random_pct = 6; /* share of completion steps that take a random useful pair */
static uint32_t *pre_set, pre_size; /* output set of the prefix */
static uint32_t *work;              /* current set */
static uint32_t work_size;
static uint32_t *stamp, gen = 1;    /* stamp[v] == gen: v in the current set */

static Cmp mirror(Cmp c)
{
    Cmp m = {(uint8_t)(n - 1 - c.j), (uint8_t)(n - 1 - c.i)};
    return m;
}
static int same(Cmp a, Cmp b) { return a.i == b.i && a.j == b.j; }

static void load_prefix_set(void)
{
    ++gen;
    for (uint32_t k = 0; k < pre_size; ++k) {
        work[k] = pre_set[k];
        stamp[pre_set[k]] = gen;
    }
    work_size = pre_size;
}

/* Applies (i, j) to the current set; returns the number of vectors moved. */
static uint32_t apply(Cmp c)
{
    const uint32_t bi = 1u << c.i, bj = 1u << c.j;
    uint32_t w = 0, moved = 0;
    for (uint32_t k = 0; k < work_size; ++k) {
        const uint32_t v = work[k];
        if ((v & bi) && !(v & bj)) {
            const uint32_t u = v ^ bi ^ bj;
            ++moved;
            stamp[v] = 0;
            if (stamp[u] == gen) continue; /* merged with a vector already present */
            stamp[u] = gen;
            work[w++] = u;
        } else {
            work[w++] = v;
        }
    }
    work_size = w;
    return moved;
}

/* How much (i, j) would shrink the current set; *moves = whether it moves anything. */
static uint32_t reduction(Cmp c, int *moves)
{
    const uint32_t bi = 1u << c.i, bj = 1u << c.j;
    uint32_t r = 0;
    int mv = 0;
    for (uint32_t k = 0; k < work_size; ++k) {
        const uint32_t v = work[k];
        if ((v & bi) && !(v & bj)) {
            mv = 1;
            if (stamp[v ^ bi ^ bj] == gen) ++r;
        }
    }
    *moves = mv;
    return r;
}

/* Runs the suffix on the prefix set, keeping only comparators that move
   something (in place); returns the new length. */
static int evaluate(Cmp *s, int m)
{
    load_prefix_set();
    int w = 0;
    for (int k = 0; k < m; ++k)
        if (apply(s[k])) s[w++] = s[k];
    return w;
}

/* Appends comparators until the current set is sorted (or MAXC is reached). */
static int complete(Cmp *s, int m)
{
    while (work_size > (uint32_t)n + 1 && m < MAXC - 1) {
        Cmp cand[MAXN * MAXN];
        uint32_t red[MAXN * MAXN];
        int nc = 0;
        uint32_t top = 0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                Cmp c = {(uint8_t)i, (uint8_t)j};
                if (sym && (n - 1 - j) < i) continue; /* one of each mirror pair */
                int mv;
                uint32_t r = reduction(c, &mv);
                if (!mv) continue;
                cand[nc] = c;
                red[nc] = r;
                if (r > top) top = r;
                ++nc;
            }
        if (nc == 0) break;
        int pick;
        if (rnd(100) < (uint32_t)random_pct) {
            pick = (int)rnd((uint32_t)nc);
        } else {
            int list[MAXN * MAXN], nl = 0;
            for (int q = 0; q < nc; ++q)
                if (red[q] == top) list[nl++] = q;
            pick = list[rnd((uint32_t)nl)];
        }
        Cmp c = cand[pick];
        if (apply(c)) s[m++] = c;
        if (sym) {
            Cmp mc = mirror(c);
            if (!same(mc, c) && apply(mc)) s[m++] = mc;
        }
    }
    return m;
}

/* Index of the mirror partner of s[k] in the suffix (the nearest match). */
static int partner(const Cmp *s, int m, int k)
{
    Cmp mc = mirror(s[k]);
    if (same(mc, s[k])) return k;
    int best = -1, dist = MAXC + 1;
    for (int q = 0; q < m; ++q)
        if (q != k && same(s[q], mc) && abs(q - k) < dist) {
            dist = abs(q - k);
            best = q;
        }
    return best;
}

static void remove_at(Cmp *s, int *m, int k)
{
    memmove(s + k, s + k + 1, sizeof(Cmp) * (size_t)(*m - k - 1));
    --*m;
}
static void insert_at(Cmp *s, int *m, int k, Cmp c)
{
    if (*m >= MAXC - 2) return;
    memmove(s + k + 1, s + k, sizeof(Cmp) * (size_t)(*m - k));
    s[k] = c;
    ++*m;
}
static Cmp random_cmp(void)
{
    int i = (int)rnd((uint32_t)n), j = (int)rnd((uint32_t)n - 1);
    if (j >= i) ++j;
    if (i > j) { int t = i; i = j; j = t; }
    Cmp c = {(uint8_t)i, (uint8_t)j};
    return c;
}

/* Drops s[k] and, in reflection mode, its mirror partner. */
static void drop(Cmp *s, int *m, int k)
{
    int p = sym ? partner(s, *m, k) : k;
    if (p > k) { remove_at(s, m, p); remove_at(s, m, k); }
    else if (p >= 0 && p < k) { remove_at(s, m, k); remove_at(s, m, p); }
    else remove_at(s, m, k);
}

static void mutate(Cmp *s, int *m)
{
    if (*m == 0) return;
    switch (rnd(8)) {
    case 6: { /* move one comparator to another position */
        int k = (int)rnd((uint32_t)*m), to = (int)rnd((uint32_t)*m);
        Cmp c = s[k];
        remove_at(s, m, k);
        insert_at(s, m, to <= *m ? to : *m, c);
        break;
    }
    case 7: { /* shift one end of a comparator to a neighbouring channel */
        int k = (int)rnd((uint32_t)*m);
        Cmp c = s[k];
        int d = (rng_next() & 1) ? 1 : -1;
        if (rng_next() & 1) c.i = (uint8_t)(c.i + d); else c.j = (uint8_t)(c.j + d);
        if (c.i < c.j && c.j < n && c.i < 200) s[k] = c;
        break;
    }
    case 0: /* drop one */
    case 1:
        drop(s, m, (int)rnd((uint32_t)*m));
        break;
    case 2: /* drop two */
        drop(s, m, (int)rnd((uint32_t)*m));
        if (*m) drop(s, m, (int)rnd((uint32_t)*m));
        break;
    case 3: { /* replace one (and its mirror) */
        int k = (int)rnd((uint32_t)*m);
        Cmp c = random_cmp();
        int p = sym ? partner(s, *m, k) : k;
        s[k] = c;
        if (sym && p >= 0 && p != k) {
            Cmp mc = mirror(c);
            if (same(mc, c)) remove_at(s, m, p); else s[p] = mc;
        }
        break;
    }
    case 4: { /* swap two neighbours (and the mirrored pair) */
        if (*m < 2) break;
        int k = (int)rnd((uint32_t)*m - 1);
        Cmp t = s[k]; s[k] = s[k + 1]; s[k + 1] = t;
        break;
    }
    default: { /* insert one (and its mirror) */
        Cmp c = random_cmp();
        int k = (int)rnd((uint32_t)*m + 1);
        insert_at(s, m, k, c);
        if (sym && !same(mirror(c), c)) insert_at(s, m, k + 1, mirror(c));
        break;
    }
    }
}

int main(int argc, char **argv)
{
    if (argc < 6) {
        fprintf(stderr, "usage: evolve N TARGET SEED SECONDS SYM [i j]...\n");
        return 2;
    }
    n = atoi(argv[1]);
    const int target = atoi(argv[2]);
    rng_state = strtoull(argv[3], NULL, 10);
    const double seconds = atof(argv[4]);
    sym = atoi(argv[5]);
    const int npre = (argc - 6) / 2;
    if (n < 2 || n > MAXN || npre > MAXC) return 2;
    Cmp pre[MAXC];
    for (int c = 0; c < npre; ++c) {
        pre[c].i = (uint8_t)atoi(argv[6 + 2 * c]);
        pre[c].j = (uint8_t)atoi(argv[7 + 2 * c]);
        if (pre[c].i >= pre[c].j || pre[c].j >= n) return 2;
    }
    const uint32_t nvec = 1u << n;
    pre_set = malloc(nvec * sizeof(uint32_t));
    work = malloc(nvec * sizeof(uint32_t));
    stamp = calloc(nvec, sizeof(uint32_t));
    if (!pre_set || !work || !stamp) return 3;
    ++gen;
    for (uint32_t v = 0; v < nvec; ++v) {
        work[v] = v;
        stamp[v] = gen;
    }
    work_size = nvec;
    for (int c = 0; c < npre; ++c) apply(pre[c]);
    memcpy(pre_set, work, work_size * sizeof(uint32_t));
    pre_size = work_size;

    Cmp cur[MAXC], cand[MAXC];
    int cur_m = complete(cur, (load_prefix_set(), 0));
    cur_m = evaluate(cur, cur_m);
    int best = MAXC + 1, best_m = -1;
    Cmp best_net[MAXC];
    unsigned long long since_best = 0;
    const char *env;
    unsigned worse_permille = (env = getenv("EVOLVE_WORSE")) ? (unsigned)atoi(env) : 20;
    unsigned long long restart_after = (env = getenv("EVOLVE_RESTART")) ? strtoull(env, NULL, 10) : 2000000ull;
    if ((env = getenv("EVOLVE_RANDOM"))) random_pct = atoi(env);
    const clock_t t0 = clock();
    unsigned long long iters = 0;
    for (;;) {
        if (npre + cur_m < best) {
            best = npre + cur_m;
            best_m = cur_m;
            memcpy(best_net, cur, sizeof(Cmp) * (size_t)cur_m);
            printf("size %d\n", best);
            for (int c = 0; c < npre; ++c) printf("%d %d\n", pre[c].i, pre[c].j);
            for (int c = 0; c < cur_m; ++c) printf("%d %d\n", cur[c].i, cur[c].j);
            fflush(stdout);
            if (best <= target) break;
        }
        if ((++iters & 255u) == 0 && (double)(clock() - t0) / CLOCKS_PER_SEC > seconds) break;
        int m = cur_m;
        memcpy(cand, cur, sizeof(Cmp) * (size_t)m);
        mutate(cand, &m);
        m = evaluate(cand, m);
        m = complete(cand, m);
        if (work_size != (uint32_t)n + 1) continue;
        /* equal or shorter: always; one longer: now and then (leaves plateaus);
           after many steps without a new best, restart from the best */
        if (m <= cur_m || (m == cur_m + 1 && rnd(1000) < (uint32_t)worse_permille)) {
            cur_m = m;
            memcpy(cur, cand, sizeof(Cmp) * (size_t)m);
        }
        if (npre + cur_m < best) {
            since_best = 0;
        } else if (++since_best > restart_after && best_m >= 0) {
            cur_m = best_m;
            memcpy(cur, best_net, sizeof(Cmp) * (size_t)best_m);
            since_best = 0;
        }
    }
    fprintf(stderr, "iterations %llu, best %d\n", iters, best);
    return best <= target ? 0 : 1;
}
