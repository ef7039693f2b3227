/*
 * Randomised greedy search for small sorting networks (build-time tool).
 *
 * A network is grown comparator by comparator.  The state is the set S of
 * distinct 0-1 vectors the network can output (bit i = channel i); by the 0-1
 * principle the network sorts once S holds only the n+1 sorted vectors.  A
 * comparator (i, j) maps every v in S with v_i = 1, v_j = 0 to v with those
 * two bits exchanged; the map is injective on the moved vectors and their
 * images are unmoved vectors, so the new size is |S| minus the number of
 * moved v whose image is already in S.  Each step keeps a comparator with the
 * largest such reduction (ties broken at random, sometimes a near-best one),
 * after a fixed prefix given on the command line.
 *
 * usage: search N RESTARTS SEED [i j]...      (prefix pairs, 0-based, i < j)
 * prints the smallest network found: "size K" then one "i j" line each.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static uint64_t rng_state;
static uint64_t rng_next(void)
{   /* SplitMix64 */
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

#define MAXN 16
#define MAXC 200

static int n;
static uint32_t *set_v;     /* current distinct vectors */
static uint32_t set_size;
static uint8_t *member;     /* member[v] = 1 iff v in S */

static void apply(int i, int j)
{
    uint32_t bi = 1u << i, bj = 1u << j;
    uint32_t w = 0;
    for (uint32_t k = 0; k < set_size; ++k) {
        uint32_t v = set_v[k];
        if ((v & bi) && !(v & bj)) {
            uint32_t u = v ^ bi ^ bj;
            member[v] = 0;
            if (member[u]) continue; /* merged into an existing vector */
            member[u] = 1;
            set_v[w++] = u;
        } else {
            set_v[w++] = v;
        }
    }
    set_size = w;
}

static uint32_t reduction(int i, int j)
{
    uint32_t bi = 1u << i, bj = 1u << j, r = 0;
    for (uint32_t k = 0; k < set_size; ++k) {
        uint32_t v = set_v[k];
        if ((v & bi) && !(v & bj) && member[v ^ bi ^ bj]) ++r;
    }
    return r;
}

static int moves_any(int i, int j)
{
    uint32_t bi = 1u << i, bj = 1u << j;
    for (uint32_t k = 0; k < set_size; ++k)
        if ((set_v[k] & bi) && !(set_v[k] & bj)) return 1;
    return 0;
}

int main(int argc, char **argv)
{
    if (argc < 4) {
        fprintf(stderr, "usage: search N RESTARTS SEED [i j]...\n");
        return 2;
    }
    n = atoi(argv[1]);
    long restarts = atol(argv[2]);
    rng_state = strtoull(argv[3], NULL, 10);
    int npre = (argc - 4) / 2;
    int pre_i[MAXC], pre_j[MAXC];
    if (n < 2 || n > MAXN || npre > MAXC) return 2;
    for (int c = 0; c < npre; ++c) {
        pre_i[c] = atoi(argv[4 + 2 * c]);
        pre_j[c] = atoi(argv[5 + 2 * c]);
        if (pre_i[c] < 0 || pre_j[c] >= n || pre_i[c] >= pre_j[c]) return 2;
    }
    uint32_t nvec = 1u << n;
    set_v = malloc(nvec * sizeof(uint32_t));
    member = malloc(nvec);
    int best_size = MAXC + 1;
    int best_i[MAXC], best_j[MAXC];
    int cur_i[MAXC], cur_j[MAXC];
    for (long r = 0; r < restarts; ++r) {
        memset(member, 0, nvec);
        for (uint32_t v = 0; v < nvec; ++v) {
            set_v[v] = v;
            member[v] = 1;
        }
        set_size = nvec;
        int m = 0;
        for (int c = 0; c < npre; ++c) {
            apply(pre_i[c], pre_j[c]);
            cur_i[m] = pre_i[c];
            cur_j[m] = pre_j[c];
            ++m;
        }
        while (set_size > (uint32_t)n + 1 && m < best_size - 1 && m < MAXC) {
            uint32_t top = 0;
            int cand_i[MAXN * MAXN], cand_j[MAXN * MAXN];
            uint32_t cand_r[MAXN * MAXN];
            int nc = 0;
            for (int i = 0; i < n; ++i)
                for (int j = i + 1; j < n; ++j) {
                    if (!moves_any(i, j)) continue;
                    uint32_t red = reduction(i, j);
                    cand_i[nc] = i;
                    cand_j[nc] = j;
                    cand_r[nc] = red;
                    ++nc;
                    if (red > top) top = red;
                }
            if (nc == 0) break;
            /* mostly the best reduction; now and then a near-best one */
            uint32_t floor_r = top;
            if ((rng_next() & 7u) == 0) floor_r = top - top / 8;
            int pick_list[MAXN * MAXN], np = 0;
            for (int c = 0; c < nc; ++c)
                if (cand_r[c] >= floor_r) pick_list[np++] = c;
            int c = pick_list[rng_next() % (uint64_t)np];
            apply(cand_i[c], cand_j[c]);
            cur_i[m] = cand_i[c];
            cur_j[m] = cand_j[c];
            ++m;
        }
        if (set_size == (uint32_t)n + 1 && m < best_size) {
            best_size = m;
            memcpy(best_i, cur_i, sizeof(int) * m);
            memcpy(best_j, cur_j, sizeof(int) * m);
        }
    }
    if (best_size > MAXC) {
        printf("size none\n");
        return 1;
    }
    printf("size %d\n", best_size);
    for (int c = 0; c < best_size; ++c) printf("%d %d\n", best_i[c], best_j[c]);
    return 0;
}
