/*
 * CPU oracle for speculative first-fit graph coloring.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package's smoke check and the benchmark's CPU
 * baseline leg load or run this file.  The CUDA library shares no code, header or constant
 * generator with it, and never calls it.
 *
 * What it computes (Singhal, Peri & Kalyanasundaram, "Multi-threaded Graph Coloring Algorithm
 * for Shared Memory Architecture", arXiv:1509.08267):
 *
 *  - oracle_greedy: sequential First Fit in natural vertex order (Section 3, the strategy all
 *    algorithms use; Section 5's "sequential run").  Every vertex, in id order, takes the least
 *    color c >= 0 that none of its already-colored neighbours holds.
 *
 *  - oracle_det: the barrier algorithm (Section 3.1, Algorithm 1) with every vertex its own
 *    partition, run round by round.  A round is phase 1 (tentative first fit for every worklist
 *    vertex), the barrier, then phase 2 (conflict detection, the loser of each monochromatic edge
 *    goes back on the worklist), then the second barrier.  Readings taken where the paper is
 *    silent or inconsistent:
 *      * phase 1 reads only the colors as they stood when the round began (a snapshot), so a
 *        round's result does not depend on the order worklist vertices are visited;
 *      * the "lower partition" endpoint of a conflict is the one with the larger priority key,
 *        key(v) = (SplitMix64 output number v of the stream seeded with `seed`, v), compared
 *        lexicographically; the smaller key keeps its color;
 *      * the vertex that is sent back is the worklist vertex itself (Lemma 1 and Lemma 2 recolor
 *        the vertex of the lower partition, not its neighbour);
 *      * a vertex that is sent back keeps its old color until it is recolored, and that color
 *        still forbids itself to its neighbours;
 *      * -1 means uncolored and forbids nothing; colors are 0-based (TotalColors = {0..m}).
 *
 *  - oracle_partition: Algorithm 1 literally, with p id-ordered blocks V_1..V_p, sequential first
 *    fit inside each block in phase 1 (in-block colors live, other blocks' colors from the start
 *    of the round), and in phase 2 the vertex of the lower-numbered block re-queued.
 *
 * Everything is single-threaded and unoptimised on purpose, so it can be read against the paper.
 */
#include <limits.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_GAMMA 0x9E3779B97F4A7C15ULL

/* SplitMix64 (Steele, Lea & Flood 2014; Vigna's reference splitmix64.c): the state advances by
 * GAMMA before each output, and the output is the state passed through the mixing function.
 * Returns output number `index` (0-based) of the stream whose initial state is `seed`. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t index) {
    uint64_t z = seed + (index + 1) * ORACLE_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Priority order: 1 when key(u) < key(v), i.e. u keeps its color against v. */
int oracle_key_less(uint64_t seed, int32_t u, int32_t v) {
    uint64_t hu = oracle_splitmix64(seed, (uint64_t)u);
    uint64_t hv = oracle_splitmix64(seed, (uint64_t)v);
    if (hu != hv) return hu < hv;
    return u < v;
}

/* Largest-first priority (an ordering from the paper's future work, Section 6): a vertex of larger
 * degree keeps its color; degrees of 2^20 - 1 and more count as 2^20 - 1; equal (capped) degrees
 * fall back to the hash order above.  1 when u keeps its color against v. */
#define ORACLE_DEG_CAP 1048575
int oracle_key_less_lf(uint64_t seed, int32_t u, int32_t v, int32_t du, int32_t dv) {
    if (du > ORACLE_DEG_CAP) du = ORACLE_DEG_CAP;
    if (dv > ORACLE_DEG_CAP) dv = ORACLE_DEG_CAP;
    if (du != dv) return du > dv;
    return oracle_key_less(seed, u, v);
}

void oracle_keys(uint64_t seed, int32_t n, uint64_t *out) {
    for (int32_t v = 0; v < n; ++v) out[v] = oracle_splitmix64(seed, (uint64_t)v);
}

static int32_t max_degree(int32_t n, const int32_t *rowptr) {
    int32_t m = 0;
    for (int32_t v = 0; v < n; ++v)
        if (rowptr[v + 1] - rowptr[v] > m) m = rowptr[v + 1] - rowptr[v];
    return m;
}

/* Least color c >= 0 not in {colors[u] : u in N(v), colors[u] >= 0}.  The answer is at most
 * deg(v), so only colors 0..deg(v) need to be recorded.  `seen` has deg(v)+1 zeroed bytes on
 * entry and is zeroed again on exit. */
static int32_t first_fit(int32_t v, const int32_t *rowptr, const int32_t *colidx, const int32_t *colors,
                         unsigned char *seen) {
    int32_t d = rowptr[v + 1] - rowptr[v];
    for (int32_t j = rowptr[v]; j < rowptr[v + 1]; ++j) {
        int32_t c = colors[colidx[j]];
        if (c >= 0 && c <= d) seen[c] = 1;
    }
    int32_t c = 0;
    while (seen[c]) ++c;
    memset(seen, 0, (size_t)d + 1);
    return c;
}

/* Number of distinct colors >= 0 in colors[0..n). */
int32_t oracle_distinct_colors(int32_t n, const int32_t *colors) {
    int32_t mx = -1;
    for (int32_t v = 0; v < n; ++v)
        if (colors[v] > mx) mx = colors[v];
    if (mx < 0) return 0;
    unsigned char *used = (unsigned char *)calloc((size_t)mx + 1, 1);
    int32_t k = 0;
    for (int32_t v = 0; v < n; ++v)
        if (colors[v] >= 0 && !used[colors[v]]) {
            used[colors[v]] = 1;
            ++k;
        }
    free(used);
    return k;
}

/* Directed adjacency entries (v, u) with colors[u] == colors[v]; zero for a proper coloring. */
int64_t oracle_count_conflicts(int32_t n, const int32_t *rowptr, const int32_t *colidx, const int32_t *colors) {
    int64_t bad = 0;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t j = rowptr[v]; j < rowptr[v + 1]; ++j)
            if (colors[colidx[j]] == colors[v]) ++bad;
    return bad;
}

/* Sequential First Fit in natural order.  Returns the number of colors used (-1 on OOM). */
int32_t oracle_greedy(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *colors) {
    if (n <= 0) return 0;
    unsigned char *seen = (unsigned char *)calloc((size_t)max_degree(n, rowptr) + 2, 1);
    if (!seen) return -1;
    for (int32_t v = 0; v < n; ++v) colors[v] = -1;
    int32_t used = 0;
    for (int32_t v = 0; v < n; ++v) {
        /* neighbours later in the order are still -1 and forbid nothing */
        colors[v] = first_fit(v, rowptr, colidx, colors, seen);
        if (colors[v] + 1 > used) used = colors[v] + 1;
    }
    free(seen);
    return used;
}

/* qsort context for oracle_greedy_keyorder (single-threaded use only) */
static uint64_t g_ko_seed;
static int32_t g_ko_priority;
static const int32_t *g_ko_rowptr;
static const int32_t *g_ko_colors_in;
static int ko_cmp(const void *a, const void *b) {
    int32_t u = *(const int32_t *)a, v = *(const int32_t *)b;
    if (u == v) return 0;
    int less;
    if (g_ko_priority == 1)
        less = oracle_key_less_lf(g_ko_seed, u, v, g_ko_rowptr[u + 1] - g_ko_rowptr[u], g_ko_rowptr[v + 1] - g_ko_rowptr[v]);
    else if (g_ko_priority == 2 || g_ko_priority == 3) /* a per-vertex rank in place of the degree */
        less = oracle_key_less_lf(g_ko_seed, u, v, g_ko_colors_in[u], g_ko_colors_in[v]);
    else
        less = oracle_key_less(g_ko_seed, u, v);
    return less ? -1 : 1;
}

/* Sequential First Fit in increasing key order (priority 0: hash key, 1: largest degree first,
 * 2 and 3: largest rank[v] first -- the peel level of oracle_peel_levels for the smallest-last
 * order, the given color for the recoloring pass of iterated greedy): the vertices are sorted by
 * key, then each takes the least color its already-colored neighbours do not use.  rank is read
 * for priorities 2 and 3 only (entries >= 0).  Returns the number of colors (-1 on OOM). */
int32_t oracle_greedy_keyorder(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed,
                               int32_t priority, const int32_t *colors_in, int32_t *colors) {
    if (n <= 0) return 0;
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    unsigned char *seen = (unsigned char *)calloc((size_t)max_degree(n, rowptr) + 2, 1);
    if (!order || !seen) {
        free(order);
        free(seen);
        return -1;
    }
    for (int32_t v = 0; v < n; ++v) {
        order[v] = v;
        colors[v] = -1;
    }
    g_ko_seed = seed;
    g_ko_priority = priority;
    g_ko_rowptr = rowptr;
    g_ko_colors_in = colors_in;
    qsort(order, (size_t)n, sizeof(int32_t), ko_cmp);
    int32_t used = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t v = order[i];
        colors[v] = first_fit(v, rowptr, colidx, colors, seen);
        if (colors[v] + 1 > used) used = colors[v] + 1;
    }
    free(order);
    free(seen);
    return used;
}

/* Smallest-last order by batch peeling (reading of the "other orderings" of the paper's future
 * work): res[v] starts at deg(v) and k at 0.  While vertices remain: k <- max(k, least res among
 * them); then, while some remaining vertex has res <= k, all such vertices are removed together as
 * the next level (1, 2, ...) and each removal lowers res of every neighbour by one.  level[v] is the
 * level that removed v; the smallest-last key colors larger levels first.  Returns the largest k,
 * which is the degeneracy of the graph (-1 on OOM). */
int32_t oracle_peel_levels(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *level) {
    if (n <= 0) return 0;
    int32_t *res = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *F = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!res || !F) {
        free(res);
        free(F);
        return -1;
    }
    for (int32_t v = 0; v < n; ++v) {
        res[v] = rowptr[v + 1] - rowptr[v];
        level[v] = 0;
    }
    int32_t k = 0, L = 0, remaining = n;
    while (remaining > 0) {
        int32_t kmin = INT32_MAX;
        for (int32_t v = 0; v < n; ++v)
            if (level[v] == 0 && res[v] < kmin) kmin = res[v];
        if (kmin > k) k = kmin;
        for (;;) {
            int32_t nf = 0;
            for (int32_t v = 0; v < n; ++v)
                if (level[v] == 0 && res[v] <= k) F[nf++] = v;
            if (nf == 0) break;
            L += 1;
            for (int32_t i = 0; i < nf; ++i) level[F[i]] = L;
            for (int32_t i = 0; i < nf; ++i)
                for (int32_t j = rowptr[F[i]]; j < rowptr[F[i] + 1]; ++j) res[colidx[j]] -= 1;
            remaining -= nf;
        }
    }
    free(res);
    free(F);
    return k;
}

/* Rounds of First Fit in key order when every vertex is colored as soon as all its smaller-key
 * neighbours are: depth[v] = 0 for an isolated vertex (colored before the first round), else 1 +
 * the largest depth among its smaller-key neighbours (1 when it has none).  Vertices are visited in
 * increasing key order, so a neighbour already visited is exactly a smaller-key one.  Returns the
 * largest depth (-1 on OOM). */
int32_t oracle_keyorder_depth(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed,
                              int32_t priority, const int32_t *colors_in, int32_t *depth) {
    if (n <= 0) return 0;
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    unsigned char *visited = (unsigned char *)calloc((size_t)n, 1);
    if (!order || !visited) {
        free(order);
        free(visited);
        return -1;
    }
    for (int32_t v = 0; v < n; ++v) {
        order[v] = v;
        depth[v] = 0;
    }
    g_ko_seed = seed;
    g_ko_priority = priority;
    g_ko_rowptr = rowptr;
    g_ko_colors_in = colors_in;
    qsort(order, (size_t)n, sizeof(int32_t), ko_cmp);
    int32_t deepest = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t v = order[i];
        visited[v] = 1;
        if (rowptr[v + 1] == rowptr[v]) continue;
        int32_t d = 0;
        for (int32_t j = rowptr[v]; j < rowptr[v + 1]; ++j)
            if (visited[colidx[j]] && colidx[j] != v && depth[colidx[j]] > d) d = depth[colidx[j]];
        depth[v] = d + 1;
        if (depth[v] > deepest) deepest = depth[v];
    }
    free(order);
    free(visited);
    return deepest;
}

/*
 * Deterministic speculative coloring (Algorithm 1, one vertex per partition, hash priority).
 *
 *   C <- all -1, W <- V (ascending), r <- 0
 *   while W is not empty:
 *       r <- r + 1
 *       S <- C                                                 (what phase 1 may read)
 *       for v in W:  C[v] <- least c >= 0 not in {S[u] : u in N(v)}        (phase 1)
 *       -- barrier --
 *       L <- {v in W : some u in N(v) has C[u] == C[v] and key(u) < key(v)}  (phase 2)
 *       W <- L
 *       -- barrier --
 *
 * key: priority 0, the hash order (oracle_key_less); 1, largest degree first (oracle_key_less_lf);
 * 2 and 3, largest rank[v] first (the same comparison with rank[v] in place of the degree).
 * Outputs the colors, the number of distinct colors and the number of rounds.  When `stats_cap`
 * > 0, wl_size[r-1] = |W_r| and wl_degsum[r-1] = sum of deg(v) over W_r for the first stats_cap
 * rounds.  When `last_round` is not NULL, last_round[v] = the last round whose worklist held v.
 * Returns 0, or -1 if W is still non-empty after `max_rounds` rounds, or -2 on OOM.
 */
int oracle_det_prio(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed, int32_t priority,
                    const int32_t *rank, int32_t max_rounds, int32_t *C, int32_t *ncolors, int32_t *rounds,
                    int64_t *wl_size, int64_t *wl_degsum, int32_t stats_cap, int32_t *last_round) {
    *ncolors = 0;
    *rounds = 0;
    if (n <= 0) return 0;
    int32_t *S = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *W = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *L = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    unsigned char *seen = (unsigned char *)calloc((size_t)max_degree(n, rowptr) + 2, 1);
    if (!S || !W || !L || !seen) {
        free(S);
        free(W);
        free(L);
        free(seen);
        return -2;
    }
    for (int32_t v = 0; v < n; ++v) {
        C[v] = -1;
        W[v] = v;
    }
    int32_t wn = n, r = 0, status = 0;
    while (wn > 0) {
        if (r >= max_rounds) {
            status = -1;
            break;
        }
        r += 1;
        if (last_round)
            for (int32_t i = 0; i < wn; ++i) last_round[W[i]] = r;
        if (r <= stats_cap) {
            int64_t ds = 0;
            for (int32_t i = 0; i < wn; ++i) ds += rowptr[W[i] + 1] - rowptr[W[i]];
            wl_size[r - 1] = wn;
            wl_degsum[r - 1] = ds;
        }
        memcpy(S, C, (size_t)n * sizeof(int32_t));
        for (int32_t i = 0; i < wn; ++i) C[W[i]] = first_fit(W[i], rowptr, colidx, S, seen);
        int32_t ln = 0;
        for (int32_t i = 0; i < wn; ++i) {
            int32_t v = W[i];
            for (int32_t j = rowptr[v]; j < rowptr[v + 1]; ++j) {
                int32_t u = colidx[j];
                int keeps = priority == 1   ? oracle_key_less_lf(seed, u, v, rowptr[u + 1] - rowptr[u],
                                                                 rowptr[v + 1] - rowptr[v])
                            : priority >= 2 ? oracle_key_less_lf(seed, u, v, rank[u], rank[v])
                                            : oracle_key_less(seed, u, v);
                if (C[u] == C[v] && keeps) {
                    L[ln++] = v;
                    break;
                }
            }
        }
        int32_t *t = W;
        W = L;
        L = t;
        wn = ln;
    }
    *rounds = r;
    *ncolors = oracle_distinct_colors(n, C);
    free(S);
    free(W);
    free(L);
    free(seen);
    return status;
}

/* oracle_det_prio with the hash priority (priority 0). */
int oracle_det(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed, int32_t max_rounds,
               int32_t *C, int32_t *ncolors, int32_t *rounds, int64_t *wl_size, int64_t *wl_degsum,
               int32_t stats_cap, int32_t *last_round) {
    return oracle_det_prio(n, rowptr, colidx, seed, 0, NULL, max_rounds, C, ncolors, rounds, wl_size, wl_degsum,
                           stats_cap, last_round);
}

/*
 * Algorithm 1 with p blocks: V_i = ids [floor((i-1)n/p), floor(i*n/p)) for i = 1..p (ids are
 * 0-based here).  Phase 1: inside each block, its worklist vertices are colored one after
 * another in id order; a vertex sees the current colors of its own block (including ones just
 * assigned in this phase) and the colors other blocks had when the round began.  Phase 2: a
 * worklist vertex v of block i is re-queued when a neighbour u in a block j > i has the same
 * color (the paper's i < j rule: the lower partition is recolored).  Neighbours inside the same
 * block never conflict, since each saw the other's final color.  Returns 0, -1 (round cap) or -2.
 */
int oracle_partition(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t p, int32_t max_rounds,
                     int32_t *C, int32_t *ncolors, int32_t *rounds, int64_t *wl_size, int32_t stats_cap) {
    *ncolors = 0;
    *rounds = 0;
    if (n <= 0) return 0;
    if (p < 1) p = 1;
    if (p > n) p = n;
    int32_t *block = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *S = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    unsigned char *onW = (unsigned char *)malloc((size_t)n);
    unsigned char *nextW = (unsigned char *)malloc((size_t)n);
    int32_t dmax = max_degree(n, rowptr);
    unsigned char *seen = (unsigned char *)calloc((size_t)dmax + 2, 1);
    if (!block || !S || !onW || !nextW || !seen) {
        free(block);
        free(S);
        free(onW);
        free(nextW);
        free(seen);
        return -2;
    }
    for (int32_t i = 0; i < p; ++i) {
        int64_t lo = (int64_t)i * n / p, hi = (int64_t)(i + 1) * n / p;
        for (int64_t v = lo; v < hi; ++v) block[v] = i;
    }
    for (int32_t v = 0; v < n; ++v) {
        C[v] = -1;
        onW[v] = 1;
    }
    int64_t wn = n;
    int32_t r = 0, status = 0;
    while (wn > 0) {
        if (r >= max_rounds) {
            status = -1;
            break;
        }
        r += 1;
        if (r <= stats_cap) wl_size[r - 1] = wn;
        memcpy(S, C, (size_t)n * sizeof(int32_t));
        /* phase 1, block by block (blocks are independent given S) */
        for (int32_t v = 0; v < n; ++v) {
            if (!onW[v]) continue;
            int32_t d = rowptr[v + 1] - rowptr[v];
            for (int32_t j = rowptr[v]; j < rowptr[v + 1]; ++j) {
                int32_t u = colidx[j];
                int32_t c = (block[u] == block[v]) ? C[u] : S[u];
                if (c >= 0 && c <= d) seen[c] = 1;
            }
            int32_t c = 0;
            while (seen[c]) ++c;
            memset(seen, 0, (size_t)d + 1);
            C[v] = c;
        }
        /* phase 2 */
        wn = 0;
        for (int32_t v = 0; v < n; ++v) {
            nextW[v] = 0;
            if (!onW[v]) continue;
            for (int32_t j = rowptr[v]; j < rowptr[v + 1]; ++j) {
                int32_t u = colidx[j];
                if (block[u] > block[v] && C[u] == C[v]) {
                    nextW[v] = 1;
                    ++wn;
                    break;
                }
            }
        }
        unsigned char *t = onW;
        onW = nextW;
        nextW = t;
    }
    *rounds = r;
    *ncolors = oracle_distinct_colors(n, C);
    free(block);
    free(S);
    free(onW);
    free(nextW);
    free(seen);
    return status;
}
