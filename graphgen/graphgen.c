/*
 * Seeded synthetic graph generators (input plumbing only).
 *
 * This module builds the undirected simple graphs that both the CPU oracle and the CUDA library
 * color: Erdos-Renyi G(n, M), R-MAT, the 3-D 27-point stencil and the 2-D 5-point grid, all
 * emitted as int32 CSR with rows sorted by neighbour id, symmetric, without self-loops or
 * duplicate entries.  It holds none of the coloring method's arithmetic.
 *
 * Randomness: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; Vigna's public-domain splitmix64.c),
 * used counter-style: draw number k of the stream seeded with s is mix(s + (k + 1) * GAMMA).
 * Because each draw is addressed by its index, the graphs do not depend on thread count.
 *
 * Built as a shared library by graphgen/__init__.py (or the package build) with plain gcc;
 * OpenMP is used when the compiler offers it and changes no output.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Draw number `k` (0-based) of the SplitMix64 stream seeded with `seed`. */
uint64_t gg_draw(uint64_t seed, uint64_t k) { return gg_mix(seed + (k + 1) * GG_GAMMA); }

/* Uniform double in [0, 1) from the top 53 bits. */
static inline double gg_unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* Uniform integer in [0, n) by multiply-shift on the top 32 bits (n < 2^31). */
static inline int32_t gg_below(uint64_t x, int32_t n) {
    return (int32_t)(((x >> 32) * (uint64_t)(uint32_t)n) >> 32);
}

/*
 * Erdos-Renyi G(n, M): M vertex pairs (u, v), u != v, drawn uniformly with replacement.
 * Pair i uses draws 2j and 2j+1 for the j-th attempt; attempts with u == v are discarded.
 * Returns the number of pairs written (M), or -1 on bad arguments.
 */
int64_t gg_er_pairs(int32_t n, int64_t M, uint64_t seed, int32_t *src, int32_t *dst) {
    if (n < 2 || M < 0) return (M == 0) ? 0 : -1;
    uint64_t k = 0;
    for (int64_t i = 0; i < M;) {
        int32_t u = gg_below(gg_draw(seed, k), n);
        int32_t v = gg_below(gg_draw(seed, k + 1), n);
        k += 2;
        if (u == v) continue;
        src[i] = u;
        dst[i] = v;
        ++i;
    }
    return M;
}

/* One R-MAT edge attempt: `scale` quadrant choices, most significant bit first. */
static inline void gg_rmat_one(int scale, double a, double ab, double abc, uint64_t seed, uint64_t attempt,
                               int64_t *ps, int64_t *pd) {
    int64_t s = 0, d = 0;
    uint64_t base = attempt * (uint64_t)scale;
    for (int l = 0; l < scale; ++l) {
        double r = gg_unit(gg_draw(seed, base + (uint64_t)l));
        int64_t bit = (int64_t)1 << (scale - 1 - l);
        if (r < a) {
        } else if (r < ab) {
            d |= bit;
        } else if (r < abc) {
            s |= bit;
        } else {
            s |= bit;
            d |= bit;
        }
    }
    *ps = s;
    *pd = d;
}

/*
 * R-MAT (Chakrabarti, Zhan & Faloutsos 2004) with quadrant probabilities a, b, c, 1-a-b-c and
 * no noise.  Attempts are drawn in the 2^scale id space; when n < 2^scale an attempt with an
 * endpoint >= n is discarded and the next attempt index is used, until M pairs are kept.
 * Self-loops are kept here and dropped by gg_csr_from_pairs.  Returns M or -1.
 */
int64_t gg_rmat_pairs(int32_t n, int scale, int64_t M, double a, double b, double c, uint64_t seed,
                      int32_t *src, int32_t *dst) {
    if (n < 1 || scale < 1 || scale > 31 || M < 0) return -1;
    if ((int64_t)n > ((int64_t)1 << scale)) return -1;
    double ab = a + b, abc = a + b + c;
    if ((int64_t)n == ((int64_t)1 << scale)) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < M; ++i) {
            int64_t s, d;
            gg_rmat_one(scale, a, ab, abc, seed, (uint64_t)i, &s, &d);
            src[i] = (int32_t)s;
            dst[i] = (int32_t)d;
        }
        return M;
    }
    uint64_t attempt = 0;
    for (int64_t i = 0; i < M;) {
        int64_t s, d;
        gg_rmat_one(scale, a, ab, abc, seed, attempt++, &s, &d);
        if (s >= n || d >= n) continue;
        src[i] = (int32_t)s;
        dst[i] = (int32_t)d;
        ++i;
    }
    return M;
}

/* Seeded uniform permutation of 0..n-1 (Fisher-Yates, draw k for position n-1-k). */
void gg_permutation(int32_t n, uint64_t seed, int32_t *perm) {
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    uint64_t k = 0;
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = gg_below(gg_draw(seed, k++), i + 1);
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

static int gg_cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/*
 * Undirected simple CSR from a list of vertex pairs: every pair (s, d) with s != d contributes
 * both directions, ids are relabelled through `perm` when it is not NULL (new id = perm[old]),
 * rows are sorted and duplicates removed.  `colidx` needs room for 2*M entries; `rowptr` for n+1.
 * Returns nnz, or -1 when nnz would not fit in int32.
 */
int64_t gg_csr_from_pairs(int32_t n, int64_t M, const int32_t *src, const int32_t *dst, const int32_t *perm,
                          int32_t *rowptr, int32_t *colidx) {
    int64_t *cursor = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cursor) return -1;
    /* degrees with duplicates */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        int32_t s = src[i], d = dst[i];
        if (s == d) continue;
        if (perm) {
            s = perm[s];
            d = perm[d];
        }
        __atomic_fetch_add(&cursor[s + 1], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&cursor[d + 1], 1, __ATOMIC_RELAXED);
    }
    for (int32_t v = 0; v < n; ++v) cursor[v + 1] += cursor[v];
    int64_t total = cursor[n];
    int64_t *start = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!start) {
        free(cursor);
        return -1;
    }
    memcpy(start, cursor, ((size_t)n + 1) * sizeof(int64_t));
    /* scatter both directions; the order inside a row is fixed by the sort below */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        int32_t s = src[i], d = dst[i];
        if (s == d) continue;
        if (perm) {
            s = perm[s];
            d = perm[d];
        }
        int64_t ps = __atomic_fetch_add(&cursor[s], 1, __ATOMIC_RELAXED);
        int64_t pd = __atomic_fetch_add(&cursor[d], 1, __ATOMIC_RELAXED);
        colidx[ps] = d;
        colidx[pd] = s;
    }
    /* sort and deduplicate each row in place; cursor[v] becomes the unique count */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t v = 0; v < n; ++v) {
        int64_t b = start[v], e = start[v + 1];
        int32_t *row = colidx + b;
        int64_t len = e - b;
        if (len > 1) qsort(row, (size_t)len, sizeof(int32_t), gg_cmp_i32);
        int64_t w = 0;
        for (int64_t j = 0; j < len; ++j)
            if (w == 0 || row[j] != row[w - 1]) row[w++] = row[j];
        cursor[v] = w;
    }
    /* compact rows forward (new offsets never exceed old ones) */
    int64_t out = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t len = cursor[v];
        if (out > INT32_MAX - len) {
            free(cursor);
            free(start);
            return -1;
        }
        if (out != start[v] && len > 0) memmove(colidx + out, colidx + start[v], (size_t)len * sizeof(int32_t));
        rowptr[v] = (int32_t)out;
        out += len;
    }
    rowptr[n] = (int32_t)out;
    (void)total;
    free(cursor);
    free(start);
    return out;
}

/* Directed entries of the L x L x L 27-point stencil: (3L-2)^3 - L^3. */
int64_t gg_stencil27_nnz(int32_t L) {
    if (L < 1) return 0;
    int64_t t = 3 * (int64_t)L - 2;
    return t * t * t - (int64_t)L * L * L;
}

/*
 * 3-D 27-point stencil on an L x L x L grid, id = x + L*(y + L*z) (x fastest).  A vertex is
 * adjacent to every other grid point at Chebyshev distance 1.  Neighbours are emitted in
 * (dz, dy, dx) lexicographic order, which is ascending id order.  Returns nnz or -1 on overflow.
 */
int64_t gg_stencil27(int32_t L, int32_t *rowptr, int32_t *colidx) {
    int64_t nnz = gg_stencil27_nnz(L);
    int64_t n = (int64_t)L * L * L;
    if (nnz > INT32_MAX || n > INT32_MAX) return -1;
    /* row starts: degree = (#x offsets)(#y offsets)(#z offsets) - 1 */
    int64_t acc = 0;
    for (int64_t z = 0; z < L; ++z) {
        int cz = 1 + (z > 0) + (z < L - 1);
        for (int64_t y = 0; y < L; ++y) {
            int cy = 1 + (y > 0) + (y < L - 1);
            for (int64_t x = 0; x < L; ++x) {
                int cx = 1 + (x > 0) + (x < L - 1);
                rowptr[x + L * (y + L * z)] = (int32_t)acc;
                acc += (int64_t)cx * cy * cz - 1;
            }
        }
    }
    rowptr[n] = (int32_t)acc;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < L; ++z)
        for (int64_t y = 0; y < L; ++y)
            for (int64_t x = 0; x < L; ++x) {
                int64_t v = x + L * (y + L * z);
                int64_t p = rowptr[v];
                for (int dz = -1; dz <= 1; ++dz) {
                    int64_t zz = z + dz;
                    if (zz < 0 || zz >= L) continue;
                    for (int dy = -1; dy <= 1; ++dy) {
                        int64_t yy = y + dy;
                        if (yy < 0 || yy >= L) continue;
                        for (int dx = -1; dx <= 1; ++dx) {
                            int64_t xx = x + dx;
                            if (xx < 0 || xx >= L) continue;
                            if (dx == 0 && dy == 0 && dz == 0) continue;
                            colidx[p++] = (int32_t)(xx + L * (yy + L * zz));
                        }
                    }
                }
            }
    return acc;
}

/* Directed entries of the Lx x Ly 5-point grid. */
int64_t gg_grid5_nnz(int32_t Lx, int32_t Ly) {
    if (Lx < 1 || Ly < 1) return 0;
    return 2 * ((int64_t)(Lx - 1) * Ly + (int64_t)Lx * (Ly - 1));
}

/* 2-D 5-point grid, id = x + Lx*y; neighbours in ascending id order.  Returns nnz or -1. */
int64_t gg_grid5(int32_t Lx, int32_t Ly, int32_t *rowptr, int32_t *colidx) {
    int64_t n = (int64_t)Lx * Ly;
    int64_t nnz = gg_grid5_nnz(Lx, Ly);
    if (n > INT32_MAX || nnz > INT32_MAX) return -1;
    int64_t p = 0;
    for (int64_t y = 0; y < Ly; ++y)
        for (int64_t x = 0; x < Lx; ++x) {
            rowptr[x + Lx * y] = (int32_t)p;
            if (y > 0) colidx[p++] = (int32_t)(x + Lx * (y - 1));
            if (x > 0) colidx[p++] = (int32_t)(x - 1 + Lx * y);
            if (x < Lx - 1) colidx[p++] = (int32_t)(x + 1 + Lx * y);
            if (y < Ly - 1) colidx[p++] = (int32_t)(x + Lx * (y + 1));
        }
    rowptr[n] = (int32_t)p;
    return p;
}

/*
 * A whole batch of graphs generated in parallel, one graph per thread at a time (each graph's
 * output depends only on its own parameters).  Graph g is ER (kind 0: M = floor(n*param/2 + 1/2)
 * pairs) or R-MAT (kind 1: M = floor(n*param + 1/2) pairs, scale = ceil(log2 n), a/b/c as given,
 * ids permuted with the stream seed + perm_offset).  Graph g's local rowptr goes to
 * rowptr + vtx_off[g] + g and its local column ids to colidx + cap_off[g] (room for 2M entries);
 * nnz_out[g] receives its entry count.  gg_batch_pack then moves the column ids together.
 * Returns 0 or -1.
 */
static int gg_one_graph(int kind, int32_t n, double param, uint64_t seed, double a, double b, double c,
                        uint64_t perm_offset, int32_t *rowptr, int32_t *colidx, int64_t *nnz_out) {
    int64_t M = kind == 0 ? (int64_t)(n * param / 2.0 + 0.5) : (int64_t)(n * param + 0.5);  /* floor(x + 1/2) */
    if (n < 2) M = 0;
    int32_t *src = (int32_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int32_t));
    int32_t *dst = (int32_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int32_t));
    int32_t *perm = NULL;
    int32_t *rp = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *ci = (int32_t *)malloc((size_t)(2 * M > 0 ? 2 * M : 1) * sizeof(int32_t));
    if (!src || !dst || !rp || !ci) {
        free(src);
        free(dst);
        free(rp);
        free(ci);
        return -1;
    }
    if (kind == 0) {
        gg_er_pairs(n, M, seed, src, dst);
    } else {
        int scale = 1;
        while (((int64_t)1 << scale) < n) ++scale;
        /* sequential attempt loop (n is generally not a power of two) */
        double ab = a + b, abc = a + b + c;
        uint64_t attempt = 0;
        for (int64_t i = 0; i < M;) {
            int64_t s, d;
            gg_rmat_one(scale, a, ab, abc, seed, attempt++, &s, &d);
            if (s >= n || d >= n) continue;
            src[i] = (int32_t)s;
            dst[i] = (int32_t)d;
            ++i;
        }
        perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
        if (!perm) {
            free(src);
            free(dst);
            free(rp);
            free(ci);
            return -1;
        }
        gg_permutation(n, seed + perm_offset, perm);
    }
    /* serial CSR build (the batch is parallel across graphs) */
    int64_t *cursor = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t i = 0; i < M; ++i) {
        int32_t s = src[i], d = dst[i];
        if (s == d) continue;
        if (perm) {
            s = perm[s];
            d = perm[d];
        }
        cursor[s + 1]++;
        cursor[d + 1]++;
    }
    for (int32_t v = 0; v < n; ++v) cursor[v + 1] += cursor[v];
    int64_t *start = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    memcpy(start, cursor, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < M; ++i) {
        int32_t s = src[i], d = dst[i];
        if (s == d) continue;
        if (perm) {
            s = perm[s];
            d = perm[d];
        }
        ci[cursor[s]++] = d;
        ci[cursor[d]++] = s;
    }
    int64_t out = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t bb = start[v], e = start[v + 1];
        if (e - bb > 1) qsort(ci + bb, (size_t)(e - bb), sizeof(int32_t), gg_cmp_i32);
        rp[v] = (int32_t)out;
        for (int64_t j = bb; j < e; ++j)
            if (j == bb || ci[j] != ci[j - 1]) ci[out++] = ci[j];
    }
    rp[n] = (int32_t)out;
    *nnz_out = out;
    if (rowptr) {
        memcpy(rowptr, rp, ((size_t)n + 1) * sizeof(int32_t));
        memcpy(colidx, ci, (size_t)out * sizeof(int32_t));
    }
    free(cursor);
    free(start);
    free(src);
    free(dst);
    free(perm);
    free(rp);
    free(ci);
    return 0;
}

int gg_batch(int32_t G, const int32_t *kind, const int32_t *n, const double *param, const uint64_t *seed, double a,
             double b, double c, uint64_t perm_offset, const int64_t *vtx_off, const int64_t *cap_off,
             int32_t *rowptr, int32_t *colidx, int64_t *nnz_out) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int32_t g = 0; g < G; ++g) {
        int64_t nz = 0;
        if (gg_one_graph(kind[g], n[g], param[g], seed[g], a, b, c, perm_offset, rowptr + vtx_off[g] + g,
                         colidx + cap_off[g], &nz) != 0)
            bad |= 1;
        nnz_out[g] = nz;
    }
    return bad ? -1 : 0;
}

/* Moves graph g's column ids from cap_off[g] to edge_off[g] (edge_off[g] <= cap_off[g], increasing). */
void gg_batch_pack(int32_t G, const int64_t *cap_off, const int64_t *edge_off, int32_t *colidx) {
    for (int32_t g = 0; g < G; ++g) {
        int64_t len = edge_off[g + 1] - edge_off[g];
        if (len > 0 && cap_off[g] != edge_off[g])
            memmove(colidx + edge_off[g], colidx + cap_off[g], (size_t)len * sizeof(int32_t));
    }
}
