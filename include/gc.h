/*
 * gc.h -- C ABI of the GB300 speculative graph-coloring library (libgc.so).
 *
 * The library colors undirected simple graphs with the barrier-synchronised speculative method of
 * Singhal, Peri & Kalyanasundaram, "Multi-threaded Graph Coloring Algorithm for Shared Memory
 * Architecture" (arXiv:1509.08267), Section 3.1, Algorithm 1: every vertex on the worklist takes
 * the least color none of its neighbours uses (First Fit, Section 3), a conflict pass sends one
 * endpoint of every monochromatic edge back to the worklist (Algorithm 1, phase 2), and rounds
 * repeat until the worklist is empty.  Lemma 1 (Section 4) gives a proper coloring at the end;
 * every color is at most deg(v) <= Delta, so at most Delta+1 colors are used (Section 2.1).
 *
 * Graph format (all entry points).  Undirected simple graph G = (V, E) of Section 2.1 in CSR:
 *   rowptr  int32[n+1], rowptr[0] = 0, non-decreasing, rowptr[n] = nnz (number of directed entries)
 *   colidx  int32[nnz], row v = colidx[rowptr[v] .. rowptr[v+1]) lists the neighbours of v
 * Each undirected edge {u, v} appears as both (u, v) and (v, u); no self-loops, no duplicates.
 * Vertex ids are 0-based (the paper numbers them 1..|V|).  The coloring kernels check rowptr
 * monotonicity, neighbour ranges and self-loops on the fly; symmetry and duplicates are the
 * caller's promise unless checked with gc_validate_graph (an asymmetric input can yield an
 * improper coloring).
 *
 * Pointers.  Every array argument may be device memory of the current CUDA device (for example a
 * torch tensor's data_ptr) or host memory (pageable or pinned); the library tells them apart with
 * cudaPointerGetAttributes and stages host arrays through its own device buffers.  The caller owns
 * every array it passes; the library never keeps a pointer past the call.  Scalar outputs
 * (ncolors, rounds of gc_color) are host pointers.
 *
 * Scratch.  The library keeps a per-device context with cached device scratch that grows to the
 * largest problem seen; gc_release_scratch frees it.
 *
 * Errors.  Every entry point returns a gc_status.  On error the outputs are left untouched and
 * gc_last_error() returns a message for the calling thread.  No entry point falls back to a CPU
 * implementation: without a usable CUDA device every call returns GC_ERR_CUDA.
 *
 * Colors.  0-based int32.  ncolors = number of distinct colors in the result ("Number of Colors
 * Used", Section 5.2).  rounds = number of tentative-coloring phases executed (Algorithm 1's while
 * loop iterations): 0 for n = 0, 1 for a graph without edges.
 *
 * Modes.
 *   GC_MODE_DETERMINISTIC  Phase 1 of round r reads only the colors as they stood when round r
 *       began, and the endpoint of a monochromatic edge with the larger priority key is re-queued.
 *       key(v) = (h(v), v) compared lexicographically, h(v) = output number v (0-based) of the
 *       SplitMix64 generator seeded with `seed` (Steele, Lea & Flood 2014).  The result (colors,
 *       ncolors, rounds) is a function of the graph and the seed only, identical for every launch
 *       configuration and batch composition.
 *   GC_MODE_INPLACE  Phase 1 reads neighbour colors live, as the paper's threads do; the result
 *       depends on scheduling.  It is always a proper coloring with color(v) <= deg(v), and the
 *       number of rounds never exceeds n.
 *   GC_MODE_PARTITION  Algorithm 1 as printed: the vertices are split into p blocks of consecutive
 *       ids (block i = [floor(i n / p), floor((i+1) n / p)), gc_options.partitions); in phase 1 each
 *       block colors its worklist vertices one after another in id order, seeing its own block's
 *       colors live and other blocks' colors as the round began; in phase 2 a vertex is re-queued
 *       when a neighbour in a higher block has its color.  The result is a function of the graph
 *       and p (seed unused); Lemma 2 bounds the rounds by p + 1.  gc_color / gc_color_ex only.
 *   GC_MODE_ORDERED  No speculation: a vertex stays uncolored while a neighbour with a smaller
 *       key is uncolored, then takes First Fit once (the order that Algorithm 3's neighbourhood
 *       locks impose, as a wait rule instead of locks).  Each vertex counts its smaller-key
 *       neighbours; a round colors the vertices whose count is 0 and counts down their uncolored
 *       neighbours.  Colors equal sequential First Fit in increasing key order (with
 *       GC_PRIORITY_LARGEST_FIRST: largest degree first); the number of rounds is the most
 *       vertices on a path of increasing keys, and round r's worklist statistics count the
 *       vertices colored in round r.
 */
#ifndef GC_H
#define GC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GC_OK = 0,
    GC_ERR_INVALID_ARG = -1,     /* bad argument: NULL pointer, negative size, unknown mode */
    GC_ERR_INVALID_GRAPH = -2,   /* CSR breaks the graph format above */
    GC_ERR_OOM = -3,             /* device or pinned memory could not be allocated / admitted */
    GC_ERR_CUDA = -4,            /* a CUDA call failed (message has the CUDA error string) */
    GC_ERR_NO_CONVERGENCE = -5,  /* the worklist was not empty after the round cap */
    GC_ERR_TIMEOUT = -6,         /* a grid-barrier wait exceeded its limit; the kernel returned */
    GC_ERR_BUSY = -7             /* server request still running (gc_server_poll) */
} gc_status;

enum { GC_MODE_DETERMINISTIC = 0, GC_MODE_INPLACE = 1, GC_MODE_PARTITION = 2, GC_MODE_ORDERED = 3 };

/* Priority keys (which endpoint of a monochromatic edge keeps its color: the smaller key).
 *   GC_PRIORITY_HASH           key(v) = (h(v), v)
 *   GC_PRIORITY_LARGEST_FIRST  key(v) = (-min(deg(v), 2^20 - 1), h(v), v): larger degrees first, an
 *                              ordering the paper lists as future work (Section 6)
 *   GC_PRIORITY_SMALLEST_LAST  key(v) = (-min(level(v), 2^20 - 1), h(v), v) with level(v) the
 *                              smallest-last peel level of gc_smallest_last: vertices peeled last
 *                              first.  In GC_MODE_ORDERED this is First Fit in (batch) smallest-last
 *                              order, which uses at most degeneracy + 1 colors.  Single graphs only
 *                              (gc_color / gc_color_ex; not GC_MODE_PARTITION, not batches). */
enum { GC_PRIORITY_HASH = 0, GC_PRIORITY_LARGEST_FIRST = 1, GC_PRIORITY_SMALLEST_LAST = 2 };

/* Flags for gc_options.flags */
#define GC_FLAG_STATS 1u     /* fill gc_stats' per-round worklist sizes and scanned entries */
#define GC_FLAG_TIMING 2u    /* record CUDA events around the round kernel (gc_stats.kernel_ms) */
#define GC_FLAG_VALIDATE 4u  /* run gc_validate_graph(GC_VALIDATE_ALL) before coloring */
#define GC_FLAG_FULL_SWEEP 8u  /* deterministic mode: re-read every adjacency entry of a vertex each round
                                  instead of only the neighbours that can still change (same results) */

/* Flags for gc_validate_graph */
#define GC_VALIDATE_SORTED 1     /* rows strictly increasing (implies no duplicate entries) */
#define GC_VALIDATE_SYMMETRIC 2  /* (u, v) present whenever (v, u) is; requires sorted rows */
#define GC_VALIDATE_ALL 3

/* Tuning and control knobs; a zero field means "library default".  Pass NULL for all defaults. */
typedef struct gc_options {
    void *stream;              /* cudaStream_t to run on; NULL = the context's own stream */
    int32_t max_rounds;        /* round cap; 0 = n + 1 (a worklist shrinks every round) */
    int32_t small_max_degree;  /* vertices up to this degree get one thread each (1..127); default 127 */
    int32_t chunk;             /* adjacency entries per warp work item for larger vertices (32..8192, multiple of 32);
                                  default 1024 (ordered mode: at most 128; 64 by default on a single graph) */
    int32_t block_size;        /* threads per block of the round kernel (256 is the only size); default 256 */
    int32_t blocks_per_sm;     /* resident blocks per SM for the round kernel.  0: the library picks the
                                  80-register variant (3 blocks per SM) when most adjacency entries are
                                  in vertices of degree > small_max_degree, else the 64-register one (4);
                                  3 or 4: that variant; 1 or 2: the 64-register one, capped.  It also
                                  sets the ordered mode's blocks per SM (default 1 on a single graph,
                                  3 on a batch) and caps the smallest-last peeling kernels (3 per SM) */
    int64_t spin_limit_ns;     /* grid-barrier wait limit in ns; 0 = 1e9.  A wait that runs out makes
                                  the call return GC_ERR_TIMEOUT with the device still usable */
    uint32_t flags;            /* GC_FLAG_* */
    int32_t partitions;        /* GC_MODE_PARTITION: number of blocks p (clamped to 1..n); 0 = one per
                                  resident warp of the round kernel */
    int32_t priority;          /* deterministic, in-place and ordered modes: GC_PRIORITY_HASH (default),
                                  GC_PRIORITY_LARGEST_FIRST or GC_PRIORITY_SMALLEST_LAST */
    int32_t core_vertices;     /* deterministic mode: once the worklist has at most this many vertices, the
                                  remaining rounds run with every worklist vertex's color in shared memory
                                  (same results).  0 = the most one block's shared memory holds (about
                                  200k on GB300: one byte and one bit per vertex); < 0 = never */
    int32_t core_entries;      /* deterministic mode: the most adjacency entries the shared-memory rounds take
                                  (their rows are rebuilt once, at the hand-over); 0 = min(nnz, 2^27).  Above
                                  2^27 it is clamped.  Only a graph with more entries than this counts its
                                  worklists' entries every round to find the hand-over */
    int32_t tail_vertices;     /* deterministic mode, after the core phase: once the worklist has at most this
                                  many vertices, the remaining rounds run on one thread-block cluster
                                  (same results).  0 = 384; at most what the cluster holds (4,096 with
                                  16 blocks, 2,048 with 8), larger values are clamped; < 0 = never */
    int32_t reserved[3];
} gc_options;

/* Optional run statistics (gc_color_ex / gc_color_batch_ex).  The caller may provide arrays
 * wl_size / wl_degsum / round_ns of round_cap entries; entry r-1 receives |W_r|, the sum of deg(v)
 * over W_r and the round's duration for round r (GC_FLAG_STATS). */
typedef struct gc_stats {
    int32_t rounds;            /* rounds executed (largest over the batch for gc_color_batch_ex) */
    int32_t ncolors;           /* distinct colors (sum over the batch for gc_color_batch_ex) */
    int32_t max_color;         /* largest color used (largest over the batch) */
    int32_t round_cap;         /* capacity of wl_size / wl_degsum (input) */
    int64_t *wl_size;          /* caller array or NULL */
    int64_t *wl_degsum;        /* caller array or NULL */
    int64_t *round_ns;         /* caller array or NULL: device time of each round in ns (GC_FLAG_STATS) */
    int64_t worklist_total;    /* sum over rounds of |W_r| (GC_FLAG_STATS) */
    int64_t entries_scanned;   /* adjacency entries the round kernel read (GC_FLAG_STATS); without
                                  compaction this is sum_r sum_{v in W_r} deg(v) (twice that in-place) */
    float kernel_ms;           /* round-kernel device time (GC_FLAG_TIMING) */
    float setup_ms;            /* binning/setup kernel device time (GC_FLAG_TIMING) */
    int32_t grid_blocks;       /* blocks of the persistent round kernel */
    int32_t block_size;        /* threads per block of the round kernel */
    int64_t *round_reads;      /* caller array or NULL: adjacency entries the round kernel read in each
                                  round (GC_FLAG_STATS); they sum to entries_scanned */
    int32_t reserved[4];
} gc_stats;

/*
 * gc_color -- color one graph (Algorithm 1, Section 3.1).
 *   n          number of vertices (>= 0)
 *   rowptr     int32[n+1]   CSR row offsets (device or host)
 *   colidx     int32[nnz]   CSR neighbour ids (device or host); may be NULL when nnz = 0
 *   mode       GC_MODE_DETERMINISTIC, GC_MODE_INPLACE, GC_MODE_PARTITION or GC_MODE_ORDERED
 *   seed       priority-hash seed (deterministic mode; in-place mode uses it for tie-breaks too)
 *   colors_out int32[n]     receives the colors (device or host)
 *   ncolors    host int32*  receives the number of distinct colors (may be NULL)
 *   rounds     host int32*  receives the number of rounds (may be NULL)
 * Synchronous: returns after the colors are in colors_out.
 * Errors: GC_ERR_INVALID_ARG, GC_ERR_INVALID_GRAPH, GC_ERR_OOM, GC_ERR_CUDA,
 *         GC_ERR_NO_CONVERGENCE, GC_ERR_TIMEOUT; outputs untouched on error.
 */
int gc_color(int32_t n, const int32_t *rowptr, const int32_t *colidx, int mode, uint64_t seed,
             int32_t *colors_out, int32_t *ncolors, int32_t *rounds);

/* gc_color with options (may be NULL) and statistics (may be NULL). */
int gc_color_ex(int32_t n, const int32_t *rowptr, const int32_t *colidx, int mode, uint64_t seed,
                int32_t *colors_out, int32_t *ncolors, int32_t *rounds, const gc_options *opt,
                gc_stats *stats);

/*
 * gc_recolor -- one pass of iterated greedy recoloring (Culberson, 1992), a color-count reduction
 * of the kind the paper lists as future work (Section 6).  First Fit in key order (the ordered
 * mode) with key(v) = (-min(colors_in[v], 2^20 - 1), h_seed(v), v): the color classes of colors_in
 * one after another, the largest color first.  When colors_in is a proper coloring with colors
 * below 2^20 - 1, each class's vertices are pairwise non-adjacent and come one after another, so a
 * vertex of the i-th nonempty class (counting from the largest color, 0-based) gets a color <= i:
 * colors_out uses at most as many colors as colors_in, and repeated passes never increase the count.
 *   colors_in  int32[n], every entry >= 0 (GC_ERR_INVALID_ARG otherwise); device or host memory; it
 *              may be the same array as colors_out
 *   other arguments as gc_color_ex (mode is GC_MODE_ORDERED; opt->priority is ignored).
 */
int gc_recolor(int32_t n, const int32_t *rowptr, const int32_t *colidx, const int32_t *colors_in, uint64_t seed,
               int32_t *colors_out, int32_t *ncolors, int32_t *rounds, const gc_options *opt, gc_stats *stats);

/*
 * gc_smallest_last -- smallest-last levels by batch peeling (the ordering of
 * GC_PRIORITY_SMALLEST_LAST).  res(v) starts at deg(v) and a threshold k at 0; while vertices
 * remain, k becomes max(k, the least res among them), then, level after level, every remaining
 * vertex with res <= k is removed together and lowers res of each neighbour by one.
 *   level_out   int32[n] (device or host) receives the level (1, 2, ...) that removed each vertex
 *   nlevels     host int32* receives the number of levels (may be NULL)
 *   degeneracy  host int32* receives the largest threshold, the graph's degeneracy (may be NULL)
 *   opt         stream, spin_limit_ns and GC_FLAG_VALIDATE are used (may be NULL)
 * Errors as gc_color.
 */
int gc_smallest_last(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *level_out, int32_t *nlevels,
                     int32_t *degeneracy, const gc_options *opt);

/*
 * gc_color_batch -- color G independent graphs in one persistent launch (every graph runs
 * Algorithm 1 on its own; a round of the launch is a round of every graph still active).
 *   G          number of graphs (>= 0)
 *   vtx_off    int64[G+1]  graph g's vertices are colors_out[vtx_off[g] .. vtx_off[g+1]); vtx_off[0] = 0
 *   edge_off   int64[G+1]  graph g's neighbour ids are colidx[edge_off[g] .. edge_off[g+1]); edge_off[0] = 0
 *   rowptr     int32[vtx_off[G] + G]  graph g's own local CSR row offsets (n_g + 1 entries, starting
 *              at 0) are rowptr[vtx_off[g] + g .. vtx_off[g+1] + g]
 *   colidx     int32[edge_off[G]]     local (0-based within graph g) neighbour ids
 *   mode, seed as gc_color; the priority key uses graph-local ids, so graph g's colors equal what
 *              gc_color gives for it alone in deterministic mode
 *   colors_out int32[vtx_off[G]]  local colors per graph
 *   ncolors    int32[G]  distinct colors per graph (device or host; may be NULL)
 *   rounds     int32[G]  rounds per graph = the last round whose worklist held one of its vertices
 *              (device or host; may be NULL)
 * Totals are limited to vtx_off[G] < 2^31 vertices; edge offsets are 64-bit.
 */
int gc_color_batch(int32_t G, const int64_t *vtx_off, const int64_t *edge_off, const int32_t *rowptr,
                   const int32_t *colidx, int mode, uint64_t seed, int32_t *colors_out, int32_t *ncolors,
                   int32_t *rounds);

int gc_color_batch_ex(int32_t G, const int64_t *vtx_off, const int64_t *edge_off, const int32_t *rowptr,
                      const int32_t *colidx, int mode, uint64_t seed, int32_t *colors_out, int32_t *ncolors,
                      int32_t *rounds, const gc_options *opt, gc_stats *stats);

/*
 * gc_validate_graph -- check the graph format of Section 2.1 on the device.
 * Always checks rowptr[0] = 0, monotone rowptr, 0 <= colidx < n and no self-loops; `flags`
 * (GC_VALIDATE_*) adds sorted/duplicate-free rows and symmetry.  Returns GC_OK or
 * GC_ERR_INVALID_GRAPH (message names the first offending vertex/entry found), or an argument /
 * CUDA error.
 */
int gc_validate_graph(int32_t n, const int32_t *rowptr, const int32_t *colidx, int flags);

/*
 * gc_color_noalloc -- deterministic coloring of one graph without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot call cudaMalloc
 * (code running inside an allocator or a memory-pool callback, or under a framework that owns every
 * device allocation and forbids side allocations).  It gives exactly gc_color's deterministic
 * result, but works in a fixed scratch array built into the library (about 5.8 MB of device memory,
 * held by every GPU that has loaded the library's device code, until the process exits), so it
 * accepts at most
 * 16,384 vertices and 2^20 adjacency entries; larger graphs return GC_ERR_INVALID_ARG with the
 * outputs untouched.
 *   n, seed    as gc_color (mode is always GC_MODE_DETERMINISTIC)
 *   rowptr, colidx, colors_out   device memory of the current device (no host arrays)
 *   ncolors, rounds              host int32* (may be NULL)
 *   stream     cudaStream_t the work is queued on (NULL = the legacy default stream); the call
 *              returns after the stream has finished it
 * The first call on a device looks up the scratch array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  That first call may
 * itself allocate: CUDA loads a library's device code lazily by default, so the first call on a
 * device (or after cudaDeviceReset) is what loads this module, its scratch array and its kernels.
 * Make one call (a warm-up on any small graph) before entering the code that must not allocate;
 * later calls allocate nothing.  The call reads rowptr[n] on the host and returns only after the
 * stream has finished its work.  Every call reuses the same array and clears what must start
 * empty, so calls whose work overlaps on the GPU (from several host threads or streams at once)
 * race and must be serialised by the caller.
 */
int gc_color_noalloc(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed, int32_t *colors_out,
                     int32_t *ncolors, int32_t *rounds, void *stream);

/*
 * gc_det_round -- one round of the deterministic mode over a given list of worklist vertices, for a
 * caller that splits a graph's vertices into blocks (Algorithm 1's partitions V_1..V_p, one per GPU
 * or process) and exchanges the changed colors between rounds itself.  The mode's rounds read only
 * the colors as the round began, so the blocks can run a round independently: with the previous
 * round's new colors exchanged, the result is identical to gc_color's whatever the split.
 *   n, rowptr, colidx, seed   the whole graph and the priority seed, as gc_color
 *   colors_cur   int32[n]      C_r, every vertex's color as round r begins (C_1 = 0 for every vertex)
 *   worklist     int32[nwork]  the block's vertices on W_r (any order; each id at most once)
 *   colors_next  int32[nwork]  receives C_{r+1} of each: the least color absent from C_r over its
 *                              neighbours if it lost, else its C_r color
 *   lost         int32[nwork]  receives 1 if the vertex lost (a neighbour with the same C_r color and a
 *                              smaller key, Algorithm 1's phase 2), so it is on W_{r+1}; else 0
 * Arrays may be device or host memory.  Synchronous.  Errors: GC_ERR_INVALID_ARG (NULL arrays, a
 * worklist entry outside [0, n)), GC_ERR_INVALID_GRAPH (malformed rows or entries), GC_ERR_CUDA;
 * outputs unspecified on error.
 */
int gc_det_round(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed, const int32_t *colors_cur,
                 const int32_t *worklist, int32_t nwork, int32_t *colors_next, int32_t *lost);

/* Message for the last error on the calling thread ("" if none). Valid until the next call. */
const char *gc_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int gc_version(void);

/* Frees the calling device's cached scratch (the next call re-allocates). */
int gc_release_scratch(void);

/*
 * ---- Serving: continuous batching of independent coloring requests ----
 *
 * A server owns device memory pools of `pool_vertices` vertex slots and `pool_entries` adjacency
 * entries and a worker thread that runs rounds of the batched round kernel over every admitted
 * request.  gc_server_submit copies the request's CSR (into the pool right away when nothing waits
 * ahead of it and it fits, else into host memory) and queues it; the worker admits queued requests
 * between rounds whenever their footprint fits the free pool space (first fit), so requests that
 * arrive while others are on the GPU join the running batch at the next round boundary.  Each
 * request carries its own mode and seed: deterministic requests share one pool and launch, in-place
 * requests another (the two modes keep different vertex state); inside a pool every graph has its
 * own priority seed.  A deterministic request's colors are identical to gc_color's for the same
 * graph and seed.  A device error reported by a launch (for example a grid-barrier wait that ran
 * out) fails the requests resident in that pool with that status; the pool is reset and the server
 * keeps serving.
 */
typedef struct gc_server gc_server;

typedef struct gc_server_config {
    int64_t pool_vertices;   /* vertex capacity of each resident pool (> 0) */
    int64_t pool_entries;    /* adjacency-entry capacity of each resident pool (> 0) */
    int32_t max_requests;    /* maximum requests resident at once per pool (slots); 0 = 4096 */
    int32_t mode;            /* the pool allocated with the server: GC_MODE_DETERMINISTIC or GC_MODE_INPLACE
                                (the other mode's pool is allocated by its first request) */
    int64_t spin_limit_ns;   /* grid-barrier wait limit of the round launches; 0 = 1e9 */
    int32_t device;          /* CUDA device ordinal; -1 = current */
    int32_t solo_entries;    /* a request with at least this many adjacency entries fills the GPU by itself:
                                it skips the pool and is colored alone by the worker (as gc_color_ex
                                does, core and tail phases included) between launches of the batch;
                                0 = 2^24; < 0 = never (every request joins the batch) */
    int32_t reserved[6];
} gc_server_config;

struct gc_server_stats {
    int64_t submitted, completed, rejected;
    int64_t rounds_run;          /* batched rounds executed by the worker (both pools) */
    int64_t vertices_colored, edges_colored;  /* totals over completed requests (edges = nnz/2) */
    double p50_ms, p99_ms;       /* submit-to-done latency over completed requests */
    double busy_s;               /* wall time with at least one request resident */
    double wall_s;               /* time since the server was created */
    int32_t resident;            /* requests currently resident on the device */
    int32_t queued;              /* requests waiting for admission */
    int64_t failed;              /* requests that ended with a device error (their pool was reset) */
    int32_t reserved[4];
};

/* Creates the worker thread and the pool of cfg->mode. Errors: INVALID_ARG, OOM, CUDA. */
int gc_server_create(const gc_server_config *cfg, gc_server **out);

/* Queues one graph (host or device CSR as in gc_color; copied before return).  Non-blocking.
 *   mode   GC_MODE_DETERMINISTIC or GC_MODE_INPLACE (the request's own; see gc_color)
 *   seed   the request's priority seed (see gc_color)
 * A request with at least cfg.solo_entries entries is copied to device memory here and colored alone
 * (it needs no pool space).
 * GC_ERR_OOM if the graph can never fit a pool (or the mode's pool, or a copy of a request colored
 * alone, cannot be allocated);
 * GC_ERR_INVALID_GRAPH for malformed row offsets; GC_ERR_INVALID_ARG for an unknown mode.
 * Neighbour ids and self-loops are checked on the device when the request is admitted; a request
 * that fails that check is dropped and its gc_server_poll returns GC_ERR_INVALID_GRAPH. */
int gc_server_submit(gc_server *s, int32_t n, const int32_t *rowptr, const int32_t *colidx, int mode, uint64_t seed,
                     uint64_t *req_id);

/* Waits up to timeout_ms (0 = do not wait, <0 = forever) for request req_id.  On completion copies
 * its colors into colors_out (host or device, n entries; may be NULL), sets ncolors / rounds (host
 * pointers, may be NULL), forgets the request and returns GC_OK or the request's error status.
 * Returns GC_ERR_BUSY while it is still queued or running, GC_ERR_INVALID_ARG for an unknown id. */
int gc_server_poll(gc_server *s, uint64_t req_id, int32_t timeout_ms, int32_t *colors_out,
                   int32_t *ncolors, int32_t *rounds);

/* Counters and latency percentiles so far (gc_server_stats_get is the same call). */
int gc_server_stats(gc_server *s, struct gc_server_stats *out);
int gc_server_stats_get(gc_server *s, struct gc_server_stats *out);

/* Stops the worker (finishing resident requests), frees the pools. */
void gc_server_destroy(gc_server *s);

#ifdef __cplusplus
}
#endif

#endif /* GC_H */
