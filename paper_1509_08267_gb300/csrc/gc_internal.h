// Internal declarations shared by the library's translation units (kernels, C ABI, server).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "gc.h"

namespace gc {

// Adjacency entries a warp loads per step of a work item (kStep / 32 per lane, issued together).
#ifndef GC_STEP
#define GC_STEP 128
#endif
constexpr int kStep = GC_STEP;

// Accumulator slot of a vertex of degree > T1 (its row is split into warp work items):
//   [0, kAccWords)  round window: colors 0..511 of the neighbours read this round
//   kAccFlag        conflict flag of this round
//   kAccDone        work items of this round finished (when the last item finishes the vertex)
//   kAccSurv        compact mode: list entries whose neighbour was not final when read this round
//   kAccNewLen      compact mode: entries written to the other list region this round
// Compact mode only, kept for the whole run (the slot belongs to the vertex):
//   [kAccFin, kAccFin+kAccWords)  colors 0..511 of neighbours found final
//   kAccSrc         where the vertex's list of possibly-changing neighbours is: 0 its CSR row,
//                   1 region A, 2 region B of its space in the list pool
//   kAccLen         entries in that list
//   kAccOffLo/Hi    offset of region A in the list pool (region B follows it, each deg entries)
//   kAccDeg         the vertex's degree
// The round part (words [0, 20)) is zero whenever a round starts: only vertices with several work
// items use it, and whoever finishes such a vertex clears it.
constexpr int kAccWords = 16;
constexpr int kAccFlag = 16;
constexpr int kAccDone = 17;
constexpr int kAccSurv = 18;
constexpr int kAccNewLen = 19;
constexpr int kAccFin = 32;
constexpr int kAccSrc = 48;
constexpr int kAccLen = 49;
constexpr int kAccOffLo = 51;
constexpr int kAccOffHi = 52;
constexpr int kAccDeg = 53;
constexpr int kAccStride = 64;  // 256 B per slot
// Ordered mode: vertices of degree <= min(T1, kOrdSmall) are one thread's work; larger rows are
// split into work items of min(CH, kOrdChunk) entries; a vertex of several items merges them in an
// accumulator slot of kOrdSlotWords words (window 0..15, done counter kAccDone).
constexpr int kOrdSmall = 8;
constexpr int kOrdMid = 32;  // degree <= kOrdMid (and > the small bound): an 8-lane group each
// Priority of the recoloring pass (gc_recolor): key(v) = (-min(c(v), 2^20 - 1), h(v), v) for the
// given coloring c, the color classes in decreasing color order.
constexpr int32_t kPriorityRecolor = 3;
constexpr int kOrdChunk = 128;
constexpr int kOrdSingleChunk = 64;  // default work-item size of the ordered mode on a single graph
constexpr int kOrdSlotWords = 32;

// Worklist counters: three sets used round-robin (read / append / clear), kCnt words each.
constexpr int kCnt = 4;
//   kCntSmall   vertices of degree <= T1
//   kCntItems   larger vertices (their accumulator slots, in non-compact mode, are numbered by it)
//   kCntChunks  work items
//   kCntMulti   deterministic mode: larger vertices with more than one work item
constexpr int kCntSmall = 0, kCntItems = 1, kCntChunks = 2, kCntMulti = 3;

// Bytes per work item in the work-item buffers (deterministic items are 48 bytes, in-place 16).
constexpr size_t kItemBytes = 48;

// Grid barrier of the persistent round kernels: arrivals so far in the current launch (launch_rounds
// zeroes it before every launch).
struct alignas(128) GridBar {
    unsigned count;
    unsigned pad[31];
};

// Everything the setup, round and count kernels need.  A single graph uses plain CSR addressing;
// with BATCH the vertices of graph g are the global ids [g_vbase[g], g_vbase[g] + g_n[g]), its own
// local rowptr (g_n[g] + 1 entries) starts at rowptr[g_rbase[g]] and its local neighbour ids start at
// colidx[g_ebase[g]] (g_m[g] entries).  gc_color_batch and the server both fill this table.
struct RoundParams {
    int32_t n;    // total vertices (single graph: n)
    int32_t G;    // graphs in the table
    int64_t nnz;  // single graph: adjacency entries
    const int32_t *rowptr;
    const int32_t *colidx;
    const int64_t *g_vbase;  // [G]
    const int32_t *g_n;      // [G]
    const int64_t *g_ebase;  // [G]
    const int64_t *g_rbase;  // [G]
    const int64_t *g_m;      // [G]
    int32_t *vg;             // [n] graph id per vertex (batch)
    uint64_t seed;
    const uint64_t *g_seed;  // [G] per-graph priority seeds (the server); nullptr: `seed` for every graph

    // Vertex state words: low 32 bits = color (int32, -1 = uncolored), high 32 bits = the high half
    // of the vertex's priority hash, so one gather gives a neighbour's color and priority.
    uint64_t *col0;  // deterministic: read in odd rounds, written in even ones; in-place: the live array
    uint64_t *col1;  // deterministic: written in odd rounds
    int32_t *small0, *small1;  // thread-per-vertex worklists (two parities)
    int4 *chunk0, *chunk1;     // warp work items, kItemBytes each (two parities)
    int32_t *mid0, *mid1;      // ordered mode: medium-degree ready vertices (two parities)
    int32_t *items;            // setup scratch: larger vertices found by the binning pass
    unsigned *tmp;             // [2] setup scratch counters: larger vertices, their work items
    unsigned *cnt;             // [3][kCnt] worklist counters
    unsigned *acc;             // [slots][kAccStride]
    int32_t *lists;                   // compact mode: list pool (two regions of deg entries per larger vertex)
    unsigned long long *list_total;   // compact mode: setup adds 2 * deg of every larger vertex
    unsigned long long *list_alloc;   // compact mode: expand's allocation counter in the list pool
    int32_t slot_per_vertex;          // compact mode, 1: vertex V's slot is V and its list regions start
                                      // at 2 x its first entry (no allocation; the server's layout)
    int32_t sort_shift;               // log2 of the vertex block of the thread-worklist sort (sort_shift(n))
    unsigned *deg_hist;               // [2 * sort_bins(n)] optional: setup counts thread-per-vertex rows per
                                      // (vertex block, degree) bin, zeroed by the caller; list positions per
                                      // bin follow
    GridBar *bar;
    int32_t *err;              // [4] status, vertex, entry, extra
    int32_t *passes;           // [2] first round not executed by the last launch, last round executed
    int32_t *graph_last;       // [G] last round whose worklist held a vertex of graph g
    unsigned long long *stats; // [4 * stats_cap + 1] per round |W_r|, sum of degrees, end time (ns),
                               // adjacency entries read; last entry: start time of the launch (optional)
    int32_t stats_cap;
    int32_t pass_begin;        // first round this launch runs (the worklist of that round is current)
    int32_t pass_end;          // rounds >= pass_end are not run by this launch
    int32_t cap_is_error;      // reaching pass_end with work left is GC_ERR_NO_CONVERGENCE
    int64_t spin_ns;
    int32_t T1;  // largest degree handled by one thread
    int32_t CH;  // adjacency entries per warp work item
    int32_t priority;  // GC_PRIORITY_* or kPriorityRecolor: what the 31 priority bits of a state word hold
    const int32_t *prio_rank;  // smallest last: the peel levels; recoloring: the given coloring (int32[n])
    int32_t spread;  // in-place mode: phase 1 takes the thread worklist in a spread order (set when no
                     // vertex is past T1: the degree-sorted order then balances nothing)
    // Deterministic mode from C_1 = 0: the colors of round r are at most r - 1 (a loser's First Fit
    // color exceeds the largest color around it by at most one).  A sweep that knows its vertex loses
    // and has seen every color 0..r-1 around it knows the vertex's next color (r) and stops early.
    int32_t early_exit;
    // Hand-over to the core phase (deterministic compact mode).  core_max > 0: the round kernel stops
    // at the top of the first round whose worklist has at most core_max vertices whose lists hold at
    // most core_emax entries, and sets *core_go; the core kernels (gc_core.cu) finish the coloring.
    int32_t core_max;
    int64_t core_emax;
    unsigned long long *ecnt;  // [3] entries in the lists of each counter set's worklist (core_max > 0)
    int32_t *core_go;          // set to 1 by the round kernel when it hands over
};

// Core phase (gc_core.cu).  Once the worklist is small, its vertices get local ids 0..m-1 (the core)
// and their rows are rebuilt as lists of the local ids of neighbours still on the worklist, the
// neighbour's key order in the top bit (kCoreSmaller: smaller key than the row's vertex); the colors
// of neighbours already final go into the vertex's window of final colors.  Each round every block
// keeps the colors of all m core vertices in shared memory (8 bits each, saturated at 255, the exact
// value in cex; and a FINAL bit each), so a row's neighbour colors come from shared memory instead
// of L2.  Rows are cut once into pieces of at most kCorePiece entries, which every round's list of
// active pieces hands out to the warps.
constexpr uint32_t kCoreSmaller = 0x80000000u;
constexpr int64_t kCoreEntries = int64_t{1} << 27;  // list entries the core phase takes at most
#ifndef GC_CORE_PIECE
#define GC_CORE_PIECE 4096
#endif
constexpr int kCorePiece = GC_CORE_PIECE;
// Per core vertex, kCoreRecWords words: [0, 16) the round's window of neighbour colors 0..511,
// kCoreFlag (some smaller-key neighbour has the vertex's color), kCoreDone (pieces of the vertex done
// this round) -- the round part, used by vertices with several pieces --, [kAccFin, kAccFin + 16) the
// window of final neighbours' colors, then the row's offset in the pool, degree, global id, row
// length, graph, the hand-over list and the vertex's range of pieces.
constexpr int kCoreRecWords = 64;
constexpr int kCoreFlag = 16, kCoreDone = 17;
constexpr int kCoreOffLo = 48, kCoreOffHi = 49, kCoreDeg = 50, kCoreGid = 51, kCoreFill = 52, kCoreG = 53;
constexpr int kCoreListLo = 54, kCoreListHi = 55, kCoreListLen = 56, kCorePcBeg = 57, kCorePcEnd = 58;
constexpr int kCoreTail = 59;  // the vertex's tail id (tail phase)
// Tail phase (gc_tail.cu).  Once the core's worklist has at most tail_max vertices, one thread-block
// cluster of tail_nc blocks runs the remaining rounds: the worklist vertices get tail ids 0..k-1 in
// key order, every block keeps all k colors in shared memory and owns the rows (bitmaps over the
// tail ids) of the vertices t with t % tail_nc equal to its rank, and new colors are stored into
// every block's copy through distributed shared memory.  kTailOwned rows per block.  Default
// threshold kTailDefault: a cluster has a tenth of the GPU's SMs, so the tail pays off only once a
// round's work is small (on R-MAT scale 22: 0.3 ms saved at 256-512 vertices, less at 768, a loss
// from 1,024).
constexpr int kTailOwned = 256;
constexpr int kTailDefault = 384;
struct CoreParams {
    int32_t max_v;        // vertex capacity M (shared memory holds M 8-bit colors and M FINAL bits; a
                          // multiple of 16)
    int64_t max_e;        // list entries the core may hold (the pool's size)
    int64_t max_pieces;   // piece capacity: max_e / kCorePiece + M
    unsigned *rec;        // [M][kCoreRecWords]
    int32_t *cex;         // [2][M] exact colors, double-buffered like col0 / col1
    uint8_t *c8;          // [2][M] colors saturated at 255, double-buffered like cex
    unsigned *fbits;      // [M / 32 + 1] FINAL bit of every core vertex (zero at hand-over)
    int4 *pieces;         // [max_pieces] {local vertex, pool offset, entries, flags}
    int32_t *active;      // [2][max_pieces] the pieces of each round's worklist vertices
    uint2 *log;           // [2][M] {local vertex, 8-bit color | FINAL << 8} of the vertices a round finished
    int32_t *pool;        // [max_e] the rows
    unsigned long long *bump;  // pool allocation counter
    unsigned *cnt;        // [3][4] per-round counters: vertices finished (log entries), losers, active pieces
    unsigned *m;          // [4]: larger vertices numbered by the index kernel, m, pieces
    int32_t tail_max;     // tail phase once the worklist has at most this many vertices (0: never)
    int32_t tail_nc;      // blocks of the tail's cluster (tail_max <= kTailOwned * tail_nc)
    unsigned *tail;       // [4]: 1 when the core handed over to the tail, the tail's first round
};

// Launch wrappers (gc_kernels.cu).  All return the launch's cudaError_t.
// gc_color_batch: graph table from the offset tables, graph id per vertex, graph_last = 1 (0 if empty).
cudaError_t launch_batch_tables(const RoundParams &P, const int64_t *vtx_off, const int64_t *edge_off,
                                int64_t *g_vbase, int32_t *g_n, int64_t *g_ebase, int64_t *g_rbase, int64_t *g_m,
                                cudaStream_t s);
// Binning of vertices [v_begin, v_end) into the worklist of round P.pass_begin.  g_fixed >= 0: all
// of them belong to graph g_fixed (vg is written, and graph_last[g_fixed] is raised to pass_begin
// if any of them has a neighbour); otherwise vg must be filled already.
cudaError_t launch_setup(const RoundParams &P, int mode, bool batch, int32_t v_begin, int32_t v_end,
                         int32_t g_fixed, cudaStream_t s);
// With P.deg_hist: writes the thread-per-vertex entries of [v_begin, v_end) (counted by setup) to
// the current small list in increasing order of degree.  Without it, setup appended them already.
cudaError_t launch_sort_small(const RoundParams &P, bool batch, int32_t v_begin, int32_t v_end, cudaStream_t s);
// The thread-worklist sort's vertex-block size (log2) for n vertices, and its bins for vertex ids
// below v_end (P.deg_hist holds twice as many words).
int32_t sort_shift(int64_t n);
int32_t sort_bins(int32_t v_end, int32_t shift);
// Turns the n_items larger vertices found by setup into work items of round P.pass_begin
// (n_items < 0: the count setup left in P.tmp[0] on the device).
// compact: every larger vertex gets a persistent slot and list-pool space (deterministic mode).
cudaError_t launch_expand(const RoundParams &P, int mode, bool batch, bool compact, int32_t n_items,
                          cudaStream_t s);
// compact (deterministic mode only): larger vertices sweep packed lists of the neighbours that can
// still change instead of their whole rows.
// wide: the round-kernel variant compiled for 3 resident blocks per SM (80 registers a thread)
// instead of 4 (64): for graphs whose adjacency entries are mostly in larger vertices.
cudaError_t launch_rounds(const RoundParams &P, int mode, bool batch, bool compact, int grid, int block,
                          cudaStream_t s, bool wide = false);
cudaError_t round_kernel_occupancy(int mode, bool batch, bool compact, int block, int *blocks_per_sm,
                                   bool wide = false);
// Distinct colors and largest color per graph over vertices [v_begin, v_end) (graphs g_begin..g_end-1).
// `colors_sel` != NULL: read colors from col1 when *colors_sel is odd (the deterministic buffer
// that the last round wrote), else from col0.  `out` != NULL receives the colors of
// [v_begin, v_end) (out[0] is vertex v_begin) unless err[0] != 0.
cudaError_t launch_count_colors(const RoundParams &P, bool batch, const int32_t *colors_sel, int32_t v_begin,
                                int32_t v_end, int32_t g_begin, int32_t g_end, unsigned *bitmap, int32_t *gmax,
                                int32_t *gcount, int32_t *out, cudaStream_t s);
// Ordered mode (GC_MODE_ORDERED): after the in-place launch_setup (every vertex with neighbours
// uncolored) with P.T1 <= kOrdSmall and P.CH <= kOrdChunk, with the counter sets and P.acc's slots
// zeroed, counts each vertex's smaller-key neighbours into pend[n], lists the first ready vertices
// (small ones in small0, medium ones in mid0, work items {V, q, slot, nch} in chunk0; P.mid0/mid1
// hold n entries each) and runs the cooperative round kernel on `grid` blocks.
cudaError_t ordered_kernel_occupancy(bool batch, int block, int *blocks_per_sm);
// Smallest-last levels (single graph): launch_peel_init sets res[v] = deg(v), level[v] = 0, the two
// threshold words kw[2] and adds the work items the lists may need (vertices past kOrdMid, P.CH
// entries each) to *items; launch_peel (counter sets zeroed, P.T1 <= kOrdSmall, P.CH <= kOrdChunk,
// lists as the ordered mode's; rlist0 / rlist1 int32[n] scratch with two counters rcnt) writes
// level[v] >= 1, the number of levels to passes[0] and the degeneracy to passes[1].
cudaError_t launch_peel_init(const RoundParams &P, int32_t *res, int32_t *level, unsigned *kw, unsigned *items,
                             cudaStream_t s);
cudaError_t peel_kernel_occupancy(int block, int *blocks_per_sm);
cudaError_t launch_peel(const RoundParams &P, int32_t *res, int32_t *level, unsigned *kw, int32_t *rlist0,
                        int32_t *rlist1, unsigned *rcnt, int grid, int block, cudaStream_t s);
cudaError_t launch_ordered(const RoundParams &P, bool batch, int32_t *pend, int grid, int block, cudaStream_t s);
// Partition mode (GC_MODE_PARTITION, single graph): set-up (rows checked, colors -1, W_1 = V) and
// the cooperative round kernel with p blocks of consecutive ids.
cudaError_t launch_partition_init(const RoundParams &P, cudaStream_t s);
cudaError_t partition_kernel_occupancy(int block, int *blocks_per_sm);
cudaError_t launch_partition_rounds(const RoundParams &P, int32_t p, int grid, int block, cudaStream_t s);
cudaError_t launch_validate(int32_t n, const int32_t *rowptr, const int32_t *colidx, int flags, int32_t *err,
                            cudaStream_t s);
// gc_det_round: one fused deterministic round over the worklist vertices work[0, nwork).
cudaError_t launch_det_round_block(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed,
                                  const int32_t *cur, const int32_t *work, int32_t nwork, int32_t *next, int32_t *lost,
                                  int32_t *err, cudaStream_t s);
// Core phase (after launch_rounds handed over, *P.core_go = 1; every kernel returns at once when
// it did not): local ids and rows, the round kernel, and the final colors written back to col0 and
// col1.  core_max_vertices: the largest M the shared memory of one block per SM allows.
int32_t core_max_vertices();
cudaError_t launch_core(const RoundParams &P, const CoreParams &Q, bool batch, cudaStream_t s);
// Tail phase: the largest cluster (16 or 8 blocks) the tail kernel can run as, 0 if none; the launch
// (every block returns at once unless the core handed over).
int32_t tail_cluster_size();
cudaError_t launch_tail(const RoundParams &P, const CoreParams &Q, bool batch, cudaStream_t s);

}  // namespace gc

namespace gc {
int set_last_error(int code, const char *fmt, ...);
}
