// Core phase of the deterministic mode (sm_103a).
//
// On power-law graphs the worklist of Algorithm 1 (Section 3.1) shrinks quickly in vertices but not
// in adjacency: the high-degree vertices keep conflicting with one another for hundreds of rounds
// (on R-MAT scale 22, ~100k vertices remain after round 22 and still hold 54M adjacency entries
// between them, 1.7G over the remaining ~330 rounds).  In the round kernel each of those entries is
// a dependent gather of a neighbour's state word from L2.  Once the worklist has at most M vertices,
// this phase numbers them 0..m-1 (the core) and rebuilds each one's row as the list of its
// neighbours that are still on the worklist, in local ids; neighbours already final never change
// again, so their colors go once into the vertex's window of final colors.  Every block then keeps
// the colors of all m core vertices in shared memory, 8 bits each (the color saturated at 255; the
// exact value of a saturated one is read from global memory) and a FINAL bit each, so a row's
// neighbour colors come from shared memory.
//
// The rule is unchanged: in round r a worklist vertex v loses iff a neighbour u with the same color
// in C_r has a smaller key, and a loser's next color is the least color absent from C_r over its
// neighbours.  The key order of each row entry is computed once, when the row is built (top bit of
// the entry: the neighbour's key is smaller).  A final neighbour never has v's color (v's color was
// chosen against it), so a vertex is re-queued only through its worklist neighbours; the window of
// final colors joins the round's window for the least free color.  Colors are double-buffered as in
// the round kernel (C_r read, C_{r+1} written), so the result is bit for bit that of the round kernel.
//
// Work decomposition.  Each row is cut once into pieces of at most kCorePiece entries (an empty row
// into one empty piece); a piece compacts itself in place (it drops neighbours found final once the
// worklist has lost half of its vertices since the piece last did).  Each round's list of
// active pieces (the pieces of its worklist vertices) is dealt to the warps round-robin.  A round
// is: refresh the shared colors of the vertices the previous round finished (its change log); every
// warp sweeps its pieces (the next piece's first entries and record words are loaded while the
// current one is consumed), and the warp that holds a vertex's last piece finishes the vertex (at
// once when it has one piece; else after the pieces' windows and flags have met in the vertex's
// record): least free color or FINAL, C_{r+1} written, the vertex batched per warp into the change
// log and, if it lost, its pieces into the next round's list; one grid barrier.
//
// Kernels: core_index_kernel (local ids, records, initial colors), core_fill_kernel (the rows),
// core_round_kernel (one persistent cooperative launch with one block per SM running the rounds
// until the worklist is small enough for the tail phase, gc_tail.cu, or empty),
// core_writeback_kernel (final colors back into the state words).
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "gc_device.cuh"

namespace gc {
namespace {

#ifndef GC_CORE_THREADS
#define GC_CORE_THREADS 768
#endif
constexpr int kCoreThreads = GC_CORE_THREADS;  // one block per SM: every block holds all m colors
constexpr int kCoreWarps = kCoreThreads / 32;
#ifndef GC_CORE_PER
#define GC_CORE_PER 8
#endif
constexpr int kCorePer = GC_CORE_PER;  // entries per lane per step of a piece
constexpr int kCoreStep = 32 * kCorePer;
constexpr unsigned kSat8 = 255u;  // 8-bit color: 255 or more (exact value in cex)
constexpr int kFillThreads = 256;
constexpr int kFillPer = 4;  // entries per lane per step of the row build

__device__ __forceinline__ unsigned sat8(int32_t c) {
    return c < static_cast<int32_t>(kSat8) ? static_cast<unsigned>(c) : kSat8;
}

// The core's colors as every block holds them in shared memory: an 8-bit color per vertex and a
// FINAL bit per vertex; entry m is a sentinel (FINAL, color 255, and not saturated: it reads as no
// color at all) that the padding slots of a step read.
struct Shared {
    uint8_t *col;   // [Mpad]
    unsigned *fin;  // [Mpad / 32 + 1]
    __device__ __forceinline__ unsigned color8(uint32_t v) const { return col[v]; }
    __device__ __forceinline__ unsigned final_bit(uint32_t v) const { return (fin[v >> 5] >> (v & 31)) & 1u; }
};


// The fill computes the core's first round (R0) as it rebuilds the rows when every color of rounds
// R0 and R0 + 1 is below 64 (colors of round r are at most r - 1): each row's 64-bit window of
// neighbour colors and its conflict flag go into the vertex's record, and the first core round only
// finishes the vertices.
__device__ __forceinline__ bool core_fused(int R0) { return R0 <= 63; }

// Worklist of the hand-over round R0 as the round kernel left it.
struct HandOver {
    int R0;
    unsigned nsmall, nchunks;
    const uint64_t *colc;   // state words round R0 reads
    const int32_t *smallc;  // vertices of degree <= T1
    const DetItem *itc;     // work items of larger vertices
};

__device__ __forceinline__ HandOver hand_over(const RoundParams &P) {
    HandOver h;
    h.R0 = __ldcg(P.passes);
    const unsigned *cc = P.cnt + kCnt * (h.R0 % 3);
    h.nsmall = __ldcg(cc + kCntSmall);
    h.nchunks = __ldcg(cc + kCntChunks);
    const bool odd = (h.R0 & 1) != 0;
    h.colc = odd ? P.col0 : P.col1;
    h.smallc = odd ? P.small0 : P.small1;
    h.itc = reinterpret_cast<const DetItem *>(odd ? P.chunk0 : P.chunk1);
    return h;
}

// Pool space for the rows of a warp's vertices (lanes with `take`, len entries each): one
// reservation per warp (one counter shared by the whole grid: an atomic per vertex would queue).
__device__ __forceinline__ unsigned long long core_reserve(const CoreParams &Q, bool take, int32_t len, int lane) {
    unsigned long long x = take ? static_cast<unsigned long long>(len) : 0ull, incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    unsigned long long b = 0;
    if (lane == 31 && incl) b = atomicAdd(Q.bump, incl);
    return __shfl_sync(kFull, b, 31) + incl - x;
}

// Record of core vertex `local` (global id V, graph g): its list at hand-over (`list`, len entries),
// its degree, the pool space `off` (len entries) for its row, its color in both buffers and the
// window of final colors found so far (`fin_src`: the round kernel's slot, or none).
__device__ void core_init_vertex(const RoundParams &P, const CoreParams &Q, int32_t local, int32_t V, int32_t g,
                                 const int32_t *list, int32_t len, int32_t deg, const uint64_t *colc,
                                 const unsigned *fin_src, unsigned long long off) {
    P.items[V] = local;  // local id of V (the set-up scratch is free once the rounds run)
    unsigned *rec = core_rec(Q, local);
    const int32_t c = color_of(__ldcg(colc + V));
    Q.cex[local] = c;
    Q.cex[Q.max_v + local] = c;
    Q.c8[local] = static_cast<uint8_t>(sat8(c));
    Q.c8[Q.max_v + local] = static_cast<uint8_t>(sat8(c));
    // hash key: the state word of round R0 carries the local id in place of the priority bits (the
    // row build then gets a neighbour's finality, color and local id in one gather and recomputes
    // the key from the id); nothing reads those bits of a worklist vertex again, and the write-back
    // rewrites the whole word
    if (P.priority == GC_PRIORITY_HASH)
        const_cast<uint64_t *>(colc)[V] = pack_state(c, static_cast<uint32_t>(local), false);
    const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int w = 0; w < 32; w += 4) stcg4(rec + w, z);
#pragma unroll
    for (int w = 0; w < kAccWords; w += 4) stcg4(rec + kAccFin + w, fin_src ? ldcg4(fin_src + w) : z);
    const uint64_t lp = reinterpret_cast<uint64_t>(list);
    stcg4(rec + kCoreOffLo, make_uint4(static_cast<unsigned>(off), static_cast<unsigned>(off >> 32),
                                       static_cast<unsigned>(deg), static_cast<unsigned>(V)));
    stcg4(rec + kCoreFill, make_uint4(0u, static_cast<unsigned>(g), static_cast<unsigned>(lp),
                                      static_cast<unsigned>(lp >> 32)));
    stcg4(rec + kCoreListLen, make_uint4(static_cast<unsigned>(len), 0u, 0u, 0u));
    stcg4(rec + 60, z);
}

// Local ids: the vertices of degree <= T1 in list order, then the larger vertices (numbered by their
// first work item).  Writes every core vertex's record and colors.
template <bool BATCH>
__global__ void core_index_kernel(RoundParams P, CoreParams Q) {
    if (__ldcg(P.core_go) == 0) return;
    const HandOver h = hand_over(P);
    const int lane = threadIdx.x & 31;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t base = t0 & ~int64_t{31}; base < h.nsmall; base += stride) {
        const int64_t i = base + lane;
        const bool in = i < h.nsmall;
        int32_t V = 0, deg = 0;
        Row r{};
        if (in) {
            V = __ldcg(h.smallc + i);
            r = load_row<BATCH>(P, V);
            deg = static_cast<int32_t>(r.e - r.b);
        }
        const unsigned long long off = core_reserve(Q, in, deg, lane);
        if (in) core_init_vertex(P, Q, static_cast<int32_t>(i), V, r.g, P.colidx + r.b, deg, deg, h.colc, nullptr, off);
    }
    for (int64_t base = t0 & ~int64_t{31}; base < h.nchunks; base += stride) {
        const int64_t i = base + lane;
        DetItem d{};
        bool first = false;
        if (i < h.nchunks) {
            d = item_lane(h.itc + i);
            first = d.lb == 0;
        }
        const unsigned mk = __ballot_sync(kFull, first);
        if (mk == 0) continue;
        unsigned b = 0;
        if (lane == 0) b = atomicAdd(Q.m, static_cast<unsigned>(__popc(mk)));
        b = __shfl_sync(kFull, b, 0);
        const unsigned *a = P.acc + static_cast<size_t>(d.slotf & kItemSlot) * kAccStride;
        const int32_t len = first ? static_cast<int32_t>(__ldcg(a + kAccLen)) : 0;
        const unsigned long long off = core_reserve(Q, first, len, lane);
        if (!first) continue;
        const int32_t local = static_cast<int32_t>(h.nsmall + b + __popc(mk & lanemask_lt()));
        const int32_t g = BATCH ? __ldg(P.vg + d.V) : 0;
        core_init_vertex(P, Q, local, d.V, g, d.list, len, d.deg, h.colc, a + kAccFin, off);
    }
}

// Rows of the core: one warp per vertex of degree <= T1 or per work item of a larger vertex (the
// round-R0 decomposition).  Every entry of the vertex's current list is read once: a final
// neighbour's color goes into the window of final colors, any other neighbour (a core vertex) is
// appended to the vertex's row as its local id with the key-order bit.  Entries are checked as in
// the round kernel (range, self-loop).  When the first round is fused (core_fused), every
// neighbour's color also goes into the record's round window and a smaller-key neighbour with the
// vertex's color sets its conflict flag.
template <bool BATCH>
__global__ void __launch_bounds__(kFillThreads) core_fill_kernel(RoundParams P, CoreParams Q) {
    __shared__ unsigned s_fin[kFillThreads / 32][kAccWords];
    if (__ldcg(P.core_go) == 0) return;
    const HandOver h = hand_over(P);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    const int64_t tasks = static_cast<int64_t>(h.nsmall) + h.nchunks;
    const unsigned m = h.nsmall + __ldcg(Q.m);
    unsigned *wfin = s_fin[wib];
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + wib; t < tasks; t += nw) {
        Row r;
        const int32_t *list;
        int64_t lb, le;
        int32_t V;
        if (t < h.nsmall) {
            V = __ldcg(h.smallc + t);
            r = load_row<BATCH>(P, V);
            list = P.colidx + r.b;
            lb = 0;
            le = r.e - r.b;
        } else {
            const DetItem d = item_of(item_word(h.itc, static_cast<unsigned>(t - h.nsmall), lane));
            V = d.V;
            r.vbase = d.vbase;
            r.ng = d.ng;
            r.lv = V - d.vbase;
            list = d.list;
            lb = d.lb;
            le = d.le;
        }
        const int32_t local = __ldcg(P.items + V);
        unsigned *rec = core_rec(Q, local);
        const bool hash_key = P.priority == GC_PRIORITY_HASH;
        const uint64_t seed = hash_key ? seed_of(P, V) : 0ull;
        const uint64_t hv = hash_key ? vertex_hash(seed, static_cast<uint32_t>(r.lv)) : 0ull;
        const uint32_t pv = hash_key ? 0u : prio_of(__ldcg(h.colc + V));
        const uint64_t off = static_cast<uint64_t>(__ldcg(rec + kCoreOffLo)) |
                             (static_cast<uint64_t>(__ldcg(rec + kCoreOffHi)) << 32);
        int32_t *dst = Q.pool + off;
        if (lane < kAccWords) wfin[lane] = 0u;
        __syncwarp();
        uint64_t flo = 0;
        const bool fused = core_fused(h.R0);
        const int32_t cv = fused ? color_of(__ldcg(h.colc + V)) : -1;  // C_R0 of the vertex
        uint64_t rlo = 0;         // fused: colors of the core neighbours (all below 64)
        unsigned conflict = 0;    // fused: a smaller-key core neighbour has the vertex's color
        for (int64_t j0 = lb; j0 < le; j0 += 32 * kFillPer) {
            int32_t ul[kFillPer];
            uint64_t st[kFillPer];
#pragma unroll
            for (int q = 0; q < kFillPer; ++q) {
                const int64_t j = j0 + lane + 32 * q;
                ul[q] = j < le ? __ldcg(list + j) : 0;
            }
#pragma unroll
            for (int q = 0; q < kFillPer; ++q) {
                const int64_t j = j0 + lane + 32 * q;
                st[q] = kNoNeighbour;  // no neighbour (past the end, or a malformed entry)
                if (j < le) {
                    const int32_t U = neighbour(P, r, ul[q], j);
                    if (U >= 0) st[q] = __ldcg(h.colc + U);
                }
            }
            int32_t loc[kFillPer];
#pragma unroll
            for (int q = 0; q < kFillPer; ++q) {
                loc[q] = -1;
                if (st[q] != kNoNeighbour && !final_of(st[q]))
                    loc[q] = hash_key ? static_cast<int32_t>(prio_of(st[q])) : __ldcg(P.items + r.vbase + ul[q]);
            }
            uint32_t ev[kFillPer];
            unsigned keepm = 0;
#pragma unroll
            for (int q = 0; q < kFillPer; ++q) {
                const int64_t j = j0 + lane + 32 * q;
                ev[q] = 0;
                if (st[q] != kNoNeighbour) {
                    if (final_of(st[q])) {
                        const int32_t c = color_of(st[q]);
                        if (static_cast<unsigned>(c) < 64u)
                            flo |= 1ull << c;
                        else if (static_cast<unsigned>(c) < 32u * kAccWords)
                            atomicOr(&wfin[c >> 5], 1u << (c & 31));
                    } else if (static_cast<unsigned>(loc[q]) < m) {
                        keepm |= 1u << q;
                        bool smaller;
                        if (hash_key) {
                            const uint64_t hu = vertex_hash(seed, static_cast<uint32_t>(ul[q]));
                            smaller = hu < hv || (hu == hv && ul[q] < r.lv);
                        } else {
                            smaller = key_less_in(prio_of(st[q]), pv, static_cast<uint32_t>(ul[q]),
                                                  static_cast<uint32_t>(r.lv), P, V);
                        }
                        ev[q] = static_cast<uint32_t>(loc[q]) | (smaller ? kCoreSmaller : 0u);
                        if (fused) {
                            const int32_t c = color_of(st[q]);
                            rlo |= 1ull << (c & 63);
                            conflict |= static_cast<unsigned>(smaller && c == cv);
                        }
                    } else {
                        // every vertex that is not final is on the worklist; anything else is a bug
                        set_error(P.err, GC_ERR_INVALID_GRAPH, V, j);
                    }
                }
            }
            // one reservation per step for the entries kept
            const unsigned kept = __reduce_add_sync(kFull, static_cast<unsigned>(__popc(keepm)));
            if (kept) {
                unsigned pos = 0;
                if (lane == 0) pos = atomicAdd(rec + kCoreFill, kept);
                pos = __shfl_sync(kFull, pos, 0);
#pragma unroll
                for (int q = 0; q < kFillPer; ++q) {
                    const bool keep = (keepm >> q) & 1u;
                    const unsigned km = __ballot_sync(kFull, keep);
                    if (keep) dst[pos + __popc(km & lanemask_lt())] = static_cast<int32_t>(ev[q]);
                    pos += __popc(km);
                }
            }
        }
        const unsigned f0 = __reduce_or_sync(kFull, static_cast<unsigned>(flo));
        const unsigned f1 = __reduce_or_sync(kFull, static_cast<unsigned>(flo >> 32));
        __syncwarp();
        const unsigned fw = lane == 0 ? f0 : lane == 1 ? f1 : (lane < kAccWords ? wfin[lane] : 0u);
        if (lane < kAccWords && fw) atomicOr(rec + kAccFin + lane, fw);
        if (fused) {
            const unsigned r0 = __reduce_or_sync(kFull, static_cast<unsigned>(rlo));
            const unsigned r1 = __reduce_or_sync(kFull, static_cast<unsigned>(rlo >> 32));
            const bool lose = __any_sync(kFull, conflict != 0u);
            if (lane == 0) {
                if (r0) atomicOr(rec, r0);
                if (r1) atomicOr(rec + 1, r1);
                if (lose) atomicOr(rec + kCoreFlag, 1u);
            }
        }
        __syncwarp();
    }
}


// Shared copy of the colors and FINAL bits of [0, m) (16-byte loads; the buffers hold a multiple of
// 16 that exceeds m), then the sentinel at m.  Ends with a block barrier.
__device__ __forceinline__ void load_shared(const Shared &S, const CoreParams &Q, const uint8_t *c8, int32_t m) {
    const int32_t n16 = (m + 15) >> 4;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(c8);
    uint4 *d4 = reinterpret_cast<uint4 *>(S.col);
    for (int32_t i = threadIdx.x; i < n16; i += blockDim.x) d4[i] = __ldcg(s4 + i);
    const int32_t nw = (m >> 5) + 1;
    for (int32_t i = threadIdx.x; i < nw; i += blockDim.x) S.fin[i] = __ldcg(Q.fbits + i);
    __syncthreads();
    if (threadIdx.x == 0) {
        S.col[m] = static_cast<uint8_t>(kSat8);
        S.fin[m >> 5] |= 1u << (m & 31);
    }
    __syncthreads();
}

// New shared colors of the vertices the previous round finished, from its change log.
__device__ __forceinline__ void apply_log(const Shared &S, const uint2 *log, unsigned n) {
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
        const uint2 x = __ldcg(log + i);
        S.col[x.x] = static_cast<uint8_t>(x.y & 0xffu);
        if (x.y >> 8) atomicOr(&S.fin[x.x >> 5], 1u << (x.x & 31));
    }
}

// A piece of a row: {local vertex, pool offset, entries, worklist size when it last dropped its FINAL
// neighbours (the hand-over's m at first)}.
struct Piece {
    int32_t v, off, cnt, flags;
};

__device__ __forceinline__ Piece piece_of(int4 x, int l) {
    Piece p;
    p.v = __shfl_sync(kFull, x.x, l);
    p.off = __shfl_sync(kFull, x.y, l);
    p.cnt = __shfl_sync(kFull, x.z, l);
    p.flags = __shfl_sync(kFull, x.w, l);
    return p;
}

// Bulk prefetch of a piece's entries into L2 (16-byte granules; the pool has 16 bytes of slack).
__device__ __forceinline__ void prefetch_piece(const CoreParams &Q, int32_t off, int32_t cnt) {
    if (cnt <= 0) return;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(Q.pool + off);
    const uintptr_t a = a0 & ~uintptr_t{15};
    const unsigned bytes = (static_cast<unsigned>(a0 - a) + 4u * static_cast<unsigned>(cnt) + 15u) & ~15u;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(bytes) : "memory");
}

// The round's active pieces a warp takes, in batches of up to 32 (one per lane).  In a round with
// few pieces they are dealt statically: entries gw, gw + nw, gw + 2 nw, ... of the round's list of
// pieces (the pieces of its worklist vertices; every piece in the first round).  In a round with many
// (at least kGrabMin per warp) each batch is taken from the round's grab counter, in chunks that
// shrink with what is left (guided self-scheduling: the pieces differ in size up to kCorePiece
// entries, and a warp that drew large ones would otherwise hold the whole grid at the barrier).
// Pieces without entries are taken too: they count towards their vertex's pieces done.
constexpr unsigned kGrabMin = 4;
struct PieceCursor {
    unsigned base;  // static: first list position of the current batch; dynamic: last grab's start
    int4 d;         // this lane's piece in the batch
    unsigned idx;   // its index
    unsigned act;   // lanes of the batch not yet taken
    unsigned *grab; // the round's grab counter (dynamic dealing), or nullptr
};

__device__ __forceinline__ void cursor_fill(PieceCursor &c, const CoreParams &Q, const int32_t *list, unsigned i,
                                            bool in, int lane) {
    c.d = make_int4(0, 0, 0, 0);
    c.idx = 0;
    if (in) {
        c.idx = list ? static_cast<unsigned>(__ldcg(list + i)) : i;
        c.d = __ldcg(Q.pieces + c.idx);
    }
    c.act = __ballot_sync(kFull, in);
    // the batch's second active piece (the first is loaded into registers right away)
    const unsigned second = c.act & (c.act - 1u);
    if (second && lane == __ffs(second) - 1) prefetch_piece(Q, c.d.y, c.d.z);
}

// The next batch: false when the round has no piece left for this warp.
__device__ __forceinline__ bool cursor_load(PieceCursor &c, const CoreParams &Q, const int32_t *list, unsigned nact,
                                            unsigned nw, int lane) {
    if (!c.grab) {
        if (c.base >= nact) return false;
        const unsigned i = c.base + static_cast<unsigned>(lane) * nw;
        cursor_fill(c, Q, list, i, i < nact, lane);
        return true;
    }
    const unsigned left = nact > c.base ? nact - c.base : 0u;
    unsigned chunk = left / (2u * nw);
    chunk = chunk < 1u ? 1u : (chunk > 32u ? 32u : chunk);
    unsigned b = 0;
    if (lane == 0) b = atomicAdd(c.grab, chunk);
    b = __shfl_sync(kFull, b, 0);
    c.base = b;
    if (b >= nact) return false;
    const unsigned i = b + static_cast<unsigned>(lane);
    cursor_fill(c, Q, list, i, static_cast<unsigned>(lane) < chunk && i < nact, lane);
    return true;
}

// Next piece of the warp (false when there is none); its index is *idx.  The piece after the next
// one in the batch is prefetched into L2 (the next one's first entries are loaded into registers).
__device__ __forceinline__ bool cursor_next(PieceCursor &c, const CoreParams &Q, const int32_t *list, unsigned nact,
                                            unsigned nw, int lane, Piece &out, unsigned &idx) {
    while (c.act == 0u) {
        if (!c.grab) c.base += 32u * nw;
        if (!cursor_load(c, Q, list, nact, nw, lane)) return false;
    }
    const int l = __ffs(c.act) - 1;
    c.act &= c.act - 1u;
    out = piece_of(c.d, l);
    idx = __shfl_sync(kFull, c.idx, l);
    const unsigned later = c.act & (c.act - 1u);  // the batch's pieces after the next one
    if (later && lane == __ffs(later) - 1) prefetch_piece(Q, c.d.y, c.d.z);
    return true;
}

// Entries j0 + lane + 32 q of a piece; slots past its end read the piece's own vertex (its color is
// the vertex's own, which a loser's window holds already -- the neighbour it lost to has it -- and
// which a winner never uses; without the key bit it is no conflict).
__device__ __forceinline__ void load_piece_step(const CoreParams &Q, const Piece &p, int32_t j0, int lane,
                                                int32_t (&e)[kCorePer]) {
#pragma unroll
    for (int q = 0; q < kCorePer; ++q) {
        const int32_t j = j0 + lane + 32 * q;
        e[q] = j < p.cnt ? __ldcg(Q.pool + p.off + j) : p.v;
    }
}

// One step of a piece: every slot's neighbour color into the round window (colors below 128 in
// two per-lane registers, the warp's shared window up to 512) and the conflict flag (an entry with
// the key bit whose neighbour has the vertex's color: tgt = cv | kCoreSmaller, never matched when cv
// is saturated).  COMPACT: also the FINAL neighbours' colors into the final window, and the slots
// kept (entries before `nvalid`, the entries of the step inside the piece, that are not FINAL).
// Saturated 8-bit colors (255) are looked up exactly in cex.
template <bool COMPACT>
__device__ __forceinline__ void consume_step(const Shared &S, const int32_t (&e)[kCorePer], uint32_t tgt, int32_t cv,
                                             const int32_t *cex_cur, uint64_t &lo, uint64_t &mid, uint64_t &flo,
                                             unsigned *win, unsigned *wfin, unsigned &conflict, int32_t nvalid,
                                             int lane, unsigned &keepm) {
    unsigned cs[kCorePer];
#pragma unroll
    for (int q = 0; q < kCorePer; ++q) cs[q] = S.color8(static_cast<uint32_t>(e[q]) & ~kCoreSmaller);
    unsigned sat = 0;
#pragma unroll
    for (int q = 0; q < kCorePer; ++q) {
        const unsigned c = cs[q];
        const uint64_t b = 1ull << (c & 63u);
        if (c < 64u) {
            lo |= b;
        } else if (c < 128u) {
            mid |= b;
        } else if (c < kSat8) {
            atomicOr(&win[c >> 5], 1u << (c & 31));
        }
        conflict |= static_cast<unsigned>(((static_cast<uint32_t>(e[q]) & kCoreSmaller) | c) == tgt);
        sat |= static_cast<unsigned>(c == kSat8) << q;
        if constexpr (COMPACT) {
            const uint32_t id = static_cast<uint32_t>(e[q]) & ~kCoreSmaller;
            const unsigned fin = S.final_bit(id);
            if (fin && c < kSat8) {
                if (c < 64u)
                    flo |= b;
                else
                    atomicOr(&wfin[c >> 5], 1u << (c & 31));
            }
            keepm |= static_cast<unsigned>(!fin && lane + 32 * q < nvalid) << q;
        }
    }
    if (sat) {
        // rare: colors of 255 and more, exactly
#pragma unroll 1
        for (int q = 0; q < kCorePer; ++q) {
            if (!((sat >> q) & 1u)) continue;
            const uint32_t id = static_cast<uint32_t>(e[q]) & ~kCoreSmaller;
            const int32_t c = __ldcg(cex_cur + id);
            if (static_cast<unsigned>(c) < 32u * kAccWords) {
                atomicOr(&win[c >> 5], 1u << (c & 31));
                if (COMPACT && S.final_bit(id)) atomicOr(&wfin[c >> 5], 1u << (c & 31));
            }
            if (e[q] < 0 && c == cv) conflict = 1u;
        }
    }
}

// Vertices a warp finished that are not yet in the round's lists: lane k holds the k-th as
// v | 8-bit color << 18 | kPendLose (v < 2^18: the core never has more vertices), and its range of
// pieces.
constexpr unsigned kPendLose = 1u << 26;

// The round's output for the vertices a warp finished: a change-log entry each (C_{r+1} and the
// FINAL flag), the losers' count and the losers' pieces (the next round's piece list); one
// reservation per list.
__device__ __forceinline__ void flush_pending(unsigned pend, unsigned pend_pb, unsigned pend_np, unsigned npend,
                                              unsigned *cn, uint2 *log_next, int32_t *act_next, int lane) {
    const bool act = static_cast<unsigned>(lane) < npend;
    const unsigned v = pend & 0x3ffffu;
    const bool lose = act && (pend & kPendLose) != 0u;
    const unsigned pb = lose ? pend_pb : 0u, npc = lose ? pend_np : 0u;
    const unsigned lm = __ballot_sync(kFull, lose);
    unsigned incl = npc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(kFull, incl, 31);
    unsigned lb = 0, ab = 0;
    if (lane == 0) {
        lb = atomicAdd(cn, npend);
        if (lm) atomicAdd(cn + 1, static_cast<unsigned>(__popc(lm)));
        if (total) ab = atomicAdd(cn + 2, total);
    }
    lb = __shfl_sync(kFull, lb, 0);
    ab = __shfl_sync(kFull, ab, 0);
    if (act) log_next[lb + lane] = make_uint2(v, ((pend >> 18) & 0xffu) | (lose ? 0u : 0x100u));
    // the losers' pieces, written by the whole warp one vertex at a time
    for (unsigned pm = __ballot_sync(kFull, npc > 0u); pm; pm &= pm - 1u) {
        const int l = __ffs(pm) - 1;
        const unsigned b0 = __shfl_sync(kFull, pb, l), k0 = __shfl_sync(kFull, npc, l);
        const unsigned at = ab + __shfl_sync(kFull, incl, l) - k0;
        for (unsigned k = lane; k < k0; k += 32) act_next[at + k] = static_cast<int32_t>(b0 + k);
    }
}

// The first core round when the fill computed it (core_fused): a lane per vertex finishes it from
// its record -- a loser takes the least color absent from the round window and the final window
// (both below 64), a winner becomes FINAL -- and clears the record's round part; the warp flushes
// its batch as core_round_warp does.
template <bool BATCH>
__device__ void core_first_round(const RoundParams &P, const CoreParams &Q, int32_t m, int pass, unsigned *cn,
                                 int lane, unsigned &st_read, unsigned &st_deg, unsigned &st_cnt) {
    const size_t cur = static_cast<size_t>(pass & 1), nxt = cur ^ 1u;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < static_cast<unsigned>(m);
         base += stride) {
        const unsigned v = base + lane;
        const bool in = v < static_cast<unsigned>(m);
        unsigned pend = 0, pend_pb = 0, pend_np = 0;
        if (in) {
            unsigned *rec = core_rec(Q, v);
            const uint4 w = ldcg4(rec);
            const uint4 f = ldcg4(rec + kAccFin);
            const bool lose = __ldcg(rec + kCoreFlag) != 0u;
            const int32_t cv = __ldcg(Q.cex + cur * Q.max_v + v);
            const uint64_t win = static_cast<uint64_t>(w.x | f.x) | (static_cast<uint64_t>(w.y | f.y) << 32);
            const int32_t nc = lose ? __ffsll(static_cast<long long>(~win)) - 1 : cv;
            const unsigned n8 = sat8(nc);
            Q.cex[nxt * Q.max_v + v] = nc;
            Q.c8[nxt * Q.max_v + v] = static_cast<uint8_t>(n8);
            if (!lose) atomicOr(Q.fbits + (v >> 5), 1u << (v & 31));
            const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int c = 0; c < 20; c += 4) stcg4(rec + c, z);
            const uint4 rr = ldcg4(rec + kCoreOffLo);  // offset lo, offset hi, degree, global id
            st_read += __ldcg(rec + kCoreFill);
            st_deg += rr.z;
            st_cnt += 1;
            if constexpr (BATCH) {
                if (lose) note_graph_round(P, static_cast<int32_t>(__ldcg(rec + kCoreG)), pass + 1);
            }
            pend = v | (n8 << 18) | (lose ? kPendLose : 0u);
            pend_pb = __ldcg(rec + kCorePcBeg);
            pend_np = __ldcg(rec + kCorePcEnd) - pend_pb;
        }
        const unsigned npend = static_cast<unsigned>(__popc(__ballot_sync(kFull, in)));
        flush_pending(pend, pend_pb, pend_np, npend, cn, Q.log + nxt * Q.max_v, Q.active + nxt * Q.max_pieces, lane);
    }
}

// One round for one warp: every active piece it owns, as one stream of steps (the next step's
// entries, possibly the next piece's first ones and its record words, are loaded before the current
// step is consumed).  For each piece: the round window (all neighbour colors), the conflict flag (a
// smaller-key neighbour with the vertex's color) and, when the piece compacts, the window of final
// colors of the neighbours it drops.  The vertex is finished by the warp that holds its last
// piece: at once for a vertex with one piece; else every piece ORs its windows and flag into the
// vertex's record and counts itself done, and the warp that completes the count reads the merged
// record.  Finishing: a loser takes the least color absent from the round window and the final
// window (its full row is rescanned past 512 colors), a winner becomes FINAL; C_{r+1} goes into the
// other color buffers (a winner's FINAL bit into the bitmap) and the vertex into the warp's pending
// batch for the change log and the next round's lists.
template <bool BATCH>
__device__ void core_round_warp(const RoundParams &P, const CoreParams &Q, const Shared &S, const int32_t *cex_cur,
                                const int32_t *list, unsigned nact, int32_t m, unsigned nv, int pass,
                                const uint64_t *col_r0, unsigned *cn, unsigned *grab, unsigned gw, unsigned nw,
                                int lane, unsigned *win, unsigned *wfin, unsigned &st_read, unsigned &st_deg,
                                unsigned &st_cnt) {
    PieceCursor cur;
    cur.act = 0;
    cur.grab = nact >= kGrabMin * nw ? grab : nullptr;
    cur.base = cur.grab ? 0u : gw;
    const size_t nxt = static_cast<size_t>((pass & 1) ^ 1);
    if (!cursor_load(cur, Q, list, nact, nw, lane)) return;
    Piece p;
    unsigned pidx = 0;
    if (!cursor_next(cur, Q, list, nact, nw, lane, p, pidx)) return;
    int32_t e[kCorePer];
    load_piece_step(Q, p, 0, lane, e);
    // words 32..63 of the piece's vertex record: final window, row fields, piece range
    unsigned rx = __ldcg(core_rec(Q, p.v) + 32 + lane);
    unsigned pend = 0, pend_pb = 0, pend_np = 0, npend = 0;
    for (;;) {
        // a piece starts: its windows, own color and compaction mode
        if (lane < kAccWords) {
            win[lane] = 0u;
            wfin[lane] = 0u;
        }
        __syncwarp();
        const unsigned own8 = S.color8(static_cast<uint32_t>(p.v));  // own color (never final on the worklist)
        const int32_t cv = own8 == kSat8 ? __ldcg(cex_cur + p.v) : static_cast<int32_t>(own8);
        // the conflict test's target: the key bit and the vertex's 8-bit color (never matched when it
        // is saturated; those are compared exactly)
        const uint32_t tgt = kCoreSmaller | (own8 == kSat8 ? 0x1000u : own8);
        // a piece drops its FINAL neighbours in place once the worklist has lost half of its vertices
        // since the piece last did (its `flags` field records that worklist size): more often costs
        // more in writes than it saves in reads (a quarter: 1% slower on R-MAT-22; never: 25%)
        const bool compact = 2ull * nv < static_cast<unsigned long long>(static_cast<unsigned>(p.flags));
        uint64_t lo = 0, mid = 0, flo = 0;
        unsigned conflict = 0;
        unsigned kept_total = 0;  // entries kept so far (the compaction position)
        int32_t j0 = 0;
        for (;;) {
            // what comes next: this piece's next step or the next active piece's first step
            Piece pn = p;
            unsigned pnidx = pidx;
            int32_t jn = j0 + kCoreStep;
            bool more = jn < p.cnt;
            unsigned rxn = rx;
            if (!more) {
                more = cursor_next(cur, Q, list, nact, nw, lane, pn, pnidx);
                jn = 0;
                if (more) rxn = __ldcg(core_rec(Q, pn.v) + 32 + lane);
            }
            int32_t en[kCorePer];
            if (more) load_piece_step(Q, pn, jn, lane, en);
            unsigned keepm = 0;
            if (compact)
                consume_step<true>(S, e, tgt, cv, cex_cur, lo, mid, flo, win, wfin, conflict, p.cnt - j0, lane, keepm);
            else
                consume_step<false>(S, e, tgt, cv, cex_cur, lo, mid, flo, win, wfin, conflict, p.cnt - j0, lane, keepm);
            const unsigned kept = compact ? __reduce_add_sync(kFull, static_cast<unsigned>(__popc(keepm))) : 0u;
            if (compact && kept) {
                // in place: the positions written never pass the ones already read
                unsigned pos = kept_total;
#pragma unroll
                for (int q = 0; q < kCorePer; ++q) {
                    const bool keep = (keepm >> q) & 1u;
                    const unsigned km = __ballot_sync(kFull, keep);
                    if (keep) Q.pool[p.off + pos + __popc(km & lanemask_lt())] = e[q];
                    pos += __popc(km);
                }
            }
            kept_total += kept;
            const bool piece_done = jn == 0 || !more;
            if (piece_done) {
                const bool lose_p = __any_sync(kFull, conflict != 0u);
                const unsigned lo0 = __reduce_or_sync(kFull, static_cast<unsigned>(lo));
                const unsigned lo1 = __reduce_or_sync(kFull, static_cast<unsigned>(lo >> 32));
                const unsigned lo2 = __reduce_or_sync(kFull, static_cast<unsigned>(mid));
                const unsigned lo3 = __reduce_or_sync(kFull, static_cast<unsigned>(mid >> 32));
                const unsigned f0 = __reduce_or_sync(kFull, static_cast<unsigned>(flo));
                const unsigned f1 = __reduce_or_sync(kFull, static_cast<unsigned>(flo >> 32));
                __syncwarp();
                unsigned *rec = core_rec(Q, p.v);
                // lanes 0..15: this piece's round window and final window; the final window as the
                // record held it when the piece started
                const unsigned rw = lane == 0 ? lo0 : lane == 1 ? lo1 : lane == 2 ? lo2 : lane == 3 ? lo3
                                  : (lane < kAccWords ? win[lane] : 0u);
                const unsigned fw = lane == 0 ? f0 : lane == 1 ? f1 : (lane < kAccWords ? wfin[lane] : 0u);
                const unsigned fold = lane < kAccWords ? rx : 0u;
                const unsigned npc = __shfl_sync(kFull, rx, kCorePcEnd - 32) - __shfl_sync(kFull, rx, kCorePcBeg - 32);
                if (lane == 0) {
                    st_read += static_cast<unsigned>(p.cnt);
                    if (compact)
                        reinterpret_cast<int2 *>(Q.pieces + pidx)[1] =
                            make_int2(static_cast<int32_t>(kept_total), static_cast<int32_t>(nv));
                }
                bool lose = lose_p, finish = true;
                unsigned tw = 0;  // lanes 0..15: colors 32 lane .. 32 lane + 31 around the vertex
                if (npc <= 1u) {
                    if (lane < kAccWords && (fw & ~fold)) rec[kAccFin + lane] = fold | fw;
                    tw = rw | fw | fold;
                } else {
                    if (lane < kAccWords && rw) atomicOr(rec + lane, rw);
                    if (lane < kAccWords && (fw & ~fold)) atomicOr(rec + kAccFin + lane, fw);
                    if (lane == 0 && lose_p) atomicOr(rec + kCoreFlag, 1u);
                    // the piece that completes the count (release: its merges first; acquire: the others')
                    __syncwarp();
                    unsigned done = 0;
                    if (lane == 0) done = atom_add_acq_rel(rec + kCoreDone, 1u);
                    done = __shfl_sync(kFull, done, 0);
                    finish = done == npc - 1u;
                    if (finish) {
                        __syncwarp();
                        const unsigned x = __ldcg(rec + lane);  // window (lanes 0..15), flag (lane 16)
                        const unsigned fx = lane < kAccWords ? __ldcg(rec + kAccFin + lane) : 0u;
                        lose = __shfl_sync(kFull, x, kCoreFlag) != 0u;
                        tw = lane < kAccWords ? (x | fx) : 0u;
                        __syncwarp();
                        if (lane <= kCoreDone) rec[lane] = 0u;  // the round part, for the next round
                    }
                }
                if (finish) {
                    const int32_t v = p.v;
                    int32_t nc = cv;
                    if (lose) {
                        const unsigned fm = __ballot_sync(kFull, lane < kAccWords && ~tw != 0u);
                        if (fm) {
                            const int l = __ffs(fm) - 1;
                            nc = 32 * l + __ffs(~__shfl_sync(kFull, tw, l)) - 1;
                        } else {
                            nc = core_mex_from<BATCH>(P, col_r0, static_cast<int32_t>(__shfl_sync(kFull, rx, kCoreGid - 32)),
                                                      cex_cur, win, lane, 32 * kAccWords);
                        }
                    }
                    const unsigned deg = __shfl_sync(kFull, rx, kCoreDeg - 32);
                    const unsigned n8 = sat8(nc);
                    if (lane == 0) {
                        Q.cex[nxt * Q.max_v + v] = nc;
                        Q.c8[nxt * Q.max_v + v] = static_cast<uint8_t>(n8);
                        if (!lose) atomicOr(Q.fbits + (v >> 5), 1u << (v & 31));  // final for good: one bitmap
                        st_deg += deg;
                        st_cnt += 1;
                    }
                    if constexpr (BATCH) {
                        const unsigned g = __shfl_sync(kFull, rx, kCoreG - 32);
                        if (lane == 0 && lose) note_graph_round(P, static_cast<int32_t>(g), pass + 1);
                    }
                    const unsigned pb = __shfl_sync(kFull, rx, kCorePcBeg - 32);
                    if (static_cast<unsigned>(lane) == npend) {
                        pend = static_cast<unsigned>(v) | (n8 << 18) | (lose ? kPendLose : 0u);
                        pend_pb = pb;
                        pend_np = npc;
                    }
                    if (++npend == 32u) {
                        flush_pending(pend, pend_pb, pend_np, npend, cn, Q.log + nxt * Q.max_v,
                                      Q.active + nxt * Q.max_pieces, lane);
                        npend = 0;
                    }
                }
                __syncwarp();
            }
            if (!more) {
                if (npend)
                    flush_pending(pend, pend_pb, pend_np, npend, cn, Q.log + nxt * Q.max_v,
                                  Q.active + nxt * Q.max_pieces, lane);
                return;
            }
            p = pn;
            pidx = pnidx;
            rx = rxn;
            j0 = jn;
#pragma unroll
            for (int q = 0; q < kCorePer; ++q) e[q] = en[q];
            if (piece_done) break;
        }
    }
}

#ifdef GC_CORE_PROFILE
// Per round (profiling builds only): earliest round start, latest refresh end, earliest / latest
// end of a block's sweep, worklist size (word 7).
__device__ unsigned long long g_core_prof[8 * 4096];
#define CORE_PROF(k, op) \
    if (threadIdx.x == 0 && pass - R0 < 4096) op(g_core_prof + 8 * (pass - R0) + (k), global_ns())
#else
#define CORE_PROF(k, op)
#endif

// Every remaining round: one cooperative launch, one block of kCoreThreads per SM, the packed
// colors of the core in dynamic shared memory.
template <bool BATCH>
__global__ void __launch_bounds__(kCoreThreads, 1) core_round_kernel(RoundParams P, CoreParams Q) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ unsigned s_win[kCoreWarps][kAccWords];
    __shared__ unsigned s_fin[kCoreWarps][kAccWords];
    if (__ldcg(P.core_go) == 0) return;
    const HandOver h = hand_over(P);
    const int R0 = h.R0;
    const int32_t m = static_cast<int32_t>(h.nsmall + __ldcg(Q.m));
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    // work is dealt to warps interleaved over the blocks, so a small round spreads over every SM
    const unsigned gw = static_cast<unsigned>(wib) * gridDim.x + blockIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // for the write-back
        Q.m[1] = static_cast<unsigned>(m);
        Q.m[3] = static_cast<unsigned>(R0);
    }
    Shared S;
    S.col = s_dyn;
    S.fin = reinterpret_cast<unsigned *>(s_dyn + Q.max_v);
    load_shared(S, Q, Q.c8 + static_cast<size_t>(R0 & 1) * Q.max_v, m);
    {
        // the pieces of every row: consecutive pieces of a row go to consecutive warps
        const unsigned stride = gridDim.x * blockDim.x;
        for (unsigned base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < static_cast<unsigned>(m);
             base += stride) {
            const unsigned v = base + lane;
            unsigned len = 0, np = 0;
            uint64_t off = 0;
            if (v < static_cast<unsigned>(m)) {
                const unsigned *rec = core_rec(Q, v);
                len = __ldcg(rec + kCoreFill);  // the row as the fill kernel wrote it
                off = static_cast<uint64_t>(__ldcg(rec + kCoreOffLo)) |
                      (static_cast<uint64_t>(__ldcg(rec + kCoreOffHi)) << 32);
                np = len ? (len + kCorePiece - 1) / kCorePiece : 1u;  // an empty row: one empty piece
            }
            unsigned incl = np;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned total = __shfl_sync(kFull, incl, 31);
            unsigned b = 0;
            if (lane == 0 && total) b = atomicAdd(Q.m + 2, total);
            b = __shfl_sync(kFull, b, 0);
            if (v < static_cast<unsigned>(m)) {
                unsigned *rec = core_rec(Q, v);
                rec[kCorePcBeg] = b + incl - np;
                rec[kCorePcEnd] = b + incl;
            }
            for (unsigned k = 0; k < np; ++k) {
                const unsigned lb = k * kCorePiece;
                Q.pieces[b + incl - np + k] =
                    make_int4(static_cast<int32_t>(v), static_cast<int32_t>(off + lb),
                              static_cast<int32_t>(min(len - lb, static_cast<unsigned>(kCorePiece))), m);
            }
        }
    }
    unsigned bar_target = 0;
    int pass = R0;
    if (grid_sync(P.bar, bar_target, P.err, P.spin_ns)) {
        const unsigned npieces = __ldcg(Q.m + 2);
        for (;; ++pass) {
            // the previous round's counts: {change-log entries, losers, pieces listed, -}
            const uint4 cc = ldcg4(Q.cnt + 4 * (pass % 3));
            unsigned *cn = Q.cnt + 4 * ((pass + 1) % 3);
            // |W_pass|: every core vertex in the first round, then the previous round's losers
            const unsigned nv = pass == R0 ? static_cast<unsigned>(m) : cc.y;
            if (nv == 0u) break;
            if (pass >= P.pass_end) {
                if (P.cap_is_error && blockIdx.x == 0 && threadIdx.x == 0)
                    set_error(P.err, GC_ERR_NO_CONVERGENCE, pass, 0);
                break;
            }
            // few enough for the tail phase (one cluster runs the remaining rounds): every block
            // reads the same count, so all leave here
            if (pass > R0 && nv <= static_cast<unsigned>(Q.tail_max)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    Q.tail[1] = static_cast<unsigned>(pass);
                    Q.tail[0] = 1u;
                }
                break;
            }
            if (blockIdx.x == 0 && threadIdx.x < 4) Q.cnt[4 * ((pass + 2) % 3) + threadIdx.x] = 0u;
            CORE_PROF(0, atomicMin);
#ifdef GC_CORE_PROFILE
            if (blockIdx.x == 0 && threadIdx.x == 0 && pass - R0 < 4096) g_core_prof[8 * (pass - R0) + 7] = nv;
#endif
            const int32_t *cex_cur = Q.cex + static_cast<size_t>(pass & 1) * Q.max_v;
            if (pass > R0) {
                // the vertices the previous round finished: its change log, or all colors when they are many
                const unsigned nprev = cc.x;
                if (8ull * nprev > static_cast<unsigned long long>(m))
                    load_shared(S, Q, Q.c8 + static_cast<size_t>(pass & 1) * Q.max_v, m);
                else
                    apply_log(S, Q.log + static_cast<size_t>(pass & 1) * Q.max_v, nprev);
            }
            __syncthreads();
            CORE_PROF(1, atomicMax);
            unsigned st_deg = 0, st_cnt = 0, st_read = 0;
            // the round's pieces: all of them in the first round, then those the previous round listed
            const int32_t *list = pass == R0 ? nullptr : Q.active + static_cast<size_t>(pass & 1) * Q.max_pieces;
            const unsigned nact = pass == R0 ? npieces : cc.z;
            // the round's grab counter: word 3 of its counter set (cleared two rounds ahead like the rest)
            if (pass == R0 && core_fused(R0))
                core_first_round<BATCH>(P, Q, m, pass, cn, lane, st_read, st_deg, st_cnt);
            else
                core_round_warp<BATCH>(P, Q, S, cex_cur, list, nact, m, nv, pass, h.colc, cn,
                                       Q.cnt + 4 * (pass % 3) + 3, gw, nw, lane, s_win[wib], s_fin[wib], st_read,
                                       st_deg, st_cnt);
#ifdef GC_CORE_PROFILE
            __syncthreads();
            CORE_PROF(2, atomicMin);
            CORE_PROF(3, atomicMax);
#endif
            if (P.stats) flush_stats(P, pass, st_deg, st_cnt, st_read);
            if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.passes[0] = pass;
        P.passes[1] = pass - 1;
    }
}

// Final colors of the core into both state buffers (FINAL set), where the color count reads them.
__global__ void core_writeback_kernel(RoundParams P, CoreParams Q) {
    if (__ldcg(P.core_go) == 0) return;
    // the round kernel rewrote passes[0]; it recorded m and the hand-over round here
    const int64_t m = __ldcg(Q.m + 1);
    // the priority bits from the buffer round R0 did not read (the other one may carry local ids)
    const uint64_t *prio_src = (__ldcg(Q.m + 3) & 1u) ? P.col1 : P.col0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t V = static_cast<int32_t>(__ldcg(core_rec(Q, i) + kCoreGid));
        const int32_t c = __ldcg(Q.cex + i);
        const uint64_t w = pack_state(c, prio_of(__ldcg(prio_src + V)), true);
        P.col0[V] = w;
        P.col1[V] = w;
    }
}

size_t core_smem_bytes(int64_t max_v) { return static_cast<size_t>(max_v) + 4 * static_cast<size_t>(max_v / 32 + 1); }

int core_static_smem(bool batch) {
    cudaFuncAttributes a{};
    const void *f = batch ? reinterpret_cast<const void *>(&core_round_kernel<true>)
                          : reinterpret_cast<const void *>(&core_round_kernel<false>);
    if (cudaFuncGetAttributes(&a, f) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return static_cast<int>(a.sharedSizeBytes);
}

}  // namespace

int32_t core_max_vertices() {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int st = std::max(core_static_smem(false), core_static_smem(true));
    if (st < 0) return 0;
    // the largest multiple of 64 vertices whose colors and FINAL bits leave one block resident per SM
    for (int64_t m = ((static_cast<int64_t>(optin) - st - 4) * 8 / 9) & ~int64_t{63}; m >= 64; m -= 1024) {
        const int smem = static_cast<int>(core_smem_bytes(m));
        bool ok = true;
        for (int b = 0; b < 2 && ok; ++b) {
            const void *f = b ? reinterpret_cast<const void *>(&core_round_kernel<true>)
                              : reinterpret_cast<const void *>(&core_round_kernel<false>);
            int per_sm = 0;
            ok = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
                 cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kCoreThreads, smem) == cudaSuccess &&
                 per_sm >= 1;
        }
        if (ok) return static_cast<int32_t>(m);
        cudaGetLastError();
    }
    return 0;
}

cudaError_t launch_core(const RoundParams &P, const CoreParams &Q, bool batch, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t smem = core_smem_bytes(Q.max_v);
    const void *round_fn = batch ? reinterpret_cast<const void *>(&core_round_kernel<true>)
                                 : reinterpret_cast<const void *>(&core_round_kernel<false>);
    e = cudaFuncSetAttribute(round_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, round_fn, kCoreThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = sms * 8;
    if (batch) {
        core_index_kernel<true><<<grid, 256, 0, s>>>(P, Q);
        core_fill_kernel<true><<<grid, kFillThreads, 0, s>>>(P, Q);
    } else {
        core_index_kernel<false><<<grid, 256, 0, s>>>(P, Q);
        core_fill_kernel<false><<<grid, kFillThreads, 0, s>>>(P, Q);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(&P.bar->count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    RoundParams pa = P;
    CoreParams qa = Q;
    void *args[] = {&pa, &qa};
#ifdef GC_CORE_PROFILE
    static unsigned long long h_prof[8 * 4096];
    for (int r = 0; r < 4096; ++r)
        for (int k = 0; k < 8; ++k) h_prof[8 * r + k] = (k == 0 || k == 2) ? ~0ull : 0ull;
    cudaMemcpyToSymbolAsync(g_core_prof, h_prof, sizeof h_prof, 0, cudaMemcpyHostToDevice, s);
#endif
    e = cudaLaunchCooperativeKernel(round_fn, dim3(sms), dim3(kCoreThreads), args, smem, s);
    if (e != cudaSuccess) return e;
    e = launch_tail(P, Q, batch, s);
    if (e != cudaSuccess) return e;
#ifdef GC_CORE_PROFILE
    cudaMemcpyFromSymbolAsync(h_prof, g_core_prof, sizeof h_prof, 0, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (const char *path = getenv("GC_CORE_PROFILE_OUT")) {
        if (FILE *f = fopen(path, "w")) {
            for (int r = 0; r < 4096 && h_prof[8 * r] != ~0ull; ++r) {
                for (int k = 0; k < 8; ++k) fprintf(f, "%llu ", h_prof[8 * r + k]);
                fprintf(f, "\n");
            }
            fclose(f);
        }
    }
#endif
    core_writeback_kernel<<<grid, 256, 0, s>>>(P, Q);
    return cudaGetLastError();
}

}  // namespace gc
