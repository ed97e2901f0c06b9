// Device helpers shared by the kernel translation units: the priority key, the bounded grid
// barrier, vertex state words, graph addressing, warp-aggregated appends, the deterministic work
// item and the per-round statistics.  Everything here has internal linkage (each translation unit
// gets its own copy).
#pragma once

#include "gc_internal.h"

namespace gc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;  // SplitMix64 state increment
constexpr int kBlock = 256;                          // round-kernel block size
constexpr int kMaxWarps = kBlock / 32;
constexpr int kPer = kStep / 32;  // entries per lane per step
#ifndef GC_MERGE_NOW_ITEMS
#define GC_MERGE_NOW_ITEMS 2  // deterministic rounds with at most this many items per warp finish
#endif                        // several-item vertices without a second barrier
constexpr unsigned kMergeNowItems = GC_MERGE_NOW_ITEMS;
// The round kernels come in two register budgets: compiled for 4 resident blocks per SM (64
// registers a thread; more warps, for graphs whose work is mostly one thread per vertex) and for 3
// (80 registers; fewer spills in the warp work-item sweep, for graphs whose entries are mostly in
// larger vertices).
constexpr int kNarrowBlocks = 4, kWideBlocks = 3;

// ------------------------------------------------------------------------------------------
// priority key: key(v) = (h(v), v), h(v) = SplitMix64 output number v of the stream `seed`
// (Steele, Lea & Flood 2014).  The top 31 bits of h are cached in the vertex's state word.

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t vertex_hash(uint64_t seed, uint32_t local) {
    return mix64(seed + (static_cast<uint64_t>(local) + 1ull) * kGamma);
}

// key(u) < key(v): u keeps its color against v.  pu, pv are the top 31 bits of h(u), h(v); the full
// hashes are recomputed only when those tie.
__device__ __forceinline__ bool key_less(uint32_t pu, uint32_t pv, uint32_t lu, uint32_t lv, uint64_t seed) {
    if (pu != pv) return pu < pv;
    const uint64_t hu = vertex_hash(seed, lu), hv = vertex_hash(seed, lv);
    if (hu != hv) return hu < hv;
    return lu < lv;
}

// The priority seed of the graph of global vertex V (batches may give each graph its own).
__device__ __forceinline__ uint64_t seed_of(const RoundParams &P, int32_t V) {
    return P.g_seed ? __ldg(P.g_seed + __ldg(P.vg + V)) : P.seed;
}

// key_less for two vertices of the graph of global vertex V: the seed is looked up only when the
// cached priority bits tie.
__device__ __forceinline__ bool key_less_in(uint32_t pu, uint32_t pv, uint32_t lu, uint32_t lv, const RoundParams &P,
                                            int32_t V) {
    if (pu != pv) return pu < pv;
    return key_less(pu, pv, lu, lv, seed_of(P, V));
}


__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void set_error(int32_t *err, int code, int32_t a, int64_t b) {
    if (atomicCAS(err, 0, code) == 0) {
        err[1] = a;
        err[2] = static_cast<int32_t>(b);
        err[3] = static_cast<int32_t>(b >> 32);
    }
}

// The 31 priority bits a vertex's state word carries; key_less compares them first and falls back
// to the full hash, then the id, only when they are equal.  GC_PRIORITY_HASH: the top 31 bits of
// h(v).  GC_PRIORITY_LARGEST_FIRST: 20 bits of 2^20 - 1 - min(deg(v), 2^20 - 1) (a larger degree
// is a smaller key), then the top 11 bits of h(v); equal bits imply equal capped degrees, so the
// fallback keeps the order (capped degree, hash, id).  GC_PRIORITY_SMALLEST_LAST and
// kPriorityRecolor: the same with P.prio_rank[V] in place of the degree (the peel level, larger
// levels first; the given color, larger colors first).
__device__ __forceinline__ uint32_t priority_bits(const RoundParams &P, uint32_t lv, int64_t deg, int32_t V) {
    const uint64_t h = vertex_hash(seed_of(P, V), lv);
    if (P.priority == kPriorityRecolor || P.priority == GC_PRIORITY_SMALLEST_LAST) {
        const int32_t c = P.prio_rank[V];
        if (c < 0) set_error(P.err, GC_ERR_INVALID_ARG, V, c);
        deg = c < 0 ? 0 : c;
    }
    if (P.priority != GC_PRIORITY_HASH) {
        constexpr uint32_t kCap = (1u << 20) - 1u;
        const uint32_t f = kCap - static_cast<uint32_t>(deg < kCap ? deg : kCap);
        return (f << 11) | static_cast<uint32_t>(h >> 53);
    }
    return static_cast<uint32_t>(h >> 33);
}

// ------------------------------------------------------------------------------------------
// bounded grid barrier

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// All blocks of the (co-resident, cooperative) grid meet here.  bar->count is zero when a launch
// starts and only grows: every block adds 1 (release) and waits (acquire) until the count reaches
// `target` += gridDim.x, so the last block to arrive has nothing more to do.  A wait gives up after
// spin_ns nanoseconds (status GC_ERR_TIMEOUT) or when it sees that a block has posted an error
// (read every 16 polls); the caller then leaves the kernel.  Returns true when the grid may
// continue: false after a timeout or once an error has been posted (at this barrier or, if it was
// posted after this block arrived, at the next one), the same for all threads of a block, so that
// the round loops need no error check of their own.
__device__ bool grid_sync(GridBar *bar, unsigned &target, int32_t *err, int64_t spin_ns) {
    __shared__ int s_ok;
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        int ok = 1;
        // the error flag is read as the block arrives, so that the read overlaps the wait; an error
        // posted after that is seen at the next barrier (or by the polling below)
        const int32_t posted = *reinterpret_cast<volatile int32_t *>(err);
        red_add_release(&bar->count, 1u);
        if (static_cast<int>(ld_acquire(&bar->count) - target) < 0) {
            const uint64_t t0 = global_ns();
            for (unsigned k = 1;; ++k) {
                __nanosleep(32);
                if (static_cast<int>(ld_acquire(&bar->count) - target) >= 0) break;
                if ((k & 15u) == 0u && *reinterpret_cast<volatile int32_t *>(err) != 0) {
                    ok = 0;
                    break;
                }
                if (static_cast<int64_t>(global_ns() - t0) > spin_ns) {
                    set_error(err, GC_ERR_TIMEOUT, static_cast<int32_t>(blockIdx.x), 0);
                    ok = 0;
                    break;
                }
            }
        }
        // an error ends the loop: read once per block, it reaches all of its threads through s_ok
        if (posted != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------------------------------------
// vertex state words

// State word: bits 0..31 color (int32, -1 = uncolored), bit 32 FINAL (the vertex left the worklist
// for good), bits 33..63 the top 31 bits of the vertex's priority hash h(v).
constexpr uint64_t kNoNeighbour = 0x000000007FFFFFFFull;  // color 2^31-1: past every window, equal to no color
constexpr uint64_t kFinalBit = 1ull << 32;

__device__ __forceinline__ uint64_t pack_state(int32_t color, uint32_t prio31, bool final_) {
    return (static_cast<uint64_t>(prio31) << 33) | (final_ ? kFinalBit : 0ull) | static_cast<uint32_t>(color);
}
__device__ __forceinline__ int32_t color_of(uint64_t w) { return static_cast<int32_t>(static_cast<uint32_t>(w)); }
__device__ __forceinline__ uint32_t prio_of(uint64_t w) { return static_cast<uint32_t>(w >> 33); }
__device__ __forceinline__ bool final_of(uint64_t w) { return (w & kFinalBit) != 0; }

// State words are loaded through L1 (ld.global.ca): the words of high-degree vertices are read by
// most rows and would otherwise concentrate on a few L2 slices.  Within a deterministic round the
// buffer being read is not written, and the acquire at the grid barrier makes the previous round's
// writes visible to these weak loads.
__device__ __forceinline__ uint64_t load_state(const uint64_t *p) {
    return __ldca(reinterpret_cast<const unsigned long long *>(p));
}

// Adjacency entries are streamed without allocating in L1, leaving L1 to the state words.
__device__ __forceinline__ int32_t load_entry(const int32_t *p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Four adjacency entries from a 16-byte aligned address, streamed the same way.
__device__ __forceinline__ int4 load_entry4(const int32_t *p) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

// Release/acquire increment of a work-item counter (orders the accumulator updates before it).
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// ------------------------------------------------------------------------------------------
// graph addressing

struct Row {
    int64_t b, e;   // entry range in colidx
    int32_t vbase;  // global id of the graph's vertex 0
    int32_t ng;     // vertices of the graph
    int32_t lv;     // local id
    int32_t g;      // graph id
};

template <bool BATCH>
__device__ __forceinline__ Row load_row(const RoundParams &P, int32_t V) {
    Row r;
    if constexpr (!BATCH) {
        r.b = __ldg(P.rowptr + V);
        r.e = __ldg(P.rowptr + V + 1);
        r.vbase = 0;
        r.ng = P.n;
        r.lv = V;
        r.g = 0;
    } else {
        const int32_t g = __ldg(P.vg + V);
        const int64_t v0 = __ldg(P.g_vbase + g);
        const int64_t e0 = __ldg(P.g_ebase + g);
        r.g = g;
        r.vbase = static_cast<int32_t>(v0);
        r.ng = __ldg(P.g_n + g);
        r.lv = V - r.vbase;
        const int32_t *rp = P.rowptr + __ldg(P.g_rbase + g);
        r.b = e0 + __ldg(rp + r.lv);
        r.e = e0 + __ldg(rp + r.lv + 1);
    }
    return r;
}

// Global id of neighbour `ul` (local id) read at entry j, or -1 after reporting a malformed entry.
__device__ __forceinline__ int32_t neighbour(const RoundParams &P, const Row &r, int32_t ul, int64_t j) {
    if (static_cast<uint32_t>(ul) >= static_cast<uint32_t>(r.ng) || ul == r.lv) {
        set_error(P.err, GC_ERR_INVALID_GRAPH, r.vbase + r.lv, j);
        return -1;
    }
    return r.vbase + ul;
}

// Warp-aggregated append of V (lanes with `take`) to list[counter].
__device__ __forceinline__ void warp_append(bool take, int32_t V, int32_t *list, unsigned *counter, int lane) {
    const unsigned m = __ballot_sync(kFull, take);
    if (m == 0) return;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(counter, static_cast<unsigned>(__popc(m)));
    base = __shfl_sync(kFull, base, leader);
    if (take) list[base + __popc(m & lanemask_lt())] = V;
}

__device__ __forceinline__ void note_graph_round(const RoundParams &P, int32_t g, int32_t round) {
    if (__ldcg(P.graph_last + g) < round) atomicMax(P.graph_last + g, round);
}

// First color not set in the window [0, 512) given as lo0/lo1 (colors 0..63) and win[2..15];
// -1 when all 512 are taken.
__device__ __forceinline__ int32_t first_free(unsigned lo0, unsigned lo1, const unsigned *win) {
    if (~lo0) return __ffs(~lo0) - 1;
    if (~lo1) return 32 + __ffs(~lo1) - 1;
#pragma unroll 1
    for (int w = 2; w < kAccWords; ++w) {
        const unsigned x = win[w];
        if (~x) return 32 * w + __ffs(~x) - 1;
    }
    return -1;
}

// Work item of a larger vertex in deterministic mode (48 bytes, kItemBytes).
struct DetItem {
    const int32_t *list;  // the vertex's list of neighbours (local ids): its CSR row or a list-pool region
    int32_t V;            // global vertex id
    uint32_t slotf;       // accumulator slot | kItemRewrite | kItemMulti
    int32_t lb, le;       // the item's entries [lb, le) of the list
    int32_t vbase, ng;    // global id of the graph's vertex 0, vertices of the graph
    int32_t nitems;       // the vertex's items this round
    int32_t deg;          // the vertex's degree
    int32_t pad[2];
};
static_assert(sizeof(DetItem) == kItemBytes, "work-item size");
constexpr uint32_t kItemRewrite = 1u << 31;  // the items also copy the entries still active to the other region
constexpr uint32_t kItemMulti = 1u << 30;    // the vertex has several items this round
constexpr uint32_t kItemSlot = kItemMulti - 1u;

__device__ __forceinline__ void store_item(DetItem *p, const int32_t *list, int32_t V, uint32_t slotf, int32_t lb,
                                           int32_t le, int32_t vbase, int32_t ng, int32_t nitems, int32_t deg) {
    const uint64_t l = reinterpret_cast<uint64_t>(list);
    int4 *q = reinterpret_cast<int4 *>(p);
    q[0] = make_int4(static_cast<int32_t>(l), static_cast<int32_t>(l >> 32), V, static_cast<int32_t>(slotf));
    q[1] = make_int4(lb, le, vbase, ng);
    q[2] = make_int4(nitems, deg, 0, 0);
}

// Word `lane` (< 10) of item i; item_of() assembles the item in every lane.
__device__ __forceinline__ uint32_t item_word(const DetItem *items, unsigned i, int lane) {
    return lane < 10 ? __ldcg(reinterpret_cast<const unsigned *>(items + i) + lane) : 0u;
}
__device__ __forceinline__ DetItem item_of(uint32_t w) {
    DetItem d;
    const uint64_t lo = __shfl_sync(kFull, w, 0), hi = __shfl_sync(kFull, w, 1);
    d.list = reinterpret_cast<const int32_t *>(lo | (hi << 32));
    d.V = static_cast<int32_t>(__shfl_sync(kFull, w, 2));
    d.slotf = __shfl_sync(kFull, w, 3);
    d.lb = static_cast<int32_t>(__shfl_sync(kFull, w, 4));
    d.le = static_cast<int32_t>(__shfl_sync(kFull, w, 5));
    d.vbase = static_cast<int32_t>(__shfl_sync(kFull, w, 6));
    d.ng = static_cast<int32_t>(__shfl_sync(kFull, w, 7));
    d.nitems = static_cast<int32_t>(__shfl_sync(kFull, w, 8));
    d.deg = static_cast<int32_t>(__shfl_sync(kFull, w, 9));
    return d;
}

// One item per lane (phase B's scan of the round's items).
__device__ __forceinline__ DetItem item_lane(const DetItem *p) {
    const int4 x = __ldcg(reinterpret_cast<const int4 *>(p));
    const int4 y = __ldcg(reinterpret_cast<const int4 *>(p) + 1);
    const int4 z = __ldcg(reinterpret_cast<const int4 *>(p) + 2);
    DetItem d;
    d.list = reinterpret_cast<const int32_t *>(static_cast<uint64_t>(static_cast<uint32_t>(x.x)) |
                                               (static_cast<uint64_t>(static_cast<uint32_t>(x.y)) << 32));
    d.V = x.z;
    d.slotf = static_cast<uint32_t>(x.w);
    d.lb = y.x;
    d.le = y.y;
    d.vbase = y.z;
    d.ng = y.w;
    d.nitems = z.x;
    d.deg = z.y;
    return d;
}

__device__ __forceinline__ uint4 ldcg4(const unsigned *p) { return __ldcg(reinterpret_cast<const uint4 *>(p)); }
__device__ __forceinline__ void stcg4(unsigned *p, uint4 v) { __stcg(reinterpret_cast<uint4 *>(p), v); }

// Least color in [base, base + 128) absent from the four window words w (-1 if all are set).
__device__ __forceinline__ int32_t first_free4(uint4 w, int32_t base) {
    if (~w.x) return base + __ffs(~w.x) - 1;
    if (~w.y) return base + 32 + __ffs(~w.y) - 1;
    if (~w.z) return base + 64 + __ffs(~w.z) - 1;
    if (~w.w) return base + 96 + __ffs(~w.w) - 1;
    return -1;
}

// Work items of the next round for a larger vertex that lost: how many, and the entries per item.
// Compact: the list splits evenly into items of about CH entries; in a round with fewer items than
// warps, into smaller ones (down to 128 entries) so that the next round is not one long item, but
// never into more items than the vertex had in round 1 (the buffers are sized for that).
__device__ __forceinline__ int32_t next_items(const RoundParams &P, int64_t len, int64_t deg, unsigned items_now,
                                              unsigned warps) {
    int64_t items = (len + P.CH - 1) / P.CH;
    if (items_now < warps) {
        int64_t chs = static_cast<int64_t>(P.CH) * items_now / warps;
        chs = chs < 128 ? 128 : (chs + 31) & ~int64_t{31};
        const int64_t cap = (deg + P.CH - 1) / P.CH;
        int64_t want = (len + chs - 1) / chs;
        if (want > cap) want = cap;
        if (want > items) items = want;
    }
    return items > 0 ? static_cast<int32_t>(items) : 1;
}

// Adds every thread's x to *dst: a block reduction, then one atomic per block (every thread of the
// block calls it).
__device__ __forceinline__ void flush_sum(unsigned long long *dst, unsigned long long x) {
    __shared__ unsigned long long s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_sum, x);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(dst, s_sum);
}

// The same for 32-bit sums.
__device__ __forceinline__ void flush_sum_u32(unsigned *dst, unsigned x) {
    __shared__ unsigned s_sum32;
    if (threadIdx.x == 0) s_sum32 = 0;
    __syncthreads();
    x = __reduce_add_sync(0xffffffffu, x);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_sum32, x);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum32) atomicAdd(dst, s_sum32);
}

// Per-round statistics of a round kernel (GC_FLAG_STATS).
__device__ __forceinline__ void flush_stats(const RoundParams &P, int pass, unsigned long long deg,
                                            unsigned long long cnt, unsigned long long reads) {
    // block-level reduction, then one atomic per block
    __shared__ unsigned long long s_deg, s_cnt, s_read;
    if (threadIdx.x == 0) {
        s_deg = 0;
        s_cnt = 0;
        s_read = 0;
    }
    __syncthreads();
    if (deg) atomicAdd(&s_deg, deg);
    if (cnt) atomicAdd(&s_cnt, cnt);
    if (reads) atomicAdd(&s_read, reads);
    __syncthreads();
    if (threadIdx.x == 0 && pass <= P.stats_cap) {
        unsigned long long *st = P.stats + 4 * (pass - 1);
        if (s_cnt) atomicAdd(st, s_cnt);
        if (s_deg) atomicAdd(st + 1, s_deg);
        atomicMax(st + 2, static_cast<unsigned long long>(global_ns()));
        if (s_read) atomicAdd(st + 3, s_read);
    }
}


// ------------------------------------------------------------------------------------------
// core phase (gc_core.cu) and its tail (gc_tail.cu)

// Record of core vertex v: kCoreRecWords words (layout in gc_internal.h).
__device__ __forceinline__ unsigned *core_rec(const CoreParams &Q, int64_t v) {
    return Q.rec + static_cast<size_t>(v) * kCoreRecWords;
}

// Least color >= start absent from the neighbours of global vertex V in C_r (warp-cooperative, full
// CSR row): a final neighbour's color from its state word, a core neighbour's from cex.  Used when
// the 512-color window of a vertex is full.
template <bool BATCH>
__device__ int32_t core_mex_from(const RoundParams &P, const uint64_t *col_r0, int32_t V, const int32_t *cex_cur,
                                 unsigned *win, int lane, int32_t start) {
    const Row r = load_row<BATCH>(P, V);
    for (int32_t base = start;; base += 32 * kAccWords) {
        if (lane < kAccWords) win[lane] = 0;
        __syncwarp();
        for (int64_t j = r.b + lane; j < r.e; j += 32) {
            const int32_t ul = __ldg(P.colidx + j);
            if (static_cast<uint32_t>(ul) >= static_cast<uint32_t>(r.ng)) continue;
            const uint64_t st = __ldcg(col_r0 + r.vbase + ul);
            const int32_t c = (final_of(st) ? color_of(st) : __ldcg(cex_cur + __ldcg(P.items + r.vbase + ul))) - base;
            if (static_cast<unsigned>(c) < 32u * kAccWords) atomicOr(&win[c >> 5], 1u << (c & 31));
        }
        __syncwarp();
        int32_t res = -1;
#pragma unroll 1
        for (int w = 0; w < kAccWords; ++w) {
            const unsigned x = win[w];
            if (~x) {
                res = base + 32 * w + __ffs(~x) - 1;
                break;
            }
        }
        __syncwarp();
        if (res >= 0) return res;
    }
}

}  // namespace
}  // namespace gc
