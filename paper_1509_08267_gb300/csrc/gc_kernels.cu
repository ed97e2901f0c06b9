// Device code of the speculative coloring library (sm_103a).
//
// The method is Algorithm 1 of Singhal, Peri & Kalyanasundaram (arXiv:1509.08267, Section 3.1):
// rounds of tentative First Fit on a worklist (phase 1), a barrier, conflict detection that sends
// the loser of every monochromatic edge back to the worklist (phase 2), and a second barrier.
// Here a "partition" is a single vertex, the priority between partitions is a seeded hash, and
// the barriers are grid-wide barriers of one persistent cooperative kernel.
//
// Deterministic mode.  Round r's phase 1 reads only C_{r-1}.  Because the conflict test of round
// r and the First Fit of round r+1 both read C_r, one sweep over a worklist vertex's row does
// both: it tells whether v lost in round r and, if so, v's color for round r+1.  Colors are
// double-buffered (col0 / col1), so the result does not depend on the order of the sweep.
// In-place mode.  Phase 1 reads and writes one live color array, then a barrier, then phase 2.
//
// Work decomposition per round: vertices of degree <= T1 (<= 127) take one thread each (their First
// Fit fits a 128-bit register window because the answer is at most deg(v)); larger vertices are split into
// work items of CH adjacency entries handled by one warp each.  The items of one vertex merge
// their 512-color windows and conflict flags in an accumulator slot; the warp that finishes the
// last item computes the vertex's result.  Worklists are appended with warp-aggregated atomics.
#include <climits>

#include "gc_device.cuh"

namespace gc {
namespace {


// Least color >= start absent from the row's neighbours (warp-cooperative; mex <= deg(v) bounds it).
template <bool BATCH>
__device__ int32_t mex_from(const RoundParams &P, const uint64_t *colc, const Row &r, unsigned *win, int lane,
                            int32_t start) {
    for (int32_t base = start;; base += 32 * kAccWords) {
        if (lane < kAccWords) win[lane] = 0;
        __syncwarp();
        for (int64_t j = r.b + lane; j < r.e; j += 32) {
            const int32_t ul = __ldg(P.colidx + j);
            if (static_cast<uint32_t>(ul) >= static_cast<uint32_t>(r.ng)) continue;
            const int32_t c = color_of(load_state(colc + r.vbase + ul)) - base;
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

// Appends a larger vertex with its CH-entry work items to the next worklist (warp-uniform call).
template <bool BATCH>
__device__ __forceinline__ void append_large(const RoundParams &P, int32_t V, const Row &r, int4 *chunk_next,
                                             unsigned *cnt_next, int next_round, int lane) {
    const int32_t deg = static_cast<int32_t>(r.e - r.b);
    const int32_t nch = (deg + P.CH - 1) / P.CH;
    unsigned slot = 0, cb = 0;
    if (lane == 0) {
        slot = atomicAdd(cnt_next + kCntItems, 1u);
        cb = atomicAdd(cnt_next + kCntChunks, static_cast<unsigned>(nch));
        if constexpr (BATCH) note_graph_round(P, r.g, next_round);
    }
    slot = __shfl_sync(kFull, slot, 0);
    cb = __shfl_sync(kFull, cb, 0);
    for (int32_t q = lane; q < nch; q += 32)
        chunk_next[cb + q] = make_int4(V, q, static_cast<int32_t>(slot), nch);
}

// Issues the colidx loads of one step of a work item: entries j0 + lane + 32q, q < kPer.
__device__ __forceinline__ void load_step(const RoundParams &P, int64_t j0, int64_t je, int lane, int32_t (&ul)[kPer]) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int64_t j = j0 + lane + 32 * q;
        ul[q] = j < je ? load_entry(P.colidx + j) : 0;
    }
}

// Gathers the state words of one step's neighbours (kNoNeighbour past the end or for a bad entry).
__device__ __forceinline__ void gather_step(const RoundParams &P, const Row &r, const uint64_t *colc, int64_t j0,
                                            int64_t je, int lane, const int32_t (&ul)[kPer], uint64_t (&w)[kPer]) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int64_t j = j0 + lane + 32 * q;
        w[q] = kNoNeighbour;
        if (j < je) {
            const int32_t U = neighbour(P, r, ul[q], j);
            if (U >= 0) w[q] = load_state(colc + U);
        }
    }
}

// Accumulates one step into the lane's window [0, 64), the warp's shared window [64, 512) and the
// conflict flag (a neighbour with the same color and a smaller key).
template <bool WINDOW, bool CONFLICT>
__device__ __forceinline__ void consume_step(const uint64_t (&w)[kPer], const int32_t (&ul)[kPer], int32_t cv,
                                             uint32_t pv, uint32_t lv, const RoundParams &P, int32_t V, uint64_t &lo,
                                             unsigned *win, bool &lose) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int32_t c = color_of(w[q]);
        if constexpr (WINDOW) {
            if (static_cast<unsigned>(c) < 64u)
                lo |= 1ull << c;
            else if (static_cast<unsigned>(c) < 32u * kAccWords)
                atomicOr(&win[c >> 5], 1u << (c & 31));
        }
        if constexpr (CONFLICT) {
            if (c == cv && !lose) lose = key_less_in(prio_of(w[q]), pv, static_cast<uint32_t>(ul[q]), lv, P, V);
        }
    }
}

// Sweeps entries [jb, je) of a row with one warp, kStep entries per step, the next step's colidx
// loads issued before the current step's gathers are consumed.
template <bool WINDOW, bool CONFLICT>
__device__ __forceinline__ void sweep(const RoundParams &P, const Row &r, const uint64_t *colc, int64_t jb, int64_t je,
                                      int lane, int32_t cv, uint32_t pv, uint64_t &lo, unsigned *win, bool &lose) {
    int32_t ul[kPer], un[kPer];
    uint64_t w[kPer];
    load_step(P, jb, je, lane, ul);
    for (int64_t j0 = jb; j0 < je; j0 += kStep) {
        gather_step(P, r, colc, j0, je, lane, ul, w);
        const bool more = j0 + kStep < je;
        if (more) load_step(P, j0 + kStep, je, lane, un);
        consume_step<WINDOW, CONFLICT>(w, ul, cv, pv, static_cast<uint32_t>(r.lv), P, r.vbase + r.lv, lo, win, lose);
        if (more) {
#pragma unroll
            for (int q = 0; q < kPer; ++q) ul[q] = un[q];
        }
    }
}

// Entries [j0, j0 + 4) of colidx for a thread's row, zero at and past e: one 16-byte load when
// the group is 16-byte aligned (`vec`: colidx is, and j0 is a multiple of 4) and lies before e, else
// single loads.
__device__ __forceinline__ void load4(const int32_t *colidx, bool vec, int64_t j0, int64_t e, int32_t (&u)[4]) {
    if (vec && j0 + 3 < e) {
        const int4 v = load_entry4(colidx + j0);
        u[0] = v.x;
        u[1] = v.y;
        u[2] = v.z;
        u[3] = v.w;
    } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) u[t] = j0 + t < e ? load_entry(colidx + j0 + t) : 0;
    }
}

// The state word a neighbour (local id ul) has when round 1 of the deterministic mode reads it with
// the hash priority: color 0 (C_1), not final (only isolated vertices are, and they are nobody's
// neighbour) and the top 31 bits of its hash: recomputed from the id instead of gathered.
__device__ __forceinline__ uint64_t round1_state(uint64_t seed, int32_t ul) {
    return pack_state(0, static_cast<uint32_t>(vertex_hash(seed, static_cast<uint32_t>(ul)) >> 33), false);
}

// Per-thread sweep of a short row (degree <= T1 <= 127): window [0, 128) in two 64-bit masks (the
// least free color is at most deg(v)) and conflict flag.  Four entries per step from the aligned
// group of four that holds the row's first entry; the next step's entries are loaded before the
// current step's gathers are consumed.  `need` (colors 0..r-1 of round r, or 0): the sweep stops
// once the vertex loses and mask0 holds all of them (its next color is then r).  Returns the end of
// the entries read.
template <bool BATCH, bool WINDOW, bool CONFLICT>
__device__ __forceinline__ int64_t sweep_small(const RoundParams &P, const Row &r, const uint64_t *colc, int32_t cv,
                                               uint32_t pv, uint64_t &mask0, uint64_t &mask1, bool &lose,
                                               bool r1 = false, uint64_t r1seed = 0, uint64_t need = 0) {
    constexpr int kT = 4;  // entries per step
    const bool vec = (reinterpret_cast<uintptr_t>(P.colidx) & 15u) == 0;
    int64_t j0 = vec ? (r.b & ~int64_t{3}) : r.b;
    int32_t ul[kT], un[kT];
    if (j0 < r.e) load4(P.colidx, vec, j0, r.e, ul);
    for (; j0 < r.e; j0 += kT) {
        uint64_t w[kT];
#pragma unroll
        for (int q = 0; q < kT; ++q) {
            w[q] = kNoNeighbour;
            if (j0 + q >= r.b && j0 + q < r.e) {
                const int32_t U = neighbour(P, r, ul[q], j0 + q);
                if (U >= 0) w[q] = r1 ? round1_state(r1seed, ul[q]) : load_state(colc + U);
            }
        }
        const bool more = j0 + kT < r.e;
        if (more) load4(P.colidx, vec, j0 + kT, r.e, un);
#pragma unroll
        for (int q = 0; q < kT; ++q) {
            const int32_t c = color_of(w[q]);
            if constexpr (WINDOW) {
                if (static_cast<unsigned>(c) < 64u)
                    mask0 |= 1ull << c;
                else if (static_cast<unsigned>(c) < 128u)
                    mask1 |= 1ull << (c - 64);
            }
            if constexpr (CONFLICT) {
                if (c == cv && !lose) lose = key_less_in(prio_of(w[q]), pv, static_cast<uint32_t>(ul[q]),
                                                         static_cast<uint32_t>(r.lv), P, r.vbase + r.lv);
            }
        }
        if (need && lose && (mask0 & need) == need) return min(j0 + kT, r.e);
        if (more) {
#pragma unroll
            for (int q = 0; q < kT; ++q) ul[q] = un[q];
        }
    }
    return r.e;
}

// Least color absent from a two-mask window [0, 128) (never full for degree <= 127).
__device__ __forceinline__ int32_t first_free_128(uint64_t mask0, uint64_t mask1) {
    return ~mask0 ? __ffsll(static_cast<long long>(~mask0)) - 1 : 64 + __ffsll(static_cast<long long>(~mask1)) - 1;
}

// Merges a work item's window and flag into the vertex's accumulator slot.  Returns true in the
// warp that completed the vertex's last work item; that warp then holds the merged window in
// lo0/lo1/win, the merged flag in `lose` and the slot's survivor and new-length counters in
// surv/newlen, and the round part of the slot is cleared for the next round.
//
// `snap` is this lane's word of the slot's round part as read when the item started (0 if not
// read): bits only accumulate during a round, so bits already in the snapshot need no atomic.  When
// `fin` is set, the warp that completes the vertex also reads word 32 + lane of the slot into it
// (the window of final neighbours and the list fields), in the same round trip.
template <bool WINDOW>
__device__ __forceinline__ bool merge_item(unsigned *a, int nch, int lane, unsigned &lo0, unsigned &lo1, unsigned *win,
                                           bool &lose, unsigned snap, unsigned *surv = nullptr,
                                           unsigned *newlen = nullptr, unsigned *fin = nullptr) {
    if constexpr (WINDOW) {
        const unsigned w = lane == 0 ? lo0 : lane == 1 ? lo1 : (lane < kAccWords ? win[lane] : 0u);
        if (lane < kAccWords && (w & ~snap)) atomicOr(a + lane, w);
    }
    if (lane == 0 && lose) atomicOr(a + kAccFlag, 1u);
    __syncwarp();
    unsigned done = 0;
    if (lane == 0) done = atom_add_acq_rel(a + kAccDone, 1u);
    done = __shfl_sync(kFull, done, 0);
    if (done != static_cast<unsigned>(nch - 1)) return false;
    const unsigned x = __ldcg(a + lane);  // the round part of the slot, one word per lane
    if (fin) *fin = __ldcg(a + 32 + lane);
    if constexpr (WINDOW) {
        lo0 = __shfl_sync(kFull, x, 0);
        lo1 = __shfl_sync(kFull, x, 1);
        if (lane >= 2 && lane < kAccWords) win[lane] = x;
    }
    lose = __shfl_sync(kFull, x, kAccFlag) != 0u;
    const unsigned sv = __shfl_sync(kFull, x, kAccSurv), nl = __shfl_sync(kFull, x, kAccNewLen);
    if (surv) *surv = sv;
    if (newlen) *newlen = nl;
    __syncwarp();
    a[lane] = 0u;  // the round part of the slot (words 0..31); the persistent part stays
    return true;
}

// ------------------------------------------------------------------------------------------
// deterministic mode

// Writes a vertex's state for the next round.  A vertex that did not lose is final: its color will
// not change again, so the FINAL bit goes into both buffers (the color and priority bits are the
// ones already there, so a concurrent reader of the current buffer sees the same color either way).
__device__ __forceinline__ void det_write(const uint64_t *colc, uint64_t *coln, int32_t V, bool lose, int32_t cv,
                                          int32_t nc, uint32_t pv) {
    if (lose) {
        coln[V] = pack_state(nc, pv, false);
    } else {
        const uint64_t w = pack_state(cv, pv, true);
        coln[V] = w;
        const_cast<uint64_t *>(colc)[V] = w;
    }
}

// One vertex of degree <= T1 (one thread): did it lose in this round; writes its next state.
template <bool BATCH>
__device__ __forceinline__ bool det_small(const RoundParams &P, const uint64_t *colc, uint64_t *coln, int32_t V,
                                          int32_t &deg, int32_t &nread, bool r1, uint64_t need) {
    const Row r = load_row<BATCH>(P, V);
    deg = static_cast<int32_t>(r.e - r.b);
    const uint64_t self = load_state(colc + V);
    const int32_t cv = color_of(self);
    const uint32_t pv = prio_of(self);
    uint64_t mask0 = 0, mask1 = 0;
    bool lose = false;
    nread = static_cast<int32_t>(
        sweep_small<BATCH, true, true>(P, r, colc, cv, pv, mask0, mask1, lose, r1, r1 ? seed_of(P, V) : 0, need) -
        r.b);
    det_write(colc, coln, V, lose, cv, lose ? first_free_128(mask0, mask1) : cv, pv);
    return lose;
}


// Sweep of entries [lb, le) of a larger vertex's list with one warp, kStep entries per step (the
// first step's entries are already in ul; the next step's are loaded before the current step's
// gathers are consumed).  WINDOW: every neighbour's color goes to the round window (lo: colors
// 0..63 per lane, win: 64..511 shared by the warp).  CONFLICT: a neighbour with the same color and
// a smaller key sets `lose`.  DROP: a neighbour found final is also recorded in the window of final
// neighbours (flo / wfin) and dropped; the entries still active are counted (survivors, lane 0) and, when
// `dst` is set, copied to dst at positions from *newlen (atomically when `shared_len`, else lane 0's
// running count `written`).  `need` (colors 0..r-1 of round r, or 0; never with dst): the sweep
// stops once some lane has the conflict and the warp's window with `fin64` (final colors 0..63
// known before) holds all of them -- the vertex's next color is then r; the entries not read count
// as survivors.  Returns the end of the entries read.
template <bool DROP, bool WINDOW = true, bool CONFLICT = true>
__device__ __forceinline__ int64_t sweep_item(const RoundParams &P, const Row &r, const uint64_t *colc,
                                              const int32_t *list, int64_t lb, int64_t le, int32_t (&ul)[kPer],
                                              int32_t *dst, unsigned *newlen, bool shared_len, int lane, int32_t cv,
                                              uint32_t pv, uint64_t &lo, unsigned *win, uint64_t &flo, unsigned *wfin,
                                              bool &lose, unsigned &survivors, unsigned &written, bool r1 = false,
                                              uint64_t r1seed = 0, uint64_t need = 0, uint64_t fin64 = 0) {
    int32_t un[kPer];
    uint64_t w[kPer];
    for (int64_t j0 = lb; j0 < le; j0 += kStep) {
        unsigned keepm = 0;  // DROP: bit q, entry q of this lane stays on the list
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int64_t j = j0 + lane + 32 * q;
            w[q] = kNoNeighbour;
            if (j < le) {
                const int32_t U = neighbour(P, r, ul[q], j);
                if (U >= 0) w[q] = r1 ? round1_state(r1seed, ul[q]) : load_state(colc + U);
            }
        }
        const bool more = j0 + kStep < le;
        if (more) {
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int64_t j = j0 + kStep + lane + 32 * q;
                un[q] = j < le ? __ldcg(list + j) : 0;
            }
        }
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int32_t c = color_of(w[q]);
            const bool fin = DROP && j0 + lane + 32 * q < le && final_of(w[q]);
            if constexpr (WINDOW) {
                if (static_cast<unsigned>(c) < 64u) {
                    lo |= 1ull << c;
                    if (fin) flo |= 1ull << c;
                } else if (static_cast<unsigned>(c) < 32u * kAccWords) {
                    atomicOr(&win[c >> 5], 1u << (c & 31));
                    if (fin) atomicOr(&wfin[c >> 5], 1u << (c & 31));
                }
            } else if (fin) {
                if (static_cast<unsigned>(c) < 64u)
                    flo |= 1ull << c;
                else if (static_cast<unsigned>(c) < 32u * kAccWords)
                    atomicOr(&wfin[c >> 5], 1u << (c & 31));
            }
            if constexpr (CONFLICT) {
                if (c == cv && !lose) lose = key_less_in(prio_of(w[q]), pv, static_cast<uint32_t>(ul[q]),
                                                         static_cast<uint32_t>(r.lv), P, r.vbase + r.lv);
            }
            if constexpr (DROP) {
                if (j0 + lane + 32 * q < le && !fin) keepm |= 1u << q;
            }
        }
        if constexpr (DROP) {
            // entries still active: counted, and in a rewrite round copied with one reservation per step
            const unsigned kept = __reduce_add_sync(kFull, static_cast<unsigned>(__popc(keepm)));
            if (lane == 0) survivors += kept;
            if (dst && kept) {
                unsigned pos = 0;
                if (lane == 0) {
                    if (shared_len) {
                        pos = atomicAdd(newlen, kept);
                    } else {
                        pos = written;
                        written += kept;
                    }
                }
                pos = __shfl_sync(kFull, pos, 0);
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const bool keep = (keepm >> q) & 1u;
                    const unsigned km = __ballot_sync(kFull, keep);
                    if (keep) dst[pos + __popc(km & lanemask_lt())] = ul[q];
                    pos += __popc(km);
                }
            }
        }
        if (need && __any_sync(kFull, lose)) {
            const uint64_t wl = (static_cast<uint64_t>(__reduce_or_sync(kFull, static_cast<unsigned>(lo >> 32))) << 32 |
                                 __reduce_or_sync(kFull, static_cast<unsigned>(lo))) |
                                fin64;
            if ((wl & need) == need) {
                const int64_t jend = min(le, j0 + kStep);
                if (DROP && lane == 0) survivors += static_cast<unsigned>(le - jend);
                return jend;
            }
        }
        if (more) {
#pragma unroll
            for (int q = 0; q < kPer; ++q) ul[q] = un[q];
        }
    }
    return le;
}

// Appends the next round's items of the vertices that lost in lanes with items_l > 0 (one
// warp-aggregated reservation).  slot_l: the lane's slot (compact), or -1 to take a new slot from
// the next round's count of larger vertices.  per_l: entries per item (the list splits into
// [q * per_l, min(len_l, (q + 1) * per_l))).
__device__ __forceinline__ void append_items(DetItem *next, unsigned *cnt_next, int lane, int32_t items_l,
                                             const int32_t *list_l, int32_t V, int64_t slot_l, uint32_t flags_l,
                                             int64_t len_l, int64_t per_l, int32_t vbase, int32_t ng, int32_t deg,
                                             unsigned long long *ent = nullptr) {
    const bool take = items_l > 0;
    const unsigned m = __ballot_sync(kFull, take);
    if (m == 0) return;
    // the list entries of the next worklist, added up per thread (the core hand-over reads them)
    if (ent && take) *ent += static_cast<unsigned long long>(len_l);
    unsigned incl = take ? static_cast<unsigned>(items_l) : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(kFull, incl, 31);
    const unsigned mm = __ballot_sync(kFull, items_l > 1);
    unsigned cb = 0, sb = 0;
    if (lane == 0) {
        sb = atomicAdd(cnt_next + kCntItems, static_cast<unsigned>(__popc(m)));
        cb = atomicAdd(cnt_next + kCntChunks, total);
        if (mm) atomicAdd(cnt_next + kCntMulti, static_cast<unsigned>(__popc(mm)));
    }
    cb = __shfl_sync(kFull, cb, 0);
    sb = __shfl_sync(kFull, sb, 0);
    if (!take) return;
    const uint32_t slot = slot_l >= 0 ? static_cast<uint32_t>(slot_l) : sb + __popc(m & lanemask_lt());
    const uint32_t slotf = slot | flags_l | (items_l > 1 ? kItemMulti : 0u);
    DetItem *out = next + cb + (incl - static_cast<unsigned>(items_l));
    for (int32_t q = 0; q < items_l; ++q) {
        const int64_t lb = static_cast<int64_t>(q) * per_l;
        const int64_t le = min(len_l, lb + per_l);
        store_item(out + q, list_l, V, slotf, static_cast<int32_t>(lb), static_cast<int32_t>(le), vbase, ng, items_l,
                   deg);
    }
}

// Finishes larger vertices whose items merged into their slots, one lane per vertex (lanes with
// `fin`; d = any item of the vertex): reads the merged slot, takes the least free color if the
// vertex lost, writes its state, clears the slot's round part and appends its next items.
template <bool BATCH, bool COMPACT>
__device__ __forceinline__ void det_finish(const RoundParams &P, const uint64_t *colc, uint64_t *coln, bool fin,
                                           const DetItem &d, unsigned *win, DetItem *next, unsigned *cnt_next,
                                           int pass, int lane, unsigned items_now, unsigned warps,
                                           unsigned &st_deg, unsigned &st_cnt, unsigned long long &st_ent) {
    const int32_t V = d.V;
    const uint32_t slot = d.slotf & kItemSlot;
    const int64_t deg = d.deg;
    unsigned *a = P.acc + static_cast<size_t>(slot) * kAccStride;
    uint4 st = make_uint4(0, 0, 0, 0), m0 = st, m1 = st;
    uint4 w[kAccWords / 4];
    uint64_t self = 0;
    if (fin) {
        self = load_state(colc + V);
        st = ldcg4(a + kAccFlag);  // flag, item count, survivors, new length
        if (COMPACT) {
            m0 = ldcg4(a + kAccSrc);    // src, len, (unused), offset lo
            m1 = ldcg4(a + kAccOffHi);  // offset hi, degree
        }
#pragma unroll
        for (int c = 0; c < kAccWords / 4; ++c) {
            w[c] = ldcg4(a + 4 * c);
            if (COMPACT) {
                const uint4 f = ldcg4(a + kAccFin + 4 * c);
                w[c].x |= f.x;
                w[c].y |= f.y;
                w[c].z |= f.z;
                w[c].w |= f.w;
            }
        }
    }
    const bool lose = fin && st.x != 0u;
    const bool pick = lose;
    const int32_t cv = color_of(self);
    const uint32_t pv = prio_of(self);
    int32_t nc = cv;
    if (pick) {
        nc = -1;
#pragma unroll
        for (int c = 0; c < kAccWords / 4; ++c)
            if (nc < 0) nc = first_free4(w[c], 128 * c);
    }
    // rare: all of colors 0..511 taken; the warp rescans each such row in full
    unsigned need = __ballot_sync(kFull, pick && nc < 0);
    while (need) {
        const int l = __ffs(need) - 1;
        need &= need - 1;
        Row rl = load_row<BATCH>(P, __shfl_sync(kFull, V, l));
        const int32_t x = mex_from<BATCH>(P, colc, rl, win, lane, 32 * kAccWords);
        if (lane == l) nc = x;
    }
    if (fin) {
        det_write(colc, coln, V, lose, cv, nc, pv);
        st_deg += static_cast<unsigned>(deg);
        st_cnt += 1;
        const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int c = 0; c < 20; c += 4) stcg4(a + c, z);
    }
    if constexpr (BATCH) {
        if (lose) note_graph_round(P, __ldg(P.vg + V), pass + 1);
    }
    int32_t items = 0;
    const int32_t *list = d.list;
    int64_t len = deg, per = P.CH;
    uint32_t flags = 0;
    if (lose) {
        if constexpr (COMPACT) {
            const unsigned src = m0.x, olen = m0.y;
            const bool rewrite = (d.slotf & kItemRewrite) != 0;
            const int64_t off = static_cast<int64_t>(m0.w) | (static_cast<int64_t>(m1.x) << 32);
            const unsigned nsrc = rewrite ? (src == 1 ? 2u : 1u) : src;
            const unsigned nlen = rewrite ? st.w : olen;
            flags = 8ull * st.z < 7ull * nlen ? kItemRewrite : 0u;
            items = next_items(P, nlen, deg, items_now, warps);
            a[kAccSrc] = nsrc;
            a[kAccLen] = nlen;
            if (nsrc != src) list = P.lists + off + (nsrc == 2 ? deg : 0);
            len = nlen;
            per = (len + items - 1) / items;
            if (per < 1) per = 1;
        } else {
            items = static_cast<int32_t>((deg + P.CH - 1) / P.CH);
        }
    }
    append_items(next, cnt_next, lane, items, list, V, COMPACT ? static_cast<int64_t>(slot) : -1, flags, len, per,
                 d.vbase, d.ng, static_cast<int32_t>(deg), &st_ent);
}

// Phase A, one work item of a larger vertex (one warp).  A vertex with one item is finished here.
// The items of a vertex with several merge their windows, conflict flag and (compact) final window
// and list counts into its slot with atomics; then either phase B finishes the vertex after the
// grid barrier (`merge_now` false: rounds with many items per warp, where no item waits for
// another), or the item that completes the slot's count finishes it at once (`merge_now`: sparse
// rounds, where the extra barrier would cost more than the wait).
template <bool BATCH, bool COMPACT>
__device__ void det_item(const RoundParams &P, const uint64_t *colc, uint64_t *coln, const DetItem &d,
                         unsigned *win, unsigned *wfin, unsigned *snap, DetItem *next, unsigned *cnt_next, int pass,
                         int lane, unsigned items_now, unsigned warps, bool merge_now, unsigned &st_deg,
                         unsigned &st_cnt, unsigned &st_read, bool r1, unsigned long long &st_ent, uint64_t need) {
    const int32_t V = d.V;
    const uint32_t slot = d.slotf & kItemSlot;
    const bool multi = (d.slotf & kItemMulti) != 0;
    unsigned *a = P.acc + static_cast<size_t>(slot) * kAccStride;
    Row r;
    r.b = 0;
    r.e = 0;
    r.vbase = d.vbase;
    r.ng = d.ng;
    r.lv = V - d.vbase;
    r.g = 0;
    // the first step's entries, the vertex's state and its slot: one round trip
    int32_t ul[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int64_t j = static_cast<int64_t>(d.lb) + lane + 32 * q;
        ul[q] = j < d.le ? __ldcg(d.list + j) : 0;
    }
    const uint64_t self = load_state(colc + V);
    const unsigned x = multi ? __ldcg(a + lane) : 0u;
    const unsigned sm = COMPACT ? __ldcg(a + 32 + lane) : 0u;
    if (lane < kAccWords) {
        win[lane] = 0;
        snap[lane] = x;
        if (COMPACT) {
            wfin[lane] = 0;
            snap[kAccWords + lane] = sm;
        }
    }
    const int32_t cv = color_of(self);
    const uint32_t pv = prio_of(self);
    const int64_t deg = d.deg;
    int32_t *dst = nullptr;
    unsigned src = 0, len = 0;
    int64_t off = 0;
    if constexpr (COMPACT) {
        src = __shfl_sync(kFull, sm, kAccSrc - 32);
        len = __shfl_sync(kFull, sm, kAccLen - 32);
        off = static_cast<int64_t>(__shfl_sync(kFull, sm, kAccOffLo - 32)) |
              (static_cast<int64_t>(__shfl_sync(kFull, sm, kAccOffHi - 32)) << 32);
        if (d.slotf & kItemRewrite) dst = P.lists + off + (src == 1 ? deg : 0);
    }
    __syncwarp();
    uint64_t lo = 0, flo = 0;
    bool lose = false;
    unsigned survivors = 0, written = 0;
    // final colors 0..63 already in the slot (lanes 0 and 1 hold them)
    const uint64_t fin64 = COMPACT ? (static_cast<uint64_t>(__shfl_sync(kFull, sm, 1)) << 32 | __shfl_sync(kFull, sm, 0))
                                   : 0ull;
    const int64_t jend = sweep_item<COMPACT, true, true>(P, r, colc, d.list, d.lb, d.le, ul, dst, a + kAccNewLen, multi,
                                                         lane, cv, pv, lo, win, flo, wfin, lose, survivors, written,
                                                         r1, r1 ? seed_of(P, V) : 0, dst ? 0ull : need, fin64);
    if (lane == 0) st_read += static_cast<unsigned>(jend - d.lb);
    lose = __any_sync(kFull, lose);
    unsigned lo0 = __reduce_or_sync(kFull, static_cast<unsigned>(lo));
    unsigned lo1 = __reduce_or_sync(kFull, static_cast<unsigned>(lo >> 32));
    unsigned f0 = 0, f1 = 0;
    if constexpr (COMPACT) {
        f0 = __reduce_or_sync(kFull, static_cast<unsigned>(flo));
        f1 = __reduce_or_sync(kFull, static_cast<unsigned>(flo >> 32));
    }
    __syncwarp();
    if (multi) {
        // into the slot; bits already in the snapshot need no atomic (bits only accumulate)
        if constexpr (COMPACT) {
            const unsigned fw = lane == 0 ? f0 : lane == 1 ? f1 : (lane < kAccWords ? wfin[lane] : 0u);
            if (lane < kAccWords && (fw & ~snap[kAccWords + lane])) atomicOr(a + kAccFin + lane, fw);
            if (lane == 0 && survivors) atomicAdd(a + kAccSurv, survivors);
        }
        const unsigned w = lane == 0 ? lo0 : lane == 1 ? lo1 : (lane < kAccWords ? win[lane] : 0u);
        if (lane < kAccWords && (w & ~snap[lane])) atomicOr(a + lane, w);
        if (lane == 0 && lose) atomicOr(a + kAccFlag, 1u);
        if (!merge_now) return;
        // the item that completes the count (release: its merges first; acquire: the others')
        __syncwarp();
        unsigned done = 0;
        if (lane == 0) done = atom_add_acq_rel(a + kAccDone, 1u);
        done = __shfl_sync(kFull, done, 0);
        if (done != static_cast<unsigned>(d.nitems - 1)) return;
        det_finish<BATCH, COMPACT>(P, colc, coln, lane == 0, d, win, next, cnt_next, pass, lane, items_now, warps,
                                   st_deg, st_cnt, st_ent);
        return;
    }
    // the vertex's only item: its result now
    if (lane == 0) {
        st_deg += static_cast<unsigned>(deg);
        st_cnt += 1;
    }
    if constexpr (COMPACT) {
        // round window + colors of every neighbour known to be final (kept in the slot)
        const unsigned fold = lane < kAccWords ? snap[kAccWords + lane] : 0u;
        const unsigned fx = fold | (lane == 0 ? f0 : lane == 1 ? f1 : (lane < kAccWords ? wfin[lane] : 0u));
        if (lane < kAccWords && fx != fold) a[kAccFin + lane] = fx;
        lo0 |= __shfl_sync(kFull, fx, 0);
        lo1 |= __shfl_sync(kFull, fx, 1);
        if (lane >= 2 && lane < kAccWords) win[lane] |= fx;
        __syncwarp();
    }
    int32_t nc = cv;
    if (lose) {
        nc = first_free(lo0, lo1, win);
        if (nc < 0) nc = mex_from<BATCH>(P, colc, load_row<BATCH>(P, V), win, lane, 32 * kAccWords);
    }
    if (lane == 0) det_write(colc, coln, V, lose, cv, nc, pv);
    if (!lose) return;
    if constexpr (BATCH) {
        if (lane == 0) note_graph_round(P, __ldg(P.vg + V), pass + 1);
    }
    if constexpr (COMPACT) {
        // next round's list: the fresh copy if this round wrote one; a rewrite next round once an
        // eighth of the list has become final (a quarter or a half: 0.8% and 0.2% slower on R-MAT-22
        // with the core phase, 3% and 13% without)
        const bool rewrite = dst != nullptr;
        const unsigned nsrc = rewrite ? (src == 1 ? 2u : 1u) : src;
        const unsigned nlen = rewrite ? __shfl_sync(kFull, written, 0) : len;
        const unsigned surv = __shfl_sync(kFull, survivors, 0);
        const bool nrw = 8ull * surv < 7ull * nlen;
        const int32_t items = next_items(P, nlen, deg, items_now, warps);
        if (lane == 0) {
            a[kAccSrc] = nsrc;
            a[kAccLen] = nlen;
        }
        const int32_t *list = nsrc == 0 ? d.list : P.lists + off + (nsrc == 2 ? deg : 0);
        const int64_t per = (static_cast<int64_t>(nlen) + items - 1) / items;
        append_items(next, cnt_next, lane, lane == 0 ? items : 0, list, V, slot, nrw ? kItemRewrite : 0u, nlen,
                     per > 0 ? per : 1, d.vbase, d.ng, d.deg, &st_ent);
    } else {
        append_items(next, cnt_next, lane, lane == 0 ? 1 : 0, d.list, V, -1, 0u, deg, P.CH, d.vbase, d.ng, d.deg);
    }
}

// ------------------------------------------------------------------------------------------
// in-place mode

// Phase 1 for a vertex of degree <= T1: First Fit over the live colors.
template <bool BATCH>
__device__ __forceinline__ void ip_small_assign(const RoundParams &P, uint64_t *col, int32_t V) {
    const Row r = load_row<BATCH>(P, V);
    uint64_t mask0 = 0, mask1 = 0;
    bool unused = false;
    sweep_small<BATCH, true, false>(P, r, col, 0, 0, mask0, mask1, unused);
    const uint32_t pv = prio_of(load_state(col + V));
    col[V] = pack_state(first_free_128(mask0, mask1), pv, false);
}

// Phase 2 for a vertex of degree <= T1.  FINAL: a vertex that does not lose marks itself final
// (the compact sweep drops final neighbours from lists).
template <bool BATCH, bool FINAL = false>
__device__ __forceinline__ bool ip_small_conflict(const RoundParams &P, uint64_t *col, int32_t V, int32_t &deg) {
    const Row r = load_row<BATCH>(P, V);
    deg = static_cast<int32_t>(r.e - r.b);
    const uint64_t self = load_state(col + V);
    uint64_t mask0 = 0, mask1 = 0;
    bool lose = false;
    sweep_small<BATCH, false, true>(P, r, col, color_of(self), prio_of(self), mask0, mask1, lose);
    if (FINAL && !lose) col[V] = pack_state(color_of(self), prio_of(self), true);
    return lose;
}

// Phase 1 work item of a larger vertex.
template <bool BATCH>
__device__ void ip_chunk_assign(const RoundParams &P, uint64_t *col, int4 it, unsigned *win, int lane) {
    const int32_t V = it.x, k = it.y, slot = it.z, nch = it.w;
    const Row r = load_row<BATCH>(P, V);
    const int64_t jb = r.b + static_cast<int64_t>(k) * P.CH;
    const int64_t je = min(r.e, jb + P.CH);
    if (lane < kAccWords) win[lane] = 0;
    __syncwarp();
    uint64_t lo = 0;
    bool unused = false;
    sweep<true, false>(P, r, col, jb, je, lane, 0, 0, lo, win, unused);
    unsigned lo0 = __reduce_or_sync(kFull, static_cast<unsigned>(lo));
    unsigned lo1 = __reduce_or_sync(kFull, static_cast<unsigned>(lo >> 32));
    __syncwarp();
    if (nch > 1 && !merge_item<true>(P.acc + static_cast<size_t>(slot) * kAccStride, nch, lane, lo0, lo1, win, unused, 0u))
        return;
    int32_t nc = first_free(lo0, lo1, win);
    if (nc < 0) nc = mex_from<BATCH>(P, col, r, win, lane, 32 * kAccWords);
    if (lane == 0) col[V] = pack_state(nc, prio_of(load_state(col + V)), false);
}

// Phase 2 work item of a larger vertex.
template <bool BATCH>
__device__ void ip_chunk_conflict(const RoundParams &P, const uint64_t *col, int4 it, unsigned *win, int4 *chunk_next,
                                  unsigned *cnt_next, int pass, int lane, unsigned &st_deg,
                                  unsigned &st_cnt) {
    const int32_t V = it.x, k = it.y, slot = it.z, nch = it.w;
    const Row r = load_row<BATCH>(P, V);
    const uint64_t self = load_state(col + V);
    const int64_t jb = r.b + static_cast<int64_t>(k) * P.CH;
    const int64_t je = min(r.e, jb + P.CH);
    if (k == 0 && lane == 0) {
        st_deg += static_cast<unsigned>(r.e - r.b);
        st_cnt += 1;
    }
    uint64_t lo = 0;
    bool lose = false;
    sweep<false, true>(P, r, col, jb, je, lane, color_of(self), prio_of(self), lo, win, lose);
    lose = __any_sync(kFull, lose);
    unsigned lo0 = 0, lo1 = 0;
    if (nch > 1 && !merge_item<false>(P.acc + static_cast<size_t>(slot) * kAccStride, nch, lane, lo0, lo1, win, lose, 0u))
        return;
    if (lose) append_large<BATCH>(P, V, r, chunk_next, cnt_next, pass + 1, lane);
}

// ------------------------------------------------------------------------------------------
// in-place mode with the compact sweep: work items are DetItem descriptors over each larger
// vertex's list of neighbours that can still change, as in deterministic mode.  A vertex that does
// not lose in phase 2 sets its FINAL bit (its color never changes again); later phase-2 sweeps drop
// it from their lists after checking it (a neighbour that won this very round can still share the
// color), and its color moves to the vertex's window of final neighbours, which phase 1 adds to
// the round window.

constexpr int kAccDone2 = 20;  // in-place compact: phase-2 work items finished

// Phase 1 work item: First Fit over the live colors of the list's neighbours and the window of
// final neighbours.
template <bool BATCH>
__device__ void ipc_item_assign(const RoundParams &P, uint64_t *col, const DetItem &d, unsigned *win, int lane,
                                unsigned &st_read) {
    const int32_t V = d.V;
    const uint32_t slot = d.slotf & kItemSlot;
    const bool multi = (d.slotf & kItemMulti) != 0;
    unsigned *a = P.acc + static_cast<size_t>(slot) * kAccStride;
    Row r;
    r.b = 0;
    r.e = 0;
    r.vbase = d.vbase;
    r.ng = d.ng;
    r.lv = V - d.vbase;
    r.g = 0;
    int32_t ul[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int64_t j = static_cast<int64_t>(d.lb) + lane + 32 * q;
        ul[q] = j < d.le ? __ldcg(d.list + j) : 0;
    }
    const unsigned fsnap = multi ? 0u : __ldcg(a + kAccFin + lane);
    if (lane < kAccWords) win[lane] = 0;
    __syncwarp();
    uint64_t lo = 0, flo = 0;
    bool lose = false;
    unsigned survivors = 0, written = 0;
    sweep_item<false, true, false>(P, r, col, d.list, d.lb, d.le, ul, nullptr, nullptr, false, lane, 0, 0, lo, win,
                                   flo, nullptr, lose, survivors, written);
    if (lane == 0) st_read += static_cast<unsigned>(d.le - d.lb);
    unsigned lo0 = __reduce_or_sync(kFull, static_cast<unsigned>(lo));
    unsigned lo1 = __reduce_or_sync(kFull, static_cast<unsigned>(lo >> 32));
    __syncwarp();
    unsigned f = fsnap;
    if (multi) {
        const unsigned w = lane == 0 ? lo0 : lane == 1 ? lo1 : (lane < kAccWords ? win[lane] : 0u);
        if (lane < kAccWords && w) atomicOr(a + lane, w);
        __syncwarp();
        unsigned done = 0;
        if (lane == 0) done = atom_add_acq_rel(a + kAccDone, 1u);
        done = __shfl_sync(kFull, done, 0);
        if (done != static_cast<unsigned>(d.nitems - 1)) return;
        // the last item: the merged round window, then the slot's round window and count cleared
        const unsigned x = __ldcg(a + lane);
        f = __ldcg(a + kAccFin + lane);
        lo0 = __shfl_sync(kFull, x, 0);
        lo1 = __shfl_sync(kFull, x, 1);
        if (lane >= 2 && lane < kAccWords) win[lane] = x;
        __syncwarp();
        if (lane < kAccWords) a[lane] = 0u;
        if (lane == 0) a[kAccDone] = 0u;
    }
    if (lane >= kAccWords) f = 0u;
    lo0 |= __shfl_sync(kFull, f, 0);
    lo1 |= __shfl_sync(kFull, f, 1);
    if (lane >= 2 && lane < kAccWords) win[lane] |= f;
    __syncwarp();
    int32_t nc = first_free(lo0, lo1, win);
    if (nc < 0) nc = mex_from<BATCH>(P, col, load_row<BATCH>(P, V), win, lane, 32 * kAccWords);
    if (lane == 0) col[V] = pack_state(nc, prio_of(load_state(col + V)), false);
}

// Phase 2 work item: conflict check over the list (a neighbour with the same color and a smaller
// key re-queues the vertex); neighbours found final are dropped into the window of final
// neighbours, and in a rewrite round the others are copied to the vertex's other list region.  The
// item that finishes the vertex sets its FINAL bit or appends its next items.
template <bool BATCH>
__device__ void ipc_item_conflict(const RoundParams &P, uint64_t *col, const DetItem &d, unsigned *wfin,
                                  unsigned *snapf, DetItem *next, unsigned *cnt_next, int pass, int lane,
                                  unsigned items_now, unsigned warps, unsigned &st_deg, unsigned &st_cnt,
                                  unsigned &st_read) {
    const int32_t V = d.V;
    const uint32_t slot = d.slotf & kItemSlot;
    const bool multi = (d.slotf & kItemMulti) != 0;
    unsigned *a = P.acc + static_cast<size_t>(slot) * kAccStride;
    Row r;
    r.b = 0;
    r.e = 0;
    r.vbase = d.vbase;
    r.ng = d.ng;
    r.lv = V - d.vbase;
    r.g = 0;
    int32_t ul[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int64_t j = static_cast<int64_t>(d.lb) + lane + 32 * q;
        ul[q] = j < d.le ? __ldcg(d.list + j) : 0;
    }
    const uint64_t self = load_state(col + V);
    const unsigned sm = __ldcg(a + 32 + lane);
    if (lane < kAccWords) {
        wfin[lane] = 0;
        snapf[lane] = sm;
    }
    const int32_t cv = color_of(self);
    const uint32_t pv = prio_of(self);
    const int64_t deg = d.deg;
    const unsigned src = __shfl_sync(kFull, sm, kAccSrc - 32);
    const unsigned len = __shfl_sync(kFull, sm, kAccLen - 32);
    const int64_t off = static_cast<int64_t>(__shfl_sync(kFull, sm, kAccOffLo - 32)) |
                        (static_cast<int64_t>(__shfl_sync(kFull, sm, kAccOffHi - 32)) << 32);
    int32_t *dst = (d.slotf & kItemRewrite) ? P.lists + off + (src == 1 ? deg : 0) : nullptr;
    __syncwarp();
    uint64_t lo = 0, flo = 0;
    bool lose = false;
    unsigned survivors = 0, written = 0;
    sweep_item<true, false, true>(P, r, col, d.list, d.lb, d.le, ul, dst, a + kAccNewLen, multi, lane, cv, pv, lo,
                                  nullptr, flo, wfin, lose, survivors, written);
    if (lane == 0) st_read += static_cast<unsigned>(d.le - d.lb);
    lose = __any_sync(kFull, lose);
    const unsigned f0 = __reduce_or_sync(kFull, static_cast<unsigned>(flo));
    const unsigned f1 = __reduce_or_sync(kFull, static_cast<unsigned>(flo >> 32));
    __syncwarp();
    const unsigned fw = lane == 0 ? f0 : lane == 1 ? f1 : (lane < kAccWords ? wfin[lane] : 0u);
    unsigned surv = 0, nlen_w = 0;
    if (multi) {
        if (lane < kAccWords && (fw & ~snapf[lane])) atomicOr(a + kAccFin + lane, fw);
        if (lane == 0 && survivors) atomicAdd(a + kAccSurv, survivors);
        if (lane == 0 && lose) atomicOr(a + kAccFlag, 1u);
        __syncwarp();
        unsigned done = 0;
        if (lane == 0) done = atom_add_acq_rel(a + kAccDone2, 1u);
        done = __shfl_sync(kFull, done, 0);
        if (done != static_cast<unsigned>(d.nitems - 1)) return;
        const uint4 st = ldcg4(a + kAccFlag);  // flag, (phase-1 count), survivors, new length
        lose = st.x != 0u;
        surv = st.z;
        nlen_w = st.w;
        __syncwarp();
        if (lane == 0) {
            a[kAccFlag] = 0u;
            a[kAccSurv] = 0u;
            a[kAccNewLen] = 0u;
            a[kAccDone2] = 0u;
        }
    } else {
        const unsigned fx = lane < kAccWords ? (snapf[lane] | fw) : 0u;
        if (lane < kAccWords && fx != snapf[lane]) a[kAccFin + lane] = fx;
        surv = __shfl_sync(kFull, survivors, 0);
        nlen_w = __shfl_sync(kFull, written, 0);
    }
    if (lane == 0) {
        st_deg += static_cast<unsigned>(deg);
        st_cnt += 1;
    }
    if (!lose) {
        if (lane == 0) col[V] = pack_state(cv, pv, true);
        return;
    }
    if constexpr (BATCH) {
        if (lane == 0) note_graph_round(P, __ldg(P.vg + V), pass + 1);
    }
    const bool rewrite = dst != nullptr;
    const unsigned nsrc = rewrite ? (src == 1 ? 2u : 1u) : src;
    const unsigned nlen = rewrite ? nlen_w : len;
    const bool nrw = 4ull * surv < 3ull * nlen;
    const int32_t items = next_items(P, nlen, deg, items_now, warps);
    if (lane == 0) {
        a[kAccSrc] = nsrc;
        a[kAccLen] = nlen;
    }
    const int32_t *list = nsrc == 0 ? d.list : P.lists + off + (nsrc == 2 ? deg : 0);
    const int64_t per = (static_cast<int64_t>(nlen) + items - 1) / items;
    append_items(next, cnt_next, lane, lane == 0 ? items : 0, list, V, slot, nrw ? kItemRewrite : 0u, nlen,
                 per > 0 ? per : 1, d.vbase, d.ng, d.deg);
}

// ------------------------------------------------------------------------------------------
// kernels


// Deterministic rounds.  Phase A: the work items of larger vertices, then one thread per vertex of
// degree <= T1.  Phase B (only in rounds where some vertex has several items, after a grid barrier):
// those vertices are finished from their merged slots, one lane each.
template <bool BATCH, bool COMPACT, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) det_round_kernel(RoundParams P) {
    __shared__ unsigned s_win[kMaxWarps][kAccWords];
    // per warp: the window of final neighbours found by the current item, then the item's snapshots
    // of its slot's round window and final window
    __shared__ unsigned s_aux[kMaxWarps][3 * kAccWords];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    unsigned *win = s_win[wib];
    unsigned *wfin = s_aux[wib];
    unsigned *snap = s_aux[wib] + kAccWords;
    if (P.stats && blockIdx.x == 0 && threadIdx.x == 0) P.stats[4 * P.stats_cap] = global_ns();
    unsigned bar_target = 0;
    int pass = P.pass_begin;
    for (;; ++pass) {
        unsigned *cc = P.cnt + kCnt * (pass % 3);
        unsigned *cn = P.cnt + kCnt * ((pass + 1) % 3);
        const unsigned nsmall = __ldcg(cc + kCntSmall), nitems = __ldcg(cc + kCntItems);
        const unsigned nchunks = __ldcg(cc + kCntChunks), nmulti = __ldcg(cc + kCntMulti);
        if (nsmall + nitems == 0u) break;
        if constexpr (COMPACT) {
            // small enough for the core phase: every block reads the same counters, so all leave here
            if (P.core_max > 0 && nsmall + nitems <= static_cast<unsigned>(P.core_max) &&
                (!P.ecnt || __ldcg(P.ecnt + pass % 3) <= static_cast<unsigned long long>(P.core_emax))) {
                if (blockIdx.x == 0 && threadIdx.x == 0) *P.core_go = 1;
                break;
            }
        }
        if (pass >= P.pass_end) {
            if (P.cap_is_error && blockIdx.x == 0 && threadIdx.x == 0)
                set_error(P.err, GC_ERR_NO_CONVERGENCE, pass, 0);
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x < kCnt) P.cnt[kCnt * ((pass + 2) % 3) + threadIdx.x] = 0u;
        if (P.ecnt && blockIdx.x == 0 && threadIdx.x == 0) P.ecnt[(pass + 2) % 3] = 0ull;
        const bool odd = (pass & 1) != 0;
        const uint64_t *colc = odd ? P.col0 : P.col1;
        uint64_t *coln = odd ? P.col1 : P.col0;
        const int32_t *smallc = odd ? P.small0 : P.small1;
        int32_t *smalln = odd ? P.small1 : P.small0;
        const DetItem *itc = reinterpret_cast<const DetItem *>(odd ? P.chunk0 : P.chunk1);
        // round 1 with the hash key: every neighbour's state is known without reading it
        const bool r1 = pass == 1 && P.priority == GC_PRIORITY_HASH;
        // the colors a neighbour can have in this round (0..pass-1), for the early stop of a sweep
        const uint64_t need = P.early_exit && pass <= 64 ? (~0ull >> (64 - pass)) : 0ull;
        DetItem *itn = reinterpret_cast<DetItem *>(odd ? P.chunk1 : P.chunk0);
        unsigned st_deg = 0, st_cnt = 0, st_read = 0;  // this warp's share of the round (< 2^31 each)
        unsigned long long st_ent = 0;  // list entries this thread appended to the next worklist
        // phase A: work items of larger vertices first (they dominate; the next item is read while
        // the current one runs), then one thread per small vertex
        // sparse rounds (at most kMergeNowItems items per warp) finish several-item vertices in phase A
        const bool merge_now = nchunks <= kMergeNowItems * static_cast<unsigned>(nw);
        if (static_cast<unsigned>(gw) < nchunks) {
            uint32_t w = item_word(itc, gw, lane);
            for (unsigned i = gw; i < nchunks; i += nw) {
                const DetItem d = item_of(w);
                if (i + nw < nchunks) w = item_word(itc, i + nw, lane);
                det_item<BATCH, COMPACT>(P, colc, coln, d, win, wfin, snap, itn, cn, pass, lane, nchunks,
                                         static_cast<unsigned>(nw), merge_now, st_deg, st_cnt, st_read, r1, st_ent,
                                         need);
            }
        }
        for (unsigned base = static_cast<unsigned>(gw) * 32u; base < nsmall; base += static_cast<unsigned>(nw) * 32u) {
            const unsigned i = base + lane;
            bool lose = false;
            int32_t V = 0, deg = 0, nread = 0;
            if (i < nsmall) {
                V = __ldcg(smallc + i);
                lose = det_small<BATCH>(P, colc, coln, V, deg, nread, r1, need);
                st_deg += static_cast<unsigned>(deg);
                st_read += static_cast<unsigned>(nread);
                st_cnt += 1;
                if constexpr (BATCH) {
                    if (lose) note_graph_round(P, __ldg(P.vg + V), pass + 1);
                }
            }
            warp_append(lose, V, smalln, cn + kCntSmall, lane);
            if (lose) st_ent += static_cast<unsigned long long>(deg);
        }
        // phase B
        if (nmulti != 0u && !merge_now) {
            if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) break;
            for (unsigned base = static_cast<unsigned>(gw) * 32u; base < nchunks;
                 base += static_cast<unsigned>(nw) * 32u) {
                const unsigned i = base + lane;
                DetItem d{};
                bool fin = false;
                if (i < nchunks) {
                    d = item_lane(itc + i);
                    fin = (d.slotf & kItemMulti) != 0u && d.lb == 0;
                }
                det_finish<BATCH, COMPACT>(P, colc, coln, fin, d, win, itn, cn, pass, lane, nchunks,
                                           static_cast<unsigned>(nw), st_deg, st_cnt, st_ent);
            }
        }
        if (P.stats) flush_stats(P, pass, st_deg, st_cnt, st_read);
        if (P.ecnt) flush_sum(P.ecnt + (pass + 1) % 3, st_ent);
        if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.passes[0] = pass;
        P.passes[1] = pass - 1;
    }
}

template <bool BATCH, bool COMPACT, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) ip_round_kernel(RoundParams P) {
    __shared__ unsigned s_win[kMaxWarps][kAccWords];
    __shared__ unsigned s_aux[kMaxWarps][COMPACT ? 2 * kAccWords : 1];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    unsigned *win = s_win[wib];
    uint64_t *col = P.col0;
    if (P.stats && blockIdx.x == 0 && threadIdx.x == 0) P.stats[4 * P.stats_cap] = global_ns();
    unsigned bar_target = 0;
    int pass = P.pass_begin;
    for (;; ++pass) {
        unsigned *cc = P.cnt + kCnt * (pass % 3);
        unsigned *cn = P.cnt + kCnt * ((pass + 1) % 3);
        const unsigned nsmall = __ldcg(cc + kCntSmall), nitems = __ldcg(cc + kCntItems);
        const unsigned nchunks = __ldcg(cc + kCntChunks);
        if (nsmall + nitems == 0u) break;
        if (pass >= P.pass_end) {
            if (P.cap_is_error && blockIdx.x == 0 && threadIdx.x == 0)
                set_error(P.err, GC_ERR_NO_CONVERGENCE, pass, 0);
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x < kCnt) P.cnt[kCnt * ((pass + 2) % 3) + threadIdx.x] = 0u;
        const bool odd = (pass & 1) != 0;
        const int32_t *smallc = odd ? P.small0 : P.small1;
        int32_t *smalln = odd ? P.small1 : P.small0;
        const int4 *chunkc = odd ? P.chunk0 : P.chunk1;
        int4 *chunkn = odd ? P.chunk1 : P.chunk0;
        unsigned st_deg = 0, st_cnt = 0, st_read = 0;  // this warp's share of the round (< 2^31 each)
        // phase 1: tentative First Fit on live colors
        if constexpr (COMPACT) {
            const DetItem *itc = reinterpret_cast<const DetItem *>(chunkc);
            if (static_cast<unsigned>(gw) < nchunks) {
                uint32_t w = item_word(itc, gw, lane);
                for (unsigned i = gw; i < nchunks; i += nw) {
                    const DetItem d = item_of(w);
                    if (i + nw < nchunks) w = item_word(itc, i + nw, lane);
                    ipc_item_assign<BATCH>(P, col, d, win, lane, st_read);
                }
            }
        } else {
            for (unsigned i = gw; i < nchunks; i += nw) ip_chunk_assign<BATCH>(P, col, __ldcg(chunkc + i), win, lane);
        }
        if (P.spread && nsmall > 0u) {
            // entry (t K) mod N for thread step t, K coprime with N near N / golden ratio: the
            // vertices in flight at one time are spread over the whole list instead of a run of
            // consecutive (on meshes: adjacent) ids, so far fewer of them read each other uncolored
            unsigned Kp = static_cast<unsigned>(static_cast<uint64_t>(nsmall) * 2654435769ull >> 32) | 1u;
            for (;;) {
                unsigned a = Kp, b = nsmall;
                while (b) {
                    const unsigned t = a % b;
                    a = b;
                    b = t;
                }
                if (a == 1u) break;
                Kp += 2u;
            }
            const unsigned t0 = gw * 32u + lane, dt = nw * 32u;
            unsigned pos = static_cast<unsigned>(static_cast<uint64_t>(t0 % nsmall) * Kp % nsmall);
            const unsigned dpos = static_cast<unsigned>(static_cast<uint64_t>(dt % nsmall) * Kp % nsmall);
            for (unsigned i = t0; i < nsmall; i += dt) {
                ip_small_assign<BATCH>(P, col, __ldcg(smallc + pos));
                pos += dpos;
                if (pos >= nsmall) pos -= nsmall;
            }
        } else {
            for (unsigned i = gw * 32u + lane; i < nsmall; i += nw * 32u)
                ip_small_assign<BATCH>(P, col, __ldcg(smallc + i));
        }
        if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) break;
        // phase 2: conflict detection
        if constexpr (COMPACT) {
            const DetItem *itc = reinterpret_cast<const DetItem *>(chunkc);
            DetItem *itn = reinterpret_cast<DetItem *>(chunkn);
            if (static_cast<unsigned>(gw) < nchunks) {
                uint32_t w = item_word(itc, gw, lane);
                for (unsigned i = gw; i < nchunks; i += nw) {
                    const DetItem d = item_of(w);
                    if (i + nw < nchunks) w = item_word(itc, i + nw, lane);
                    ipc_item_conflict<BATCH>(P, col, d, s_aux[wib], s_aux[wib] + kAccWords, itn, cn, pass, lane,
                                             nchunks, static_cast<unsigned>(nw), st_deg, st_cnt, st_read);
                }
            }
        } else {
            for (unsigned i = gw; i < nchunks; i += nw)
                ip_chunk_conflict<BATCH>(P, col, __ldcg(chunkc + i), win, chunkn, cn, pass, lane, st_deg, st_cnt);
        }
        // small vertices from a warp rotated by the number of larger vertices, so that the warps
        // with the first phase-2 items seldom get a group of small vertices as well
        for (unsigned base = ((gw + nw - nitems % nw) % nw) * 32u; base < nsmall; base += nw * 32u) {
            const unsigned i = base + lane;
            bool lose = false;
            int32_t V = 0, deg = 0;
            if (i < nsmall) {
                V = __ldcg(smallc + i);
                lose = ip_small_conflict<BATCH, COMPACT>(P, col, V, deg);
                st_deg += static_cast<unsigned>(deg);
                st_read += 2u * static_cast<unsigned>(deg);
                st_cnt += 1;
                if constexpr (BATCH) {
                    if (lose) note_graph_round(P, __ldg(P.vg + V), pass + 1);
                }
            }
            warp_append(lose, V, smalln, cn + kCntSmall, lane);
        }
        if (P.stats) flush_stats(P, pass, st_deg, st_cnt, COMPACT ? st_read : 2ull * st_deg);
        if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.passes[0] = pass;
        P.passes[1] = pass - 1;
    }
}

// gc_color_batch: graph table, graph id of every vertex and graph_last, from the offset tables;
// also checks the tables.  One block per graph.
__global__ void batch_tables_kernel(RoundParams P, const int64_t *vtx_off, const int64_t *edge_off, int64_t *g_vbase,
                                    int32_t *g_n, int64_t *g_ebase, int64_t *g_rbase, int64_t *g_m) {
    for (int32_t g = blockIdx.x; g < P.G; g += gridDim.x) {
        const int64_t v0 = vtx_off[g], v1 = vtx_off[g + 1];
        const int64_t e0 = edge_off[g], e1 = edge_off[g + 1];
        const bool ok = v1 >= v0 && e1 >= e0 && v1 <= P.n && (g != 0 || (v0 == 0 && e0 == 0));
        if (threadIdx.x == 0) {
            if (!ok) set_error(P.err, GC_ERR_INVALID_GRAPH, -1 - g, 0);
            g_vbase[g] = ok ? v0 : 0;
            g_n[g] = ok ? static_cast<int32_t>(v1 - v0) : 0;
            g_ebase[g] = e0;
            g_rbase[g] = v0 + g;
            g_m[g] = e1 - e0;
            P.graph_last[g] = (ok && v1 > v0) ? 1 : 0;
        }
        if (!ok) continue;
        for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) P.vg[v] = g;
    }
}

// Binning and initialisation of vertices [v_begin, v_end) for round P.pass_begin: priority cache,
// initial colors, and the round's worklist split into thread-per-vertex entries (appended to the
// current small list) and larger vertices (collected in P.items, counted in P.tmp, expanded into
// work items by expand_kernel).  Checks each row: 0 <= rowptr[v] <= rowptr[v+1] <= entries of its
// graph, rowptr of a graph's first vertex = 0, of its last vertex's end = its entries.
// Sort bins of the initial thread worklist: (vertex block of 2^P.sort_shift ids, degree).
__device__ __forceinline__ int32_t sort_bin(const RoundParams &P, int32_t V, int64_t d) {
    return (V >> P.sort_shift) * 128 + static_cast<int32_t>(d);
}

// Row of vertex V for set-up: its entry range, checked (0 <= rowptr[v] <= rowptr[v+1] <= entries of
// its graph, 0 at a graph's first vertex, the graph's entry count at its end).  g: V's graph (batch).
// Returns the degree, or -1 for a malformed row.
template <bool BATCH>
__device__ __forceinline__ int64_t checked_degree(const RoundParams &P, int32_t V, int32_t g, int64_t &b, int32_t &lv) {
    int64_t e, lim;
    int32_t ng;
    if constexpr (!BATCH) {
        b = P.rowptr[V];
        e = P.rowptr[V + 1];
        lim = P.nnz;
        lv = V;
        ng = P.n;
    } else {
        lv = V - static_cast<int32_t>(P.g_vbase[g]);
        ng = P.g_n[g];
        const int32_t *rp = P.rowptr + P.g_rbase[g];
        b = rp[lv];
        e = rp[lv + 1];
        lim = P.g_m[g];
    }
    const bool ok = b >= 0 && b <= e && e <= lim && (lv != 0 || b == 0) && (lv != ng - 1 || e == lim);
    return ok ? e - b : -1;
}

// Binning and initialisation of vertices [v_begin, v_end) for round P.pass_begin: priority cache,
// initial colors, and the round's worklist split into thread-per-vertex entries and larger vertices
// (collected in P.items, counted in P.tmp, expanded into work items by expand_kernel).  Checks each
// row.  Thread-per-vertex entries are appended to the current small list, or, when P.deg_hist is
// set, only counted per (vertex block, degree) for sort_small_kernel and scatter_small_kernel,
// which write the list block by block (2^P.sort_shift consecutive ids each) and by increasing
// degree inside a block: the 32 rows a warp sweeps side by side have similar lengths, and when the
// state words do not fit in L2 (large graphs, batches) the vertices in flight at any moment (and,
// in a batch, their graphs' neighbours) stay within a few blocks whose state words L2 holds.
template <bool BATCH, int MODE>
__global__ void __launch_bounds__(256) setup_kernel(RoundParams P, int32_t v_begin, int32_t v_end, int32_t g_fixed) {
    __shared__ unsigned s_hist[128];
    // block-wide reservations, one atomic per 256 vertices: larger vertices into P.items, vertices of
    // degree <= T1 into the thread worklist when it is not degree-sorted
    __shared__ unsigned s_w[8][2];
    __shared__ unsigned s_base[2];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int pass = P.pass_begin;
    unsigned *cc = P.cnt + kCnt * (pass % 3);
    int32_t *small_cur = (pass & 1) ? P.small0 : P.small1;
    const bool sort = P.deg_hist != nullptr;
    // one vertex block: a per-block histogram in shared memory, added to the global one at the end
    const bool one_block = sort && (v_end - 1) >> P.sort_shift == 0;
    if (one_block) {
        for (int t = threadIdx.x; t < 128; t += blockDim.x) s_hist[t] = 0;
        __syncthreads();
    }
    const int64_t count = static_cast<int64_t>(v_end) - v_begin;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    unsigned long long st_ent = 0;  // list entries of the round's worklist (rows of its vertices)
    unsigned long long st_list = 0;  // compact mode: list-pool entries of the larger vertices
    unsigned st_chunks = 0;          // work items of the larger vertices
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < count; base += stride) {
        const int64_t i = base + threadIdx.x;
        const int32_t V = static_cast<int32_t>(v_begin + i);
        const bool in = i < count;
        int kind = 0;  // 1 = one thread, 2 = work items
        int32_t nch = 0;
        int64_t d = 0;
        if (in) {
            int32_t g = 0;
            if constexpr (BATCH) {
                g = g_fixed;
                if (g >= 0)
                    P.vg[V] = g;
                else
                    g = P.vg[V];
            }
            int64_t b;
            int32_t lv;
            d = checked_degree<BATCH>(P, V, g, b, lv);
            if (d < 0) {
                set_error(P.err, GC_ERR_INVALID_GRAPH, V, b);
                d = 0;
            }
            const uint32_t pv = priority_bits(P, static_cast<uint32_t>(lv), d, V);
            // an isolated vertex takes color 0 in round 1 and never changes: it is final from the start
            if (MODE == GC_MODE_DETERMINISTIC) {
                // C_1 = 0 everywhere: round 1's First Fit sees no colored neighbour
                P.col0[V] = pack_state(0, pv, d == 0);
                P.col1[V] = pack_state(0, pv, d == 0);
            } else {
                P.col0[V] = pack_state(d == 0 ? 0 : -1, pv, d == 0);
            }
            if (d > 0) {
                kind = d <= P.T1 ? 1 : 2;
                nch = static_cast<int32_t>((d + P.CH - 1) / P.CH);
            }
        }
        if constexpr (BATCH) {
            if (g_fixed >= 0 && kind != 0) note_graph_round(P, g_fixed, pass);
        }
        if (kind != 0) st_ent += static_cast<unsigned long long>(d);
        if (kind == 2) {
            st_chunks += static_cast<unsigned>(nch);
            if (P.list_total) st_list += 2ull * static_cast<unsigned long long>(d);  // two list regions
        }
        if (one_block) {
            if (kind == 1) atomicAdd(&s_hist[d], 1u);
        } else if (sort) {
            // lanes with the same bin add once
            const int32_t bin = kind == 1 ? sort_bin(P, V, d) : -1;
            const unsigned same = __match_any_sync(kFull, bin);
            if (kind == 1 && lane == __ffs(same) - 1) atomicAdd(P.deg_hist + bin, static_cast<unsigned>(__popc(same)));
        }
        const unsigned m2 = __ballot_sync(kFull, kind == 2);
        const unsigned m1 = sort ? 0u : __ballot_sync(kFull, kind == 1);
        if (lane == 0) {
            s_w[wib][0] = __popc(m2);
            s_w[wib][1] = __popc(m1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned t0 = 0, t1 = 0;
            for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
                const unsigned a0 = s_w[w][0], a1 = s_w[w][1];
                s_w[w][0] = t0;
                s_w[w][1] = t1;
                t0 += a0;
                t1 += a1;
            }
            s_base[0] = t0 ? atomicAdd(P.tmp + 0, t0) : 0u;
            s_base[1] = t1 ? atomicAdd(cc + kCntSmall, t1) : 0u;
        }
        __syncthreads();
        if (kind == 2) P.items[s_base[0] + s_w[wib][0] + __popc(m2 & lanemask_lt())] = V;
        if (!sort && kind == 1) small_cur[s_base[1] + s_w[wib][1] + __popc(m1 & lanemask_lt())] = V;
        __syncthreads();  // s_w / s_base are rewritten by the next iteration
    }
    if (one_block) {
        __syncthreads();
        for (int t = threadIdx.x; t < 128; t += blockDim.x)
            if (s_hist[t]) atomicAdd(P.deg_hist + t, s_hist[t]);
    }
    flush_sum_u32(P.tmp + 1, st_chunks);
    if (P.list_total) flush_sum(P.list_total, st_list);
    if (P.ecnt) flush_sum(P.ecnt + pass % 3, st_ent);
}

// One block of kSortThreads threads: turns the (vertex block, degree) counts P.deg_hist[0, nbins)
// into list positions P.deg_hist[nbins + bin] (after the entries already on the current small
// list, bins in increasing order) and adds them to the list's count.
constexpr int kSortThreads = 1024;
__global__ void __launch_bounds__(kSortThreads) sort_small_kernel(RoundParams P, int32_t nbins) {
    __shared__ unsigned s[kSortThreads];
    const int t = threadIdx.x;
    unsigned *cc = P.cnt + kCnt * (P.pass_begin % 3);
    const int32_t per = (nbins + kSortThreads - 1) / kSortThreads;
    const int32_t b0 = t * per, b1 = min(nbins, b0 + per);
    unsigned sum = 0;
    for (int32_t i = b0; i < b1; ++i) sum += P.deg_hist[i];
    s[t] = sum;
    __syncthreads();
    for (int o = 1; o < kSortThreads; o <<= 1) {
        const unsigned x = t >= o ? s[t - o] : 0u;
        __syncthreads();
        s[t] += x;
        __syncthreads();
    }
    const unsigned base = cc[kCntSmall];
    unsigned run = base + s[t] - sum;  // exclusive prefix of this thread's first bin
    for (int32_t i = b0; i < b1; ++i) {
        const unsigned h = P.deg_hist[i];
        P.deg_hist[nbins + i] = run;
        run += h;
    }
    __syncthreads();
    if (t == kSortThreads - 1) cc[kCntSmall] = base + s[t];
}

// Writes the thread-per-vertex entries of [v_begin, v_end) (v_begin a multiple of the block size)
// at the positions sort_small_kernel assigned, with the same classification as setup_kernel; the
// order within one (vertex block, degree) bin is arbitrary.  Each iteration covers 256 consecutive
// ids, all inside one vertex block.
template <bool BATCH>
__global__ void scatter_small_kernel(RoundParams P, int32_t v_begin, int32_t v_end, int32_t nbins) {
    __shared__ unsigned s_cnt[128], s_base[128];
    int32_t *small_cur = (P.pass_begin & 1) ? P.small0 : P.small1;
    const unsigned *cursor = P.deg_hist + nbins;
    const int64_t count = static_cast<int64_t>(v_end) - v_begin;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < count;
         base += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        for (int t = threadIdx.x; t < 128; t += blockDim.x) s_cnt[t] = 0;
        __syncthreads();
        const int32_t V = static_cast<int32_t>(v_begin + base + threadIdx.x);
        int64_t d = 0;
        if (base + threadIdx.x < count) {
            const int32_t g = BATCH ? P.vg[V] : 0;
            int64_t b;
            int32_t lv;
            d = checked_degree<BATCH>(P, V, g, b, lv);
        }
        const bool small = d > 0 && d <= P.T1;
        unsigned rank = 0;
        if (small) rank = atomicAdd(&s_cnt[d], 1u);
        __syncthreads();
        const int32_t bin0 = sort_bin(P, static_cast<int32_t>(v_begin + base), 0);
        for (int t = threadIdx.x; t < 128; t += blockDim.x)
            if (s_cnt[t]) s_base[t] = atomicAdd(const_cast<unsigned *>(cursor) + bin0 + t, s_cnt[t]);
        __syncthreads();
        if (small) small_cur[s_base[d] + rank] = V;
        __syncthreads();
    }
}

// Expands the larger vertices collected by setup into work items of round P.pass_begin, with
// accumulator slots after those already taken in that round.  One warp per vertex.  COMPACT: the
// vertex keeps its slot for the whole run (slot V with P.slot_per_vertex); the slot records where
// its list is, the list's length, the vertex's space in the list pool and its degree.  Deterministic items are DetItem (a vertex's
// items split its row evenly with COMPACT, else into CH-entry pieces); in-place items are int4
// {vertex, item index, slot, items}.
template <bool BATCH, bool COMPACT, int MODE>
__global__ void __launch_bounds__(256) expand_kernel(RoundParams P, int32_t n_items) {
    // block-wide reservations: per 256 vertices one atomic per counter (the counters are shared by
    // the whole grid; one atomic per vertex would serialise on them)
    __shared__ unsigned s_w[8][4];
    __shared__ unsigned long long s_wl[8];
    __shared__ unsigned s_base[4];
    __shared__ unsigned long long s_lbase;
    if (n_items < 0) n_items = static_cast<int32_t>(__ldcg(P.tmp));  // count left on the device by setup
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int pass = P.pass_begin;
    unsigned *cc = P.cnt + kCnt * (pass % 3);
    const bool lists = COMPACT && !P.slot_per_vertex;
    for (int32_t s0 = blockIdx.x * blockDim.x; s0 < n_items; s0 += gridDim.x * blockDim.x) {
        const int32_t s = s0 + static_cast<int32_t>(threadIdx.x);
        const bool in = s < n_items;
        int32_t V = 0, deg = 0, nch = 0;
        Row r{};
        if (in) {
            V = P.items[s];
            r = load_row<BATCH>(P, V);
            deg = static_cast<int32_t>(r.e - r.b);
            nch = (deg + P.CH - 1) / P.CH;
        }
        // warp-inclusive scans of the vertex's chunks and list space
        unsigned ich = static_cast<unsigned>(nch);
        unsigned long long il = lists && in ? 2ull * static_cast<unsigned long long>(deg) : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, ich, o);
            const unsigned long long z = __shfl_up_sync(kFull, il, o);
            if (lane >= o) {
                ich += y;
                il += z;
            }
        }
        const unsigned mi = __ballot_sync(kFull, in), mm = __ballot_sync(kFull, in && nch > 1);
        if (lane == 31) {
            s_w[wib][0] = __popc(mi);
            s_w[wib][1] = ich;
            s_w[wib][2] = __popc(mm);
            s_wl[wib] = il;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned t[3] = {0, 0, 0};
            unsigned long long tl = 0;
            for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
                const unsigned a0 = s_w[w][0], a1 = s_w[w][1], a2 = s_w[w][2];
                const unsigned long long al = s_wl[w];
                s_w[w][0] = t[0];
                s_w[w][1] = t[1];
                s_w[w][2] = t[2];
                s_wl[w] = tl;
                t[0] += a0;
                t[1] += a1;
                t[2] += a2;
                tl += al;
            }
            s_base[0] = t[0] ? atomicAdd(cc + kCntItems, t[0]) : 0u;
            s_base[1] = t[1] ? atomicAdd(cc + kCntChunks, t[1]) : 0u;
            if ((MODE == GC_MODE_DETERMINISTIC || COMPACT) && t[2]) atomicAdd(cc + kCntMulti, t[2]);
            s_lbase = lists && tl ? atomicAdd(P.list_alloc, tl) : 0ull;
        }
        __syncthreads();
        // this lane's slot, first chunk and list offset
        unsigned slot = s_base[0] + s_w[wib][0] + __popc(mi & lanemask_lt());
        const unsigned cb = s_base[1] + s_w[wib][1] + ich - static_cast<unsigned>(nch);
        const unsigned long long loff =
            s_lbase + s_wl[wib] + il - (lists && in ? 2ull * static_cast<unsigned long long>(deg) : 0ull);
        if (COMPACT && P.slot_per_vertex) slot = static_cast<unsigned>(V);
        __syncthreads();  // s_w / s_base are rewritten by the next iteration
        // the warp writes each of its vertices' slot and work items together
        for (unsigned pm = mi; pm; pm &= pm - 1u) {
            const int l = __ffs(pm) - 1;
            const int32_t Vl = __shfl_sync(kFull, V, l);
            const int32_t degl = __shfl_sync(kFull, deg, l);
            const int32_t nchl = __shfl_sync(kFull, nch, l);
            const unsigned slotl = __shfl_sync(kFull, slot, l), cbl = __shfl_sync(kFull, cb, l);
            const int64_t rb = static_cast<int64_t>(__shfl_sync(kFull, static_cast<unsigned long long>(r.b), l));
            const int32_t vb = __shfl_sync(kFull, r.vbase, l), ngl = __shfl_sync(kFull, r.ng, l);
            unsigned *acc = P.acc + static_cast<size_t>(slotl) * kAccStride;
            acc[lane] = 0u;
            unsigned hi = 0u;
            if (COMPACT) {
                // the list starts as the CSR row; the two list regions in the pool
                const unsigned long long off = P.slot_per_vertex ? 2ull * static_cast<unsigned long long>(rb)
                                                                 : __shfl_sync(kFull, loff, l);
                if (lane == kAccLen - 32) hi = static_cast<unsigned>(degl);
                if (lane == kAccOffLo - 32) hi = static_cast<unsigned>(off);
                if (lane == kAccOffHi - 32) hi = static_cast<unsigned>(off >> 32);
                if (lane == kAccDeg - 32) hi = static_cast<unsigned>(degl);
            }
            acc[32 + lane] = hi;
            if constexpr (MODE == GC_MODE_DETERMINISTIC || COMPACT) {
                DetItem *cur = reinterpret_cast<DetItem *>((pass & 1) ? P.chunk0 : P.chunk1);
                const int32_t per = COMPACT ? (degl + nchl - 1) / nchl : P.CH;
                const uint32_t slotf = slotl | (nchl > 1 ? kItemMulti : 0u);
                for (int32_t q = lane; q < nchl; q += 32) {
                    const int32_t lb = q * per;
                    store_item(cur + cbl + q, P.colidx + rb, Vl, slotf, lb, min(degl, lb + per), vb, ngl, nchl, degl);
                }
            } else {
                int4 *cur = (pass & 1) ? P.chunk0 : P.chunk1;
                for (int32_t q = lane; q < nchl; q += 32)
                    cur[cbl + q] = make_int4(Vl, q, static_cast<int32_t>(slotl), nchl);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// partition mode: Algorithm 1 with p blocks of consecutive ids

// Block i (0-based) of p over n vertices holds ids [floor(i n / p), floor((i + 1) n / p)).
__device__ __forceinline__ int32_t part_lo(int64_t i, int64_t n, int64_t p) { return static_cast<int32_t>(i * n / p); }

// Set-up of partition mode: rows checked, every color -1 in both buffers, every vertex on W_1.
__global__ void part_init_kernel(RoundParams P) {
    unsigned *cc = P.cnt + kCnt * (1 % 3);
    if (blockIdx.x == 0 && threadIdx.x == 0) cc[kCntSmall] = static_cast<unsigned>(P.n);
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < P.n; v += gridDim.x * blockDim.x) {
        int64_t b;
        int32_t lv;
        if (checked_degree<false>(P, v, 0, b, lv) < 0) set_error(P.err, GC_ERR_INVALID_GRAPH, v, b);
        P.col0[v] = pack_state(-1, 0, false);
        P.col1[v] = pack_state(-1, 0, false);
        P.small0[v] = 1;
    }
}

// First Fit of vertex V in phase 1 (one warp): a neighbour in V's own block [lo, hi) counts with its
// live color (this warp colored the block's earlier vertices a moment ago), any other with the
// color it had when the round began (S).  Window of 512 colors at a time in shared memory.
__device__ __forceinline__ int32_t part_first_fit(const RoundParams &P, const uint64_t *C, const uint64_t *S, int32_t V,
                                                  int32_t lo, int32_t hi, unsigned *win, int lane) {
    const int64_t b = P.rowptr[V], e = P.rowptr[V + 1];
    for (int32_t base = 0;; base += 32 * kAccWords) {
        if (lane < kAccWords) win[lane] = 0;
        __syncwarp();
        for (int64_t j = b + lane; j < e; j += 32) {
            const int32_t u = __ldg(P.colidx + j);
            if (static_cast<uint32_t>(u) >= static_cast<uint32_t>(P.n) || u == V) {
                set_error(P.err, GC_ERR_INVALID_GRAPH, V, j);
                continue;
            }
            const int32_t c = color_of(u >= lo && u < hi ? __ldcg(reinterpret_cast<const unsigned long long *>(C) + u)
                                                         : __ldcg(reinterpret_cast<const unsigned long long *>(S) + u)) -
                              base;
            if (static_cast<unsigned>(c) < 32u * kAccWords) atomicOr(&win[c >> 5], 1u << (c & 31));
        }
        __syncwarp();
        int32_t res = -1;
        const unsigned x = lane < kAccWords ? win[lane] : 0xffffffffu;
        const unsigned m = __ballot_sync(kFull, x != 0xffffffffu);
        if (m) {
            const int l = __ffs(m) - 1;
            res = base + 32 * l + __ffs(~__shfl_sync(kFull, x, l)) - 1;
        }
        __syncwarp();
        if (res >= 0) return res;
    }
}

// Partition mode (Algorithm 1 of Section 3.1 taken literally: partition priority instead of a hash):
// p blocks of consecutive ids, one warp per block at a time.  Phase 1: a block's worklist vertices
// take First Fit one after another in id order.  Grid barrier.  Phase 2: a worklist vertex is
// re-queued when a neighbour in a higher block has its color (the lower block recolors).  Grid
// barrier.  Colors live in col0 (current) and col1 (as the round began); small0[v] = r puts v on W_r.
__global__ void __launch_bounds__(kBlock, kNarrowBlocks) part_round_kernel(RoundParams P, int32_t p) {
    __shared__ unsigned s_win[kMaxWarps][kAccWords];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    unsigned *win = s_win[wib];
    uint64_t *C = P.col0, *S = P.col1;
    int32_t *onw = P.small0;
    const int64_t n = P.n;
    if (P.stats && blockIdx.x == 0 && threadIdx.x == 0) P.stats[4 * P.stats_cap] = global_ns();
    unsigned bar_target = 0;
    int pass = P.pass_begin;
    for (;; ++pass) {
        unsigned *cc = P.cnt + kCnt * (pass % 3);
        unsigned *cn = P.cnt + kCnt * ((pass + 1) % 3);
        const unsigned nwl = __ldcg(cc + kCntSmall);
        if (nwl == 0u) break;
        if (pass >= P.pass_end) {
            if (P.cap_is_error && blockIdx.x == 0 && threadIdx.x == 0)
                set_error(P.err, GC_ERR_NO_CONVERGENCE, pass, 0);
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x < kCnt) P.cnt[kCnt * ((pass + 2) % 3) + threadIdx.x] = 0u;
        unsigned st_deg = 0;
        // phase 1
        for (int32_t i = gw; i < p; i += nw) {
            const int32_t lo = part_lo(i, n, p), hi = part_lo(i + 1, n, p);
            for (int32_t base = lo; base < hi; base += 32) {
                const int32_t v = base + lane;
                unsigned m = __ballot_sync(kFull, v < hi && __ldcg(onw + v) == pass);
                while (m) {
                    const int32_t V = base + __ffs(m) - 1;
                    m &= m - 1;
                    const int32_t c = part_first_fit(P, C, S, V, lo, hi, win, lane);
                    if (lane == 0) {
                        C[V] = pack_state(c, 0, false);
                        st_deg += static_cast<unsigned>(P.rowptr[V + 1] - P.rowptr[V]);
                    }
                    __syncwarp();
                }
            }
        }
        if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) break;
        // phase 2
        unsigned lost = 0;
        for (int32_t i = gw; i < p; i += nw) {
            const int32_t lo = part_lo(i, n, p), hi = part_lo(i + 1, n, p);
            for (int32_t base = lo; base < hi; base += 32) {
                const int32_t v = base + lane;
                unsigned m = __ballot_sync(kFull, v < hi && __ldcg(onw + v) == pass);
                while (m) {
                    const int32_t V = base + __ffs(m) - 1;
                    m &= m - 1;
                    const uint64_t cvw = __ldcg(reinterpret_cast<const unsigned long long *>(C) + V);
                    const int32_t cv = color_of(cvw);
                    bool hit = false;
                    for (int64_t j = P.rowptr[V] + lane; j < P.rowptr[V + 1] && !hit; j += 32) {
                        const int32_t u = __ldg(P.colidx + j);
                        if (u >= hi && u < P.n &&
                            color_of(__ldcg(reinterpret_cast<const unsigned long long *>(C) + u)) == cv)
                            hit = true;
                    }
                    const bool lose = __any_sync(kFull, hit);
                    if (lane == 0) {
                        S[V] = cvw;  // the color phase 1 of the next round sees from other blocks
                        if (lose) {
                            onw[V] = pass + 1;
                            ++lost;
                        }
                    }
                }
            }
        }
        if (lane == 0 && lost) atomicAdd(cn + kCntSmall, lost);
        if (P.stats) flush_stats(P, pass, st_deg, (blockIdx.x == 0 && threadIdx.x == 0) ? nwl : 0u, 2ull * st_deg);
        if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.passes[0] = pass;
        P.passes[1] = pass - 1;
    }
}

// ------------------------------------------------------------------------------------------
// ordered mode: First Fit in key order without speculation.  pend[v] counts v's neighbours with a
// smaller key that are still uncolored; a vertex whose count is 0 is ready: it takes First Fit over
// its colored neighbours (exactly those with a smaller key) and, in the same sweep, counts itself
// down at each uncolored neighbour (each has a larger key and waits for it).  A neighbour whose count
// reaches 0 is ready in the next round.  Two adjacent vertices are never ready in the same round,
// so every state a ready vertex reads was written before the round began or stays uncolored in it.
//
// A ready vertex of degree <= P.T1 (at most kOrdSmall) is one thread's work, one of degree <=
// kOrdMid an 8-lane group's (four per warp); a larger one is split into work items of P.CH (at most
// kOrdChunk) entries, one warp each, so that a round lasts about as long as one item however large
// its hubs are.  The items of one vertex merge their windows in an accumulator slot (kOrdSlotWords
// words) and the warp that finishes last picks the color.  Every vertex is listed at most once in
// the whole run (its count reaches 0 once), so the small and medium lists never hold more than n
// vertices and the item lists no more than the sum over larger v of ceil(deg(v) / P.CH) items.

constexpr int kOrdPer = kOrdChunk / 32;  // entries per lane per step of a work item
constexpr int kOrdMidLanes = 8;          // lanes per medium vertex
constexpr int kOrdMidPer = kOrdMid / kOrdMidLanes;  // entries per lane of a medium vertex

// The lists a round fills for the next one.
struct OrdLists {
    int32_t *small;  // vertices of degree <= P.T1           (count cnt[kCntSmall])
    int32_t *mid;    // vertices of degree <= kOrdMid         (count cnt[kCntMulti])
    int4 *items;     // work items {V, q, slot, nch}          (count cnt[kCntChunks]; slots cnt[kCntItems])
    unsigned *cnt;   // the round's counter set
};

__device__ __forceinline__ OrdLists ord_lists(const RoundParams &P, int pass) {
    const bool odd = (pass & 1) != 0;
    return OrdLists{odd ? P.small0 : P.small1, odd ? P.mid0 : P.mid1, odd ? P.chunk0 : P.chunk1,
                    P.cnt + kCnt * (pass % 3)};
}

// Warp-wide exclusive prefix sum of x; `total` receives the sum over all lanes.
__device__ __forceinline__ unsigned warp_exclusive_sum(unsigned x, int lane, unsigned &total) {
    unsigned incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    total = __shfl_sync(kFull, incl, 31);
    return incl - x;
}

// Lists the ready vertices U[k] (those with ready[k]; up to K per lane) in L, with one atomic per
// list and warp: by degree on the small or the medium list, or as ceil(deg / P.CH) work items with
// an accumulator slot when there are several (warp-uniform call).
template <bool BATCH, int K>
__device__ void ord_list(const RoundParams &P, const bool (&ready)[K], const int32_t (&U)[K], const OrdLists &L,
                         int lane) {
    bool any = false;
#pragma unroll
    for (int k = 0; k < K; ++k) any |= ready[k];
    if (!__any_sync(kFull, any)) return;
    unsigned nch[K];  // work items of a larger vertex; 0 for a small or medium one or none
    uint8_t kind[K];  // 0 none, 1 small, 2 medium, 3 items
    unsigned ns = 0, nd = 0, ni = 0, nm = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        nch[k] = 0;
        kind[k] = 0;
        if (ready[k]) {
            const Row r = load_row<BATCH>(P, U[k]);
            const int64_t deg = r.e - r.b;
            kind[k] = deg <= P.T1 ? 1 : deg <= kOrdMid ? 2 : 3;
            if (kind[k] == 3) nch[k] = static_cast<unsigned>((deg + P.CH - 1) / P.CH);
        }
        ns += kind[k] == 1 ? 1u : 0u;
        nd += kind[k] == 2 ? 1u : 0u;
        ni += nch[k];
        nm += nch[k] > 1u ? 1u : 0u;
    }
    unsigned ts, td, ti, tm;
    unsigned sb = warp_exclusive_sum(ns, lane, ts);
    unsigned db = warp_exclusive_sum(nd, lane, td);
    unsigned ib = warp_exclusive_sum(ni, lane, ti);
    unsigned mb = warp_exclusive_sum(nm, lane, tm);
    unsigned b0 = 0, b1 = 0, b2 = 0, b3 = 0;
    if (lane == 0) {
        if (ts) b0 = atomicAdd(L.cnt + kCntSmall, ts);
        if (td) b1 = atomicAdd(L.cnt + kCntMulti, td);
        if (ti) b2 = atomicAdd(L.cnt + kCntChunks, ti);
        if (tm) b3 = atomicAdd(L.cnt + kCntItems, tm);
    }
    sb += __shfl_sync(kFull, b0, 0);
    db += __shfl_sync(kFull, b1, 0);
    ib += __shfl_sync(kFull, b2, 0);
    mb += __shfl_sync(kFull, b3, 0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (kind[k] == 1) {
            L.small[sb++] = U[k];
        } else if (kind[k] == 2) {
            L.mid[db++] = U[k];
        } else if (kind[k] == 3) {
            const int32_t slot = nch[k] > 1u ? static_cast<int32_t>(mb++) : -1;
            for (unsigned q = 0; q < nch[k]; ++q)
                L.items[ib + q] = make_int4(U[k], static_cast<int32_t>(q), slot, static_cast<int32_t>(nch[k]));
            ib += nch[k];
        }
    }
}

// Counts down the neighbours U[k] (those with take[k]): the ones whose count was `fire` before the
// decrement are listed (warp-uniform call).  Ordered mode: pend, fire 1 (the last smaller-key
// neighbour was colored).  Peeling: the residual degrees, fire k + 1 (the degree reached k).
template <bool BATCH, int K>
__device__ __forceinline__ void ord_release(const RoundParams &P, int32_t *pend, const bool (&take)[K],
                                            const int32_t (&U)[K], const OrdLists &L, int lane,
                                            int32_t fire = 1) {
    bool ready[K];
#pragma unroll
    for (int k = 0; k < K; ++k) ready[k] = take[k] && atomicSub(pend + U[k], 1) == fire;
    ord_list<BATCH, K>(P, ready, U, L, lane);
}

// Does neighbour u (local id lu, state word read on demand) have a smaller key than v?  With the
// hash key both keys are recomputed from the ids (the same order as key_less: the 31 priority bits
// are the top of the hash), so no state word is read; the other keys compare the state words.
template <bool HASH>
__device__ __forceinline__ bool smaller_key(const RoundParams &P, const unsigned long long *st, int32_t U,
                                            uint32_t lu, uint32_t lv, uint64_t hv, uint32_t pv) {
    if constexpr (HASH) {
        const uint64_t hu = vertex_hash(P.seed, lu);
        return hu != hv ? hu < hv : lu < lv;
    } else {
        return key_less(prio_of(__ldcg(st + U)), pv, lu, lv, P.seed);
    }
}

// pend[v] for every vertex, and the first round's lists (vertices with neighbours, none of them
// with a smaller key).  A warp takes 32 consecutive vertices, one per lane: a lane counts a row of
// up to 32 entries itself (four entries at a time), and the warp counts the longer rows one after
// another with all lanes; the ready vertices are listed together.  Vertices without neighbours
// were colored by setup.
template <bool BATCH, bool HASH>
__global__ void ord_count_kernel(RoundParams P, int32_t *pend) {
    constexpr int64_t kLaneRow = 32;  // longest row one lane counts alone
    const int lane = threadIdx.x & 31;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    const OrdLists L = ord_lists(P, P.pass_begin);
    const unsigned long long *st = reinterpret_cast<const unsigned long long *>(P.col0);
    for (int64_t base = (static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
         base < P.n; base += nw * 32) {
        const int32_t V = static_cast<int32_t>(base + lane);
        const bool valid = base + lane < P.n;
        Row r{};
        int64_t deg = 0;
        uint64_t hv = 0;
        uint32_t pv = 0;
        if (valid) {
            r = load_row<BATCH>(P, V);
            deg = r.e - r.b;
            if constexpr (HASH)
                hv = vertex_hash(P.seed, static_cast<uint32_t>(r.lv));
            else
                pv = prio_of(__ldcg(st + V));
        }
        unsigned c = 0;
        if (deg > 0 && deg <= kLaneRow) {
            for (int64_t j = r.b; j < r.e; j += 4) {
                int32_t u[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) u[t] = j + t < r.e ? load_entry(P.colidx + j + t) : 0;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (j + t >= r.e) continue;
                    const int32_t U = neighbour(P, r, u[t], j + t);
                    if (U >= 0 && smaller_key<HASH>(P, st, U, static_cast<uint32_t>(u[t]),
                                                    static_cast<uint32_t>(r.lv), hv, pv))
                        ++c;
                }
            }
        }
        unsigned big = __ballot_sync(kFull, deg > kLaneRow);
        while (big) {
            const int l = __ffs(big) - 1;
            big &= big - 1;
            const int32_t Vb = __shfl_sync(kFull, V, l);
            const Row rb = load_row<BATCH>(P, Vb);
            const uint64_t hb = __shfl_sync(kFull, hv, l);
            const uint32_t pb = __shfl_sync(kFull, pv, l);
            unsigned cb = 0;
            for (int64_t j = rb.b + lane; j < rb.e; j += 32) {
                const int32_t ul = load_entry(P.colidx + j);
                const int32_t U = neighbour(P, rb, ul, j);
                if (U >= 0 &&
                    smaller_key<HASH>(P, st, U, static_cast<uint32_t>(ul), static_cast<uint32_t>(rb.lv), hb, pb))
                    ++cb;
            }
            cb = __reduce_add_sync(kFull, cb);
            if (lane == l) c = cb;
        }
        if (valid) pend[V] = static_cast<int32_t>(c);
        const bool ready[1] = {valid && deg > 0 && c == 0};
        const int32_t Vs[1] = {V};
        ord_list<BATCH, 1>(P, ready, Vs, L, lane);
    }
}

// Ready vertices of degree <= P.T1 <= kOrdSmall, one per lane (lanes with `valid`; warp-uniform
// call): every entry loaded, then every state gathered, then the least color absent (at most
// deg(v) < 64) and the releases.
template <bool BATCH>
__device__ __forceinline__ void ord_small(const RoundParams &P, uint64_t *col, int32_t *pend, bool valid, int32_t V,
                                          const OrdLists &L, int pass, int lane, unsigned &st_deg,
                                          unsigned &st_cnt) {
    Row r{};
    int32_t deg = 0;
    uint64_t self = 0;
    if (valid) {
        r = load_row<BATCH>(P, V);
        deg = static_cast<int32_t>(r.e - r.b);
        self = load_state(col + V);
    }
    int32_t ul[kOrdSmall];
    uint64_t w[kOrdSmall];
#pragma unroll
    for (int k = 0; k < kOrdSmall; ++k) ul[k] = k < deg ? load_entry(P.colidx + r.b + k) : 0;
#pragma unroll
    for (int k = 0; k < kOrdSmall; ++k) {
        w[k] = kNoNeighbour;
        if (k < deg) {
            const int32_t U = neighbour(P, r, ul[k], r.b + k);
            if (U >= 0) w[k] = load_state(col + U);
        }
    }
    uint64_t mask = 0;
    bool take[kOrdSmall];
    int32_t U[kOrdSmall];
#pragma unroll
    for (int k = 0; k < kOrdSmall; ++k) {
        const int32_t c = color_of(w[k]);
        if (c >= 0 && c < 64) mask |= 1ull << c;
        take[k] = c < 0;
        U[k] = r.vbase + ul[k];
    }
    ord_release<BATCH, kOrdSmall>(P, pend, take, U, L, lane);
    if (valid) {
        col[V] = pack_state(__ffsll(static_cast<long long>(~mask)) - 1, prio_of(self), true);
        if constexpr (BATCH) note_graph_round(P, r.g, pass);
        st_deg += static_cast<unsigned>(deg);
        st_cnt += 1;
    }
}

// Ready vertices of degree in (P.T1, kOrdMid], one per 8-lane group (groups with `valid`;
// warp-uniform call): entry gl + 8k of the row in lane gl of the group, the group's colors OR-ed
// into one mask (the least color absent is at most deg(v) <= kOrdMid < 64).
template <bool BATCH>
__device__ __forceinline__ void ord_mid(const RoundParams &P, uint64_t *col, int32_t *pend, bool valid, int32_t V,
                                        const OrdLists &L, int pass, int lane, unsigned &st_deg, unsigned &st_cnt) {
    const int gl = lane & (kOrdMidLanes - 1);
    Row r{};
    int32_t deg = 0;
    if (valid) {
        r = load_row<BATCH>(P, V);
        deg = static_cast<int32_t>(r.e - r.b);
    }
    const uint64_t self = valid && gl == 0 ? load_state(col + V) : 0;
    int32_t ul[kOrdMidPer];
    uint64_t w[kOrdMidPer];
#pragma unroll
    for (int k = 0; k < kOrdMidPer; ++k) {
        const int32_t e = gl + kOrdMidLanes * k;
        ul[k] = e < deg ? load_entry(P.colidx + r.b + e) : 0;
    }
#pragma unroll
    for (int k = 0; k < kOrdMidPer; ++k) {
        const int32_t e = gl + kOrdMidLanes * k;
        w[k] = kNoNeighbour;
        if (e < deg) {
            const int32_t U = neighbour(P, r, ul[k], r.b + e);
            if (U >= 0) w[k] = load_state(col + U);
        }
    }
    uint64_t mask = 0;
    bool take[kOrdMidPer];
    int32_t U[kOrdMidPer];
#pragma unroll
    for (int k = 0; k < kOrdMidPer; ++k) {
        const int32_t c = color_of(w[k]);
        if (c >= 0 && c < 64) mask |= 1ull << c;
        take[k] = c < 0;
        U[k] = r.vbase + ul[k];
    }
#pragma unroll
    for (int o = 1; o < kOrdMidLanes; o <<= 1) mask |= __shfl_xor_sync(kFull, mask, o);
    ord_release<BATCH, kOrdMidPer>(P, pend, take, U, L, lane);
    if (valid && gl == 0) {
        col[V] = pack_state(__ffsll(static_cast<long long>(~mask)) - 1, prio_of(self), true);
        if constexpr (BATCH) note_graph_round(P, r.g, pass);
        st_deg += static_cast<unsigned>(deg);
        st_cnt += 1;
    }
}

// One work item {V, q, slot, nch} of a larger ready vertex (one warp): entries
// [q P.CH, (q + 1) P.CH) of its row.  Colors of colored neighbours go into the window [0, 512)
// (0..63 in registers, the rest in win); the last of the vertex's items picks the color.
template <bool BATCH>
__device__ void ord_item(const RoundParams &P, uint64_t *col, int32_t *pend, int4 it, unsigned *win,
                         const OrdLists &L, int pass, int lane, unsigned &st_deg, unsigned &st_cnt) {
    const int32_t V = it.x, q = it.y, slot = it.z, nch = it.w;
    const Row r = load_row<BATCH>(P, V);
    const int64_t jb = r.b + static_cast<int64_t>(q) * P.CH;
    const int64_t je = min(r.e, jb + P.CH);
    if (lane < kAccWords) win[lane] = 0;
    __syncwarp();
    uint64_t lo = 0;
    for (int64_t j0 = jb; j0 < je; j0 += 32 * kOrdPer) {
        int32_t ul[kOrdPer];
        uint64_t w[kOrdPer];
#pragma unroll
        for (int k = 0; k < kOrdPer; ++k) {
            const int64_t j = j0 + lane + 32 * k;
            ul[k] = j < je ? load_entry(P.colidx + j) : 0;
        }
#pragma unroll
        for (int k = 0; k < kOrdPer; ++k) {
            const int64_t j = j0 + lane + 32 * k;
            w[k] = kNoNeighbour;
            if (j < je) {
                const int32_t U = neighbour(P, r, ul[k], j);
                if (U >= 0) w[k] = load_state(col + U);
            }
        }
        bool take[kOrdPer];
        int32_t U[kOrdPer];
#pragma unroll
        for (int k = 0; k < kOrdPer; ++k) {
            const int32_t c = color_of(w[k]);
            if (c >= 0 && c < 64)
                lo |= 1ull << c;
            else if (c >= 64 && c < 32 * kAccWords)
                atomicOr(&win[c >> 5], 1u << (c & 31));
            take[k] = c < 0;
            U[k] = r.vbase + ul[k];
        }
        ord_release<BATCH, kOrdPer>(P, pend, take, U, L, lane);
    }
    unsigned lo0 = __reduce_or_sync(kFull, static_cast<unsigned>(lo));
    unsigned lo1 = __reduce_or_sync(kFull, static_cast<unsigned>(lo >> 32));
    __syncwarp();
    if (lane == 0) {
        st_deg += static_cast<unsigned>(je - jb);
        st_cnt += q == 0 ? 1u : 0u;
    }
    bool unused = false;
    if (nch > 1 && !merge_item<true>(P.acc + static_cast<size_t>(slot) * kOrdSlotWords, nch, lane, lo0, lo1, win,
                                     unused, 0u))
        return;
    int32_t nc = first_free(lo0, lo1, win);
    // every neighbour with a larger key is still uncolored, so the whole row's colors are the
    // smaller-key neighbours' colors
    if (nc < 0) nc = mex_from<BATCH>(P, col, r, win, lane, 32 * kAccWords);
    if (lane == 0) {
        col[V] = pack_state(nc, prio_of(load_state(col + V)), true);
        if constexpr (BATCH) note_graph_round(P, r.g, pass);
    }
    __syncwarp();
}

// Rounds of the ordered mode: each round runs the ready work items (one warp each), the medium
// vertices (four per warp) and the small ones (32 per warp), each kind starting at the warp after
// the previous kind's last, so that few warps get two; the vertices they release form the next
// round's lists.  When the lists run dry, a vertex still uncolored means the input was not
// symmetric.
template <bool BATCH>
__global__ void __launch_bounds__(kBlock, kWideBlocks) ord_round_kernel(RoundParams P, int32_t *pend) {
    __shared__ unsigned s_win[kMaxWarps][kAccWords];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    const unsigned gw = blockIdx.x * (blockDim.x >> 5) + wib;
    unsigned *win = s_win[wib];
    uint64_t *col = P.col0;
    if (P.stats && blockIdx.x == 0 && threadIdx.x == 0) P.stats[4 * P.stats_cap] = global_ns();
    unsigned bar_target = 0;
    bool drained = false;
    int pass = P.pass_begin;
    for (;; ++pass) {
        const OrdLists C = ord_lists(P, pass), L = ord_lists(P, pass + 1);
        const unsigned nsmall = __ldcg(C.cnt + kCntSmall), nmid = __ldcg(C.cnt + kCntMulti);
        const unsigned nitems = __ldcg(C.cnt + kCntChunks);
        if (nsmall + nmid + nitems == 0u) {
            drained = true;
            break;
        }
        if (pass >= P.pass_end) {
            if (P.cap_is_error && blockIdx.x == 0 && threadIdx.x == 0)
                set_error(P.err, GC_ERR_NO_CONVERGENCE, pass, 0);
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x < kCnt) P.cnt[kCnt * ((pass + 2) % 3) + threadIdx.x] = 0u;
        unsigned st_deg = 0, st_cnt = 0;
        for (unsigned i = gw; i < nitems; i += nw)
            ord_item<BATCH>(P, col, pend, __ldcg(C.items + i), win, L, pass, lane, st_deg, st_cnt);
        const unsigned mid_groups = (nmid + 3u) / 4u;
        for (unsigned b = (gw + nw - nitems % nw) % nw; b < mid_groups; b += nw) {
            const unsigned i = 4u * b + static_cast<unsigned>(lane >> 3);
            ord_mid<BATCH>(P, col, pend, i < nmid, i < nmid ? __ldcg(C.mid + i) : 0, L, pass, lane, st_deg, st_cnt);
        }
        const unsigned skip = (nitems + mid_groups) % nw;
        for (unsigned base = ((gw + nw - skip) % nw) * 32u; base < nsmall; base += nw * 32u) {
            const unsigned i = base + lane;
            ord_small<BATCH>(P, col, pend, i < nsmall, i < nsmall ? __ldcg(C.small + i) : 0, L, pass, lane, st_deg,
                             st_cnt);
        }
        if (P.stats) flush_stats(P, pass, st_deg, st_cnt, st_deg);
        if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) break;
    }
    if (drained) {
        for (int64_t V = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; V < P.n;
             V += static_cast<int64_t>(gridDim.x) * blockDim.x)
            if (color_of(__ldcg(reinterpret_cast<const unsigned long long *>(col) + V)) < 0)
                set_error(P.err, GC_ERR_INVALID_GRAPH, static_cast<int32_t>(V), -1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.passes[0] = pass;
        P.passes[1] = pass - 1;
    }
}

// ------------------------------------------------------------------------------------------
// smallest-last order (GC_PRIORITY_SMALLEST_LAST, single graphs): batch peeling.  res[v] starts
// at deg(v), level[v] at 0 (present), the threshold k at 0.  While vertices remain, k becomes
// max(k, least res among them); then, level after level, every present vertex with res <= k is
// removed together (level[v] = the level's number) and lowers res of each neighbour by one.  A
// present vertex whose res falls from k + 1 to k joins the next level, so every level after the
// first of a threshold is listed by the decrements (one atomic each, as the ordered mode's counts),
// and each vertex is listed once.  The lists and their degree classes are the ordered mode's.
// Decrements of removed vertices are harmless: their res is already <= k and never fires.

// res, level and the two threshold words (the least res of a search, alternating).
__global__ void peel_init_kernel(RoundParams P, int32_t *res, int32_t *level, unsigned *kw, unsigned *items) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) kw[0] = kw[1] = 0x7fffffffu;
    for (int64_t base = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) & ~31ll; base < P.n;
         base += stride) {
        const int64_t V = base + lane;
        unsigned nch = 0;
        if (V < P.n) {
            int64_t b;
            int32_t lv;
            int64_t d = checked_degree<false>(P, static_cast<int32_t>(V), 0, b, lv);
            if (d < 0) {
                set_error(P.err, GC_ERR_INVALID_GRAPH, static_cast<int32_t>(V), b);
                d = 0;
            }
            res[V] = static_cast<int32_t>(d);
            level[V] = 0;
            if (d > kOrdMid) nch = static_cast<unsigned>((d + P.CH - 1) / P.CH);
        }
        nch = __reduce_add_sync(kFull, nch);
        if (lane == 0 && nch) atomicAdd(items, nch);
    }
}

// One level for the vertices of degree <= P.T1, one per lane (lanes with `valid`).
__device__ __forceinline__ void peel_small(const RoundParams &P, int32_t *res, int32_t *level, bool valid, int32_t V,
                                           int32_t k, int32_t L, const OrdLists &N, int lane) {
    int64_t b = 0;
    int32_t deg = 0;
    if (valid) {
        b = __ldg(P.rowptr + V);
        deg = static_cast<int32_t>(__ldg(P.rowptr + V + 1) - b);
        level[V] = L;
    }
    bool take[kOrdSmall];
    int32_t U[kOrdSmall];
#pragma unroll
    for (int q = 0; q < kOrdSmall; ++q) {
        U[q] = q < deg ? load_entry(P.colidx + b + q) : 0;
        take[q] = q < deg && static_cast<uint32_t>(U[q]) < static_cast<uint32_t>(P.n) && U[q] != V;
        if (q < deg && !take[q]) set_error(P.err, GC_ERR_INVALID_GRAPH, V, b + q);
    }
    ord_release<false, kOrdSmall>(P, res, take, U, N, lane, k + 1);
}

// One level for the vertices of degree in (P.T1, kOrdMid], one per 8-lane group.
__device__ __forceinline__ void peel_mid(const RoundParams &P, int32_t *res, int32_t *level, bool valid, int32_t V,
                                         int32_t k, int32_t L, const OrdLists &N, int lane) {
    const int gl = lane & (kOrdMidLanes - 1);
    int64_t b = 0;
    int32_t deg = 0;
    if (valid) {
        b = __ldg(P.rowptr + V);
        deg = static_cast<int32_t>(__ldg(P.rowptr + V + 1) - b);
        if (gl == 0) level[V] = L;
    }
    bool take[kOrdMidPer];
    int32_t U[kOrdMidPer];
#pragma unroll
    for (int q = 0; q < kOrdMidPer; ++q) {
        const int32_t e = gl + kOrdMidLanes * q;
        U[q] = e < deg ? load_entry(P.colidx + b + e) : 0;
        take[q] = e < deg && static_cast<uint32_t>(U[q]) < static_cast<uint32_t>(P.n) && U[q] != V;
        if (e < deg && !take[q]) set_error(P.err, GC_ERR_INVALID_GRAPH, V, b + e);
    }
    ord_release<false, kOrdMidPer>(P, res, take, U, N, lane, k + 1);
}

// One level for a work item {V, q, slot, nch} of a larger vertex (one warp).
__device__ __forceinline__ void peel_item(const RoundParams &P, int32_t *res, int32_t *level, int4 it, int32_t k,
                                          int32_t L, const OrdLists &N, int lane) {
    const int32_t V = it.x, q = it.y;
    const int64_t b = __ldg(P.rowptr + V), e = __ldg(P.rowptr + V + 1);
    const int64_t jb = b + static_cast<int64_t>(q) * P.CH;
    const int64_t je = min(e, jb + P.CH);
    if (q == 0 && lane == 0) level[V] = L;
    for (int64_t j0 = jb; j0 < je; j0 += 32 * kOrdPer) {
        bool take[kOrdPer];
        int32_t U[kOrdPer];
#pragma unroll
        for (int t = 0; t < kOrdPer; ++t) {
            const int64_t j = j0 + lane + 32 * t;
            U[t] = j < je ? load_entry(P.colidx + j) : 0;
            take[t] = j < je && static_cast<uint32_t>(U[t]) < static_cast<uint32_t>(P.n) && U[t] != V;
            if (j < je && !take[t]) set_error(P.err, GC_ERR_INVALID_GRAPH, V, j);
        }
        ord_release<false, kOrdPer>(P, res, take, U, N, lane, k + 1);
    }
}

// The whole peeling in one cooperative launch; passes[0] receives the number of levels and
// passes[1] the last threshold (the degeneracy).  Each threshold search scans the vertices the
// previous one left (all vertices for the first), and its listing scan writes the ones it does not
// list to the other of rlist0 / rlist1 (counts rcnt[0] / rcnt[1], zero at launch), so that the
// scans shrink with the graph.
__global__ void __launch_bounds__(kBlock, kWideBlocks) peel_kernel(RoundParams P, int32_t *res, int32_t *level,
                                                                   unsigned *kw, int32_t *rlist0, int32_t *rlist1,
                                                                   unsigned *rcnt) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    const unsigned gw = blockIdx.x * (blockDim.x >> 5) + wib;
    const int64_t nthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t gtid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    unsigned bar_target = 0;
    int32_t k = 0, L = 0;
    int pass = P.pass_begin;
    bool ok = true;
    for (int f = 0; ok; ++f) {
        // the vertices to scan: all of them first, then those the previous search left
        const int32_t *rcur = (f & 1) ? rlist1 : rlist0;
        int32_t *rnext = (f & 1) ? rlist0 : rlist1;
        const int64_t nr = f == 0 ? P.n : static_cast<int64_t>(__ldcg(rcnt + (f & 1)));
        if (blockIdx.x == 0 && threadIdx.x == 0) rcnt[(f + 1) & 1] = 0u;
        // the least res among the present vertices
        unsigned m = 0x7fffffffu;
        for (int64_t i = gtid; i < nr; i += nthreads) {
            const int32_t v = f == 0 ? static_cast<int32_t>(i) : __ldcg(rcur + i);
            if (__ldcg(level + v) == 0) m = min(m, static_cast<unsigned>(__ldcg(res + v)));
        }
        m = __reduce_min_sync(kFull, m);
        if (lane == 0 && m != 0x7fffffffu) atomicMin(kw + (f & 1), m);
        if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) break;
        const unsigned kmin = __ldcg(kw + (f & 1));
        if (blockIdx.x == 0 && threadIdx.x == 0) kw[(f + 1) & 1] = 0x7fffffffu;
        if (kmin == 0x7fffffffu) break;  // every vertex removed
        if (static_cast<int32_t>(kmin) > k) k = static_cast<int32_t>(kmin);
        // the first level of this threshold: every present vertex with res <= k; the other present
        // vertices are left for the next search
        {
            const OrdLists F = ord_lists(P, pass);
            for (int64_t base = gtid & ~31ll; base < nr; base += nthreads) {
                const int64_t i = base + lane;
                int32_t v = 0;
                bool present = false, now = false;
                if (i < nr) {
                    v = f == 0 ? static_cast<int32_t>(i) : __ldcg(rcur + i);
                    present = __ldcg(level + v) == 0;
                    now = present && __ldcg(res + v) <= k;
                }
                warp_append(present && !now, v, rnext, rcnt + ((f + 1) & 1), lane);
                const bool ready[1] = {now};
                const int32_t Vs[1] = {v};
                ord_list<false, 1>(P, ready, Vs, F, lane);
            }
        }
        if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) break;
        for (;; ++pass) {
            const OrdLists C = ord_lists(P, pass), N = ord_lists(P, pass + 1);
            const unsigned nsmall = __ldcg(C.cnt + kCntSmall), nmid = __ldcg(C.cnt + kCntMulti);
            const unsigned nitems = __ldcg(C.cnt + kCntChunks);
            if (nsmall + nmid + nitems == 0u) break;
            if (blockIdx.x == 0 && threadIdx.x < kCnt) P.cnt[kCnt * ((pass + 2) % 3) + threadIdx.x] = 0u;
            ++L;
            for (unsigned i = gw; i < nitems; i += nw) peel_item(P, res, level, __ldcg(C.items + i), k, L, N, lane);
            const unsigned mid_groups = (nmid + 3u) / 4u;
            for (unsigned b = (gw + nw - nitems % nw) % nw; b < mid_groups; b += nw) {
                const unsigned i = 4u * b + static_cast<unsigned>(lane >> 3);
                peel_mid(P, res, level, i < nmid, i < nmid ? __ldcg(C.mid + i) : 0, k, L, N, lane);
            }
            const unsigned skip = (nitems + mid_groups) % nw;
            for (unsigned base = ((gw + nw - skip) % nw) * 32u; base < nsmall; base += nw * 32u) {
                const unsigned i = base + lane;
                peel_small(P, res, level, i < nsmall, i < nsmall ? __ldcg(C.small + i) : 0, k, L, N, lane);
            }
            if (!grid_sync(P.bar, bar_target, P.err, P.spin_ns)) {
                ok = false;
                break;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.passes[0] = L;
        P.passes[1] = k;
    }
}

// Final statistics over vertices [v_begin, v_end): one bit per (graph, color), largest color per
// graph, and an optional copy of the colors.
template <bool BATCH>
__global__ void __launch_bounds__(256) count_mark_kernel(RoundParams P, const int32_t *colors_sel, int32_t v_begin,
                                                         int32_t v_end, unsigned *bitmap, int32_t *gmax, int32_t *out) {
    // single graph: colors below kMarkWords * 32 are marked in a shared bitmap and the largest color is
    // reduced per block first (every thread hitting the same few words and the same maximum would
    // serialise on them)
    constexpr int kMarkWords = 128;
    __shared__ unsigned s_bits[kMarkWords];
    __shared__ int32_t s_max;
    if (!BATCH) {
        for (int t = threadIdx.x; t < kMarkWords; t += blockDim.x) s_bits[t] = 0u;
        if (threadIdx.x == 0) s_max = -1;
        __syncthreads();
    }
    const uint64_t *state = (colors_sel && (*colors_sel & 1)) ? P.col1 : P.col0;
    const bool copy = out != nullptr && P.err[0] == 0;
    const int64_t count = static_cast<int64_t>(v_end) - v_begin;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int32_t tmax = -1;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
        const int32_t V = static_cast<int32_t>(v_begin + i);
        const int32_t c = color_of(__ldcg(state + V));
        if (copy) out[i] = c;
        if (c < 0) continue;
        if (!BATCH && c < 32 * kMarkWords) {
            const unsigned m = 1u << (c & 31);
            if (!(s_bits[c >> 5] & m)) atomicOr(&s_bits[c >> 5], m);
            tmax = max(tmax, c);
            continue;
        }
        int32_t g = 0;
        int64_t bit = c;
        if constexpr (BATCH) {
            g = P.vg[V];
            bit += P.g_vbase[g];
        }
        const unsigned m = 1u << (bit & 31);
        unsigned *w = bitmap + (bit >> 5);
        if (!(__ldcg(w) & m)) atomicOr(w, m);
        if (__ldcg(gmax + g) < c) atomicMax(gmax + g, c);
    }
    if (!BATCH) {
        tmax = __reduce_max_sync(kFull, tmax);
        if ((threadIdx.x & 31) == 0 && tmax >= 0) atomicMax(&s_max, tmax);
        __syncthreads();
        for (int t = threadIdx.x; t < kMarkWords; t += blockDim.x)
            if (s_bits[t]) atomicOr(bitmap + t, s_bits[t]);
        if (threadIdx.x == 0 && s_max >= 0 && __ldcg(gmax) < s_max) atomicMax(gmax, s_max);
    }
}

// Distinct colors of graphs [g_begin, g_end): popcount of bits [base, base + gmax[g] + 1) where base
// is the graph's first vertex id (colors of graph g are < its vertex count).  One warp per graph.
template <bool BATCH>
__global__ void count_pop_kernel(RoundParams P, int32_t g_begin, int32_t g_end, const unsigned *bitmap,
                                 const int32_t *gmax, int32_t *gcount) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int32_t g = g_begin + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < g_end; g += nw) {
        const int64_t lo = BATCH ? P.g_vbase[g] : 0;
        const int64_t hi = lo + static_cast<int64_t>(gmax[g]) + 1;  // gmax = -1 for an empty graph
        unsigned cnt = 0;
        if (hi > lo) {
            for (int64_t w = (lo >> 5) + lane; w <= ((hi - 1) >> 5); w += 32) {
                unsigned x = bitmap[w];
                const int64_t wb = w << 5;
                if (wb < lo) x &= ~0u << (lo - wb);
                if (hi - wb < 32) x &= (1u << (hi - wb)) - 1u;
                cnt += __popc(x);
            }
        }
        cnt = __reduce_add_sync(kFull, cnt);
        if (lane == 0) gcount[g] = static_cast<int32_t>(cnt);
    }
}

// Graph-format check (gc_validate_graph); one warp per vertex.
__global__ void validate_kernel(int32_t n, const int32_t *rowptr, const int32_t *colidx, int flags, int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int64_t nnz = rowptr[n];
    for (int32_t v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += nw) {
        const int64_t b = rowptr[v], e = rowptr[v + 1];
        if (b < 0 || e < b || e > nnz || (v == 0 && b != 0)) {
            if (lane == 0) set_error(err, GC_ERR_INVALID_GRAPH, v, b);
            continue;
        }
        for (int64_t j = b + lane; j < e; j += 32) {
            const int32_t u = colidx[j];
            if (u < 0 || u >= n || u == v) {
                set_error(err, GC_ERR_INVALID_GRAPH, v, j);
                continue;
            }
            if ((flags & GC_VALIDATE_SORTED) && j > b && colidx[j - 1] >= u) set_error(err, GC_ERR_INVALID_GRAPH, v, j);
            if (flags & GC_VALIDATE_SYMMETRIC) {
                int64_t lo = rowptr[u], hi = rowptr[u + 1];
                if (lo < 0 || hi < lo || hi > nnz) continue;  // that row reports itself
                bool found = false;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    const int32_t x = colidx[mid];
                    if (x == v) {
                        found = true;
                        break;
                    }
                    if (x < v)
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                if (!found) set_error(err, GC_ERR_INVALID_GRAPH, v, j);
            }
        }
    }
}

// One fused deterministic round over a list of worklist vertices, for callers that own a block of
// a graph's vertices and exchange colors between rounds themselves (Algorithm 1's partitions V_i):
// reading C_r (`cur`, every vertex), vertex v = work[i] lost iff a neighbour u has C_r[u] = C_r[v]
// and key(u) < key(v); next[i] is its color for round r+1: the least color absent from C_r over
// its neighbours if it lost, else C_r[v].  One warp per vertex; the least free color is found a
// window of 1024 colors at a time.  Malformed rows or entries post GC_ERR_INVALID_GRAPH.
__global__ void det_round_block_kernel(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed,
                                       const int32_t *cur, const int32_t *work, int32_t nwork, int32_t *next,
                                       int32_t *lost, int32_t *err) {
    __shared__ unsigned s_win[8][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned *win = s_win[wib];
    const int64_t nw = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + wib; i < nwork; i += nw) {
        const int32_t v = __ldg(work + i);
        if (static_cast<uint32_t>(v) >= static_cast<uint32_t>(n)) {
            if (lane == 0) set_error(err, GC_ERR_INVALID_ARG, v, i);
            continue;
        }
        const int64_t b = __ldg(rowptr + v), e = __ldg(rowptr + v + 1);
        if (b < 0 || e < b || e > __ldg(rowptr + n)) {
            if (lane == 0) set_error(err, GC_ERR_INVALID_GRAPH, v, b);
            continue;
        }
        const int32_t cv = __ldg(cur + v);
        const uint64_t hv = vertex_hash(seed, static_cast<uint32_t>(v));
        bool lose = false;
        for (int64_t j = b + lane; j < e; j += 32) {
            const int32_t u = __ldg(colidx + j);
            if (static_cast<uint32_t>(u) >= static_cast<uint32_t>(n) || u == v) {
                set_error(err, GC_ERR_INVALID_GRAPH, v, j);
                continue;
            }
            if (__ldg(cur + u) == cv) {
                const uint64_t hu = vertex_hash(seed, static_cast<uint32_t>(u));
                lose |= hu < hv || (hu == hv && u < v);
            }
        }
        lose = __any_sync(kFull, lose);
        int32_t nc = cv;
        for (int32_t base = 0; lose; base += 1024) {
            win[lane] = 0u;
            __syncwarp();
            for (int64_t j = b + lane; j < e; j += 32) {
                const int32_t u = __ldg(colidx + j);
                if (static_cast<uint32_t>(u) >= static_cast<uint32_t>(n)) continue;
                const int32_t c = __ldg(cur + u) - base;
                if (static_cast<unsigned>(c) < 1024u) atomicOr(&win[c >> 5], 1u << (c & 31));
            }
            __syncwarp();
            const unsigned open = __ballot_sync(kFull, win[lane] != ~0u);
            if (open) {
                const int l = __ffs(open) - 1;
                nc = base + 32 * l + __ffs(~win[l]) - 1;
                break;
            }
            __syncwarp();
        }
        if (lane == 0) {
            next[i] = nc;
            lost[i] = lose ? 1 : 0;
        }
    }
}

}  // namespace

// ------------------------------------------------------------------------------------------
// launch wrappers

static int grid_for(int64_t work, int block, int cap) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return static_cast<int>(g);
}

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

cudaError_t launch_batch_tables(const RoundParams &P, const int64_t *vtx_off, const int64_t *edge_off,
                                int64_t *g_vbase, int32_t *g_n, int64_t *g_ebase, int64_t *g_rbase, int64_t *g_m,
                                cudaStream_t s) {
    batch_tables_kernel<<<grid_for(P.G, 1, 65535), 256, 0, s>>>(P, vtx_off, edge_off, g_vbase, g_n, g_ebase, g_rbase,
                                                                g_m);
    return cudaGetLastError();
}

cudaError_t launch_setup(const RoundParams &P, int mode, bool batch, int32_t v_begin, int32_t v_end,
                         int32_t g_fixed, cudaStream_t s) {
    if (v_end <= v_begin) return cudaSuccess;
    const int grid = grid_for(static_cast<int64_t>(v_end) - v_begin, 256, sm_count() * 16);
    if (batch) {
        if (mode == GC_MODE_DETERMINISTIC)
            setup_kernel<true, GC_MODE_DETERMINISTIC><<<grid, 256, 0, s>>>(P, v_begin, v_end, g_fixed);
        else
            setup_kernel<true, GC_MODE_INPLACE><<<grid, 256, 0, s>>>(P, v_begin, v_end, g_fixed);
    } else {
        if (mode == GC_MODE_DETERMINISTIC)
            setup_kernel<false, GC_MODE_DETERMINISTIC><<<grid, 256, 0, s>>>(P, v_begin, v_end, g_fixed);
        else
            setup_kernel<false, GC_MODE_INPLACE><<<grid, 256, 0, s>>>(P, v_begin, v_end, g_fixed);
    }
    return cudaGetLastError();
}

int32_t sort_shift(int64_t n) {
    // one block (a plain degree sort) while both state buffers (16 bytes a vertex) fit well inside
    // L2; blocks of 2^17 ids beyond that
    return 16 * n <= (int64_t{96} << 20) ? 30 : 17;
}

int32_t sort_bins(int32_t v_end, int32_t shift) { return ((v_end >> shift) + 1) * 128; }

cudaError_t launch_sort_small(const RoundParams &P, bool batch, int32_t v_begin, int32_t v_end, cudaStream_t s) {
    if (v_end <= v_begin || !P.deg_hist) return cudaSuccess;
    if (v_begin % 256 != 0) return cudaErrorInvalidValue;
    const int32_t nbins = sort_bins(v_end, P.sort_shift);
    sort_small_kernel<<<1, kSortThreads, 0, s>>>(P, nbins);
    const int grid = grid_for(static_cast<int64_t>(v_end) - v_begin, 256, sm_count() * 16);
    if (batch)
        scatter_small_kernel<true><<<grid, 256, 0, s>>>(P, v_begin, v_end, nbins);
    else
        scatter_small_kernel<false><<<grid, 256, 0, s>>>(P, v_begin, v_end, nbins);
    return cudaGetLastError();
}

cudaError_t launch_expand(const RoundParams &P, int mode, bool batch, bool compact, int32_t n_items,
                          cudaStream_t s) {
    if (n_items == 0) return cudaSuccess;
    const int grid = n_items < 0 ? sm_count() * 8 : grid_for(static_cast<int64_t>(n_items), 256, sm_count() * 8);
    constexpr int D = GC_MODE_DETERMINISTIC, I = GC_MODE_INPLACE;
    if (mode == GC_MODE_DETERMINISTIC) {
        if (batch) {
            if (compact)
                expand_kernel<true, true, D><<<grid, 256, 0, s>>>(P, n_items);
            else
                expand_kernel<true, false, D><<<grid, 256, 0, s>>>(P, n_items);
        } else {
            if (compact)
                expand_kernel<false, true, D><<<grid, 256, 0, s>>>(P, n_items);
            else
                expand_kernel<false, false, D><<<grid, 256, 0, s>>>(P, n_items);
        }
    } else {
        if (batch) {
            if (compact)
                expand_kernel<true, true, I><<<grid, 256, 0, s>>>(P, n_items);
            else
                expand_kernel<true, false, I><<<grid, 256, 0, s>>>(P, n_items);
        } else {
            if (compact)
                expand_kernel<false, true, I><<<grid, 256, 0, s>>>(P, n_items);
            else
                expand_kernel<false, false, I><<<grid, 256, 0, s>>>(P, n_items);
        }
    }
    return cudaGetLastError();
}

template <int MINB>
static const void *round_kernel_variant(int mode, bool batch, bool compact) {
    if (mode == GC_MODE_DETERMINISTIC) {
        if (batch)
            return compact ? reinterpret_cast<const void *>(&det_round_kernel<true, true, MINB>)
                           : reinterpret_cast<const void *>(&det_round_kernel<true, false, MINB>);
        return compact ? reinterpret_cast<const void *>(&det_round_kernel<false, true, MINB>)
                       : reinterpret_cast<const void *>(&det_round_kernel<false, false, MINB>);
    }
    if (batch)
        return compact ? reinterpret_cast<const void *>(&ip_round_kernel<true, true, MINB>)
                       : reinterpret_cast<const void *>(&ip_round_kernel<true, false, MINB>);
    return compact ? reinterpret_cast<const void *>(&ip_round_kernel<false, true, MINB>)
                   : reinterpret_cast<const void *>(&ip_round_kernel<false, false, MINB>);
}

static const void *round_kernel_fn(int mode, bool batch, bool compact, bool wide) {
    return wide ? round_kernel_variant<kWideBlocks>(mode, batch, compact)
                : round_kernel_variant<kNarrowBlocks>(mode, batch, compact);
}

cudaError_t round_kernel_occupancy(int mode, bool batch, bool compact, int block, int *blocks_per_sm, bool wide) {
    if (block != kBlock) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, round_kernel_fn(mode, batch, compact, wide),
                                                         block, 0);
}

cudaError_t launch_rounds(const RoundParams &P, int mode, bool batch, bool compact, int grid, int block,
                          cudaStream_t s, bool wide) {
    if (block != kBlock) return cudaErrorInvalidValue;
    // the grid barrier counts this launch's arrivals from zero
    cudaError_t e = cudaMemsetAsync(&P.bar->count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    RoundParams arg = P;
    void *args[] = {&arg};
    return cudaLaunchCooperativeKernel(round_kernel_fn(mode, batch, compact, wide), dim3(grid), dim3(block), args, 0,
                                       s);
}

cudaError_t launch_partition_init(const RoundParams &P, cudaStream_t s) {
    if (P.n <= 0) return cudaSuccess;
    part_init_kernel<<<grid_for(P.n, 256, sm_count() * 16), 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t partition_kernel_occupancy(int block, int *blocks_per_sm) {
    if (block != kBlock) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, part_round_kernel, block, 0);
}

cudaError_t launch_partition_rounds(const RoundParams &P, int32_t p, int grid, int block, cudaStream_t s) {
    if (block != kBlock) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(&P.bar->count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    RoundParams arg = P;
    int32_t parg = p;
    void *args[] = {&arg, &parg};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(&part_round_kernel), dim3(grid), dim3(block),
                                       args, 0, s);
}

cudaError_t ordered_kernel_occupancy(bool batch, int block, int *blocks_per_sm) {
    if (block != kBlock) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm,
        batch ? reinterpret_cast<const void *>(&ord_round_kernel<true>)
              : reinterpret_cast<const void *>(&ord_round_kernel<false>),
        block, 0);
}

cudaError_t launch_ordered(const RoundParams &P, bool batch, int32_t *pend, int grid, int block, cudaStream_t s) {
    if (block != kBlock) return cudaErrorInvalidValue;
    if (P.n <= 0) return cudaSuccess;
    const int cgrid = grid_for(static_cast<int64_t>(P.n) * 32, 256, sm_count() * 16);
    const bool hash = P.priority == GC_PRIORITY_HASH;
    if (batch) {
        if (hash)
            ord_count_kernel<true, true><<<cgrid, 256, 0, s>>>(P, pend);
        else
            ord_count_kernel<true, false><<<cgrid, 256, 0, s>>>(P, pend);
    } else {
        if (hash)
            ord_count_kernel<false, true><<<cgrid, 256, 0, s>>>(P, pend);
        else
            ord_count_kernel<false, false><<<cgrid, 256, 0, s>>>(P, pend);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(&P.bar->count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    RoundParams arg = P;
    int32_t *parg = pend;
    void *args[] = {&arg, &parg};
    return cudaLaunchCooperativeKernel(batch ? reinterpret_cast<const void *>(&ord_round_kernel<true>)
                                             : reinterpret_cast<const void *>(&ord_round_kernel<false>),
                                       dim3(grid), dim3(block), args, 0, s);
}

cudaError_t launch_peel_init(const RoundParams &P, int32_t *res, int32_t *level, unsigned *kw, unsigned *items,
                             cudaStream_t s) {
    const int grid = grid_for(P.n > 0 ? P.n : 1, 256, sm_count() * 16);
    peel_init_kernel<<<grid, 256, 0, s>>>(P, res, level, kw, items);
    return cudaGetLastError();
}

cudaError_t peel_kernel_occupancy(int block, int *blocks_per_sm) {
    if (block != kBlock) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, reinterpret_cast<const void *>(&peel_kernel),
                                                         block, 0);
}

cudaError_t launch_peel(const RoundParams &P, int32_t *res, int32_t *level, unsigned *kw, int32_t *rlist0,
                        int32_t *rlist1, unsigned *rcnt, int grid, int block, cudaStream_t s) {
    if (block != kBlock) return cudaErrorInvalidValue;
    if (P.n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(&P.bar->count, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(rcnt, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    RoundParams arg = P;
    int32_t *ra = res, *la = level, *r0 = rlist0, *r1 = rlist1;
    unsigned *ka = kw, *rc = rcnt;
    void *args[] = {&arg, &ra, &la, &ka, &r0, &r1, &rc};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(&peel_kernel), dim3(grid), dim3(block), args, 0,
                                       s);
}

cudaError_t launch_count_colors(const RoundParams &P, bool batch, const int32_t *colors_sel, int32_t v_begin,
                                int32_t v_end, int32_t g_begin, int32_t g_end, unsigned *bitmap, int32_t *gmax,
                                int32_t *gcount, int32_t *out, cudaStream_t s) {
    if (v_end > v_begin) {
        const int grid = grid_for(static_cast<int64_t>(v_end) - v_begin, 256, sm_count() * 8);
        if (batch)
            count_mark_kernel<true><<<grid, 256, 0, s>>>(P, colors_sel, v_begin, v_end, bitmap, gmax, out);
        else
            count_mark_kernel<false><<<grid, 256, 0, s>>>(P, colors_sel, v_begin, v_end, bitmap, gmax, out);
    }
    if (g_end > g_begin) {
        const int pgrid = grid_for(static_cast<int64_t>(g_end - g_begin) * 32, 256, sm_count() * 8);
        if (batch)
            count_pop_kernel<true><<<pgrid, 256, 0, s>>>(P, g_begin, g_end, bitmap, gmax, gcount);
        else
            count_pop_kernel<false><<<pgrid, 256, 0, s>>>(P, g_begin, g_end, bitmap, gmax, gcount);
    }
    return cudaGetLastError();
}

cudaError_t launch_det_round_block(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed,
                                  const int32_t *cur, const int32_t *work, int32_t nwork, int32_t *next, int32_t *lost,
                                  int32_t *err, cudaStream_t s) {
    if (nwork <= 0) return cudaSuccess;
    const int grid = grid_for(static_cast<int64_t>(nwork) * 32, 256, sm_count() * 16);
    det_round_block_kernel<<<grid, 256, 0, s>>>(n, rowptr, colidx, seed, cur, work, nwork, next, lost, err);
    return cudaGetLastError();
}

cudaError_t launch_validate(int32_t n, const int32_t *rowptr, const int32_t *colidx, int flags, int32_t *err,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = grid_for(static_cast<int64_t>(n) * 32, 256, sm_count() * 16);
    validate_kernel<<<grid, 256, 0, s>>>(n, rowptr, colidx, flags, err);
    return cudaGetLastError();
}

}  // namespace gc
