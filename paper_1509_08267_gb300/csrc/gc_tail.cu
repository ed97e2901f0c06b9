// Tail phase of the deterministic mode (sm_103a).
//
// On power-law graphs the last rounds of Algorithm 1 (Section 3.1) hold few vertices that conflict
// with one another round after round (on R-MAT scale 22, ~4,000 vertices after round 120 and still
// ~230 rounds to go, most of them with a few hundred vertices).  The core phase spends each of those
// rounds on a chain of dependent L2 round trips and a grid barrier (~10-20 us a round).  Once the
// core's worklist has at most tail_max vertices, this phase runs the remaining rounds on one
// thread-block cluster, whose blocks synchronise with the cluster barrier and exchange colors
// through distributed shared memory.
//
// The worklist W (k <= kTailOwned * cluster blocks vertices) is numbered 0..k-1 in key order, so
// that "u has a smaller key than v" is "tail id of u < tail id of v" for the conflict test of the
// rule (a worklist vertex loses iff a neighbour with the same color in C_r has a smaller key).
// Every block keeps the colors of all k vertices, double-buffered like C_r / C_{r+1}, with a FINAL
// bit; block b owns the vertices t with t % blocks == b: for each it keeps its row as a bitmap over
// the tail ids of its worklist neighbours, and a window of the colors 0..511 of its final
// neighbours (the core's, plus those dropped here).  A round: one warp per owned worklist vertex
// reads its row's colors from shared memory into lane-private windows (a late round's colors crowd
// into a few words, where the shared atomics of 32 lanes would queue; a neighbour found FINAL has
// its color folded into the final window and its bit cleared), takes the least free color if it
// lost, and stores its C_{r+1} into every block's copy (a winner is FINAL in both copies); then one
// cluster barrier.  A FINAL bit
// may be seen in the round that sets it: the color is the same in C_r and C_{r+1}, and the conflict
// test reads every row bit regardless of it.  A color past the 512-color window falls back to a
// full-row rescan (core_mex_from), for which the exact colors stay in the core's cex buffers.
#include <cstdio>
#include <cstdlib>

#include "gc_device.cuh"

namespace gc {
namespace {

constexpr int kTailThreads = 512;
constexpr int kTailWarps = kTailThreads / 32;
constexpr uint32_t kTailFinal = 0x80000000u;  // color word: FINAL

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_blocks() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Cluster barrier: release the block's shared and global writes, acquire everyone else's.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The address of the same shared variable in block `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void *p, unsigned rank) {
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_st(uint32_t a, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ void cluster_add(uint32_t a, uint32_t v) {
    asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

#ifdef GC_TAIL_PROFILE
// Profiling builds only: block 0's timeline.  Build: g_tail_build[0..7] (start, worklist, keys,
// sort, ids, rows, synced).  Per round (words 16 r ..): start, last warp done, block done, counts
// sent, cluster barrier passed, owned worklist vertices, bits read, most bits read by one warp, then
// the warps' summed clock cycles in the row scan, the window merge and the stores.
__device__ unsigned long long g_tail_build[8];
__device__ unsigned long long g_tail_prof[16 * 4096];
#define TAIL_BUILD(k) \
    if (rank == 0 && threadIdx.x == 0) g_tail_build[k] = global_ns()
#define TAIL_PROF(k, v) \
    if (rank == 0 && pass - R1 < 4096) g_tail_prof[16 * (pass - R1) + (k)] = (v)
// clock cycles since the last mark (pc0) into `acc`
#define TAIL_CLK(acc)                                \
    {                                                \
        const unsigned long long c1 = clock64();     \
        acc += c1 - pc0;                             \
        pc0 = c1;                                    \
    }
#else
#define TAIL_BUILD(k)
#define TAIL_PROF(k, v)
#define TAIL_CLK(acc)
#endif

// Dynamic shared memory of one block for kt = kTailOwned * blocks tail ids: colors [2][kt], rows
// [kTailOwned][kt / 32], final windows [kTailOwned][kAccWords], then per owned vertex its core id,
// global id, degree and graph, and the owned worklist lists [3][kTailOwned].  The key sort's scratch
// (kt keys of 16 bytes and kt ids) lies over the rows, which are built after it.
size_t tail_smem_bytes(int32_t kt) {
    return 8 * static_cast<size_t>(kt) + 32 * static_cast<size_t>(kt) + 4 * kTailOwned * kAccWords +
           16 * kTailOwned + 2 * 3 * kTailOwned;
}

template <bool BATCH>
__global__ void __launch_bounds__(kTailThreads, 1) tail_kernel(RoundParams P, CoreParams Q) {
    extern __shared__ __align__(16) unsigned char t_dyn[];
    __shared__ unsigned s_win[kTailWarps][kAccWords];  // the full-row rescan's window
    __shared__ unsigned s_pw[kAccWords][kTailThreads];  // lane-private windows of colors 0..511
    __shared__ unsigned s_warp[32];
    __shared__ unsigned s_total[3], s_nlist[3], s_k, s_step;
    // every block reads the same flag: the whole cluster returns, or none of it
    if (__ldcg(Q.tail) == 0u) return;
    const unsigned rank = cluster_rank(), ncl = cluster_blocks();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int32_t kt = kTailOwned * static_cast<int32_t>(ncl);
    const int32_t wpr = kt >> 5;  // words per row
    const int R1 = static_cast<int>(__ldcg(Q.tail + 1));
    const int R0 = static_cast<int>(__ldcg(Q.m + 3));
    TAIL_BUILD(0);
    uint32_t *col = reinterpret_cast<uint32_t *>(t_dyn);
    uint32_t *rows = col + 2 * kt;
    uint32_t *fwin = rows + kTailOwned * wpr;
    int32_t *s_core = reinterpret_cast<int32_t *>(fwin + kTailOwned * kAccWords);
    int32_t *s_gid = s_core + kTailOwned;
    uint32_t *s_deg = reinterpret_cast<uint32_t *>(s_gid + kTailOwned);
    int32_t *s_g = reinterpret_cast<int32_t *>(s_deg + kTailOwned);
    uint16_t *s_list = reinterpret_cast<uint16_t *>(s_g + kTailOwned);
    uint64_t *key1 = reinterpret_cast<uint64_t *>(rows);
    uint64_t *key2 = key1 + kt;
    int32_t *kid = reinterpret_cast<int32_t *>(key2 + kt);

    // W_R1: the losers in the change log of round R1 - 1, in log order (the same in every block)
    const uint4 cc = ldcg4(Q.cnt + 4 * (R1 % 3));
    const uint2 *log = Q.log + static_cast<size_t>(R1 & 1) * Q.max_v;
    if (threadIdx.x == 0) s_k = 0;
    __syncthreads();
    for (unsigned base = 0; base < cc.x; base += kTailThreads) {
        const unsigned i = base + threadIdx.x;
        uint2 x = make_uint2(0u, 0u);
        bool lose = false;
        if (i < cc.x) {
            x = __ldcg(log + i);
            lose = (x.y >> 8) == 0u;
        }
        const unsigned bal = __ballot_sync(kFull, lose);
        if (lane == 0) s_warp[wib] = static_cast<unsigned>(__popc(bal));
        __syncthreads();
        if (wib == 0) {
            const unsigned c = lane < kTailWarps ? s_warp[lane] : 0u;
            unsigned incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane < kTailWarps) s_warp[lane] = incl - c;
            if (lane == 31) s_step = incl;
        }
        __syncthreads();
        if (lose) {
            const unsigned pos = s_k + s_warp[wib] + static_cast<unsigned>(__popc(bal & lanemask_lt()));
            if (pos < static_cast<unsigned>(kt)) kid[pos] = static_cast<int32_t>(x.x);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_k += s_step;
        __syncthreads();
    }
    const int32_t k = static_cast<int32_t>(s_k);
    TAIL_BUILD(1);
    if (k > kt || k != static_cast<int32_t>(cc.y)) {
        // the hand-over only happens with at most tail_max <= kt vertices: a broken invariant
        if (rank == 0 && threadIdx.x == 0) set_error(P.err, GC_ERR_CUDA, R1, k);
        return;
    }

    // keys (priority bits, hash, local id), sorted ascending: the tail ids
    const bool hash_key = P.priority == GC_PRIORITY_HASH;
    const uint64_t *prio_src = (R0 & 1) ? P.col1 : P.col0;  // the state words round R0 did not read
    int32_t p2 = 1;
    while (p2 < k) p2 <<= 1;
    for (int32_t j = threadIdx.x; j < p2; j += kTailThreads) {
        if (j < k) {
            const int32_t V = static_cast<int32_t>(__ldcg(core_rec(Q, kid[j]) + kCoreGid));
            const Row r = load_row<BATCH>(P, V);
            const uint64_t h = vertex_hash(seed_of(P, V), static_cast<uint32_t>(r.lv));
            const uint32_t p31 = hash_key ? static_cast<uint32_t>(h >> 33) : prio_of(__ldcg(prio_src + V));
            key1[j] = static_cast<uint64_t>(p31) << 32 | (h >> 32);
            key2[j] = (h << 32) | static_cast<uint32_t>(r.lv);
        } else {
            key1[j] = ~0ull;
            key2[j] = ~0ull;
            kid[j] = -1;
        }
    }
    __syncthreads();
    TAIL_BUILD(2);
    // bitonic sort of p2 entries (ties of key1 and key2, between graphs of a batch, by core id)
    for (int32_t size = 2; size <= p2; size <<= 1) {
        for (int32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (int32_t i = threadIdx.x; i < (p2 >> 1); i += kTailThreads) {
                const int32_t a = 2 * stride * (i / stride) + (i & (stride - 1)), b = a + stride;
                const uint64_t a1 = key1[a], b1 = key1[b], a2 = key2[a], b2 = key2[b];
                const bool gt = a1 != b1 ? a1 > b1
                                         : (a2 != b2 ? a2 > b2
                                                     : static_cast<uint32_t>(kid[a]) > static_cast<uint32_t>(kid[b]));
                if (gt == ((a & size) == 0)) {
                    key1[a] = b1;
                    key1[b] = a1;
                    key2[a] = b2;
                    key2[b] = a2;
                    const int32_t t = kid[a];
                    kid[a] = kid[b];
                    kid[b] = t;
                }
            }
            __syncthreads();
        }
    }

    TAIL_BUILD(3);
    // tail ids into the core records (every block writes the same values, then reads its own), the
    // colors C_R1, and the owned vertices
    const int32_t *cex_r1 = Q.cex + static_cast<size_t>(R1 & 1) * Q.max_v;
    const int32_t nown = k > static_cast<int32_t>(rank) ? (k - 1 - static_cast<int32_t>(rank)) / static_cast<int32_t>(ncl) + 1 : 0;
    for (int32_t t = threadIdx.x; t < k; t += kTailThreads) {
        const int32_t core = kid[t];
        __stcg(core_rec(Q, core) + kCoreTail, static_cast<unsigned>(t));
        const uint32_t c = static_cast<uint32_t>(__ldcg(cex_r1 + core));
        col[t] = c;
        col[kt + t] = c;
        if (static_cast<unsigned>(t) % ncl == rank) s_core[t / static_cast<int32_t>(ncl)] = core;
    }
    __syncthreads();
    for (int32_t o = threadIdx.x; o < nown; o += kTailThreads) {
        const unsigned *rec = core_rec(Q, s_core[o]);
        s_gid[o] = static_cast<int32_t>(__ldcg(rec + kCoreGid));
        s_deg[o] = __ldcg(rec + kCoreDeg);
        s_g[o] = static_cast<int32_t>(__ldcg(rec + kCoreG));
        s_list[(R1 % 3) * kTailOwned + o] = static_cast<uint16_t>(o);
    }
    for (int32_t i = threadIdx.x; i < nown * kAccWords; i += kTailThreads)
        fwin[i] = __ldcg(core_rec(Q, s_core[i / kAccWords]) + kAccFin + (i % kAccWords));
    for (int32_t i = threadIdx.x; i < nown * wpr; i += kTailThreads) rows[i] = 0u;
    if (threadIdx.x < 3) {
        s_total[threadIdx.x] = 0u;
        s_nlist[threadIdx.x] = threadIdx.x == static_cast<unsigned>(R1 % 3) ? static_cast<unsigned>(nown) : 0u;
    }
    __syncthreads();
    TAIL_BUILD(4);
    // rows: the entries of each owned vertex's core pieces; a FINAL neighbour's color into the final
    // window, a worklist neighbour's tail id into the row (a warp per vertex, 8 entries per lane in
    // flight)
    for (int32_t o = wib; o < nown; o += kTailWarps) {
        const unsigned *rec = core_rec(Q, s_core[o]);
        const unsigned pb = __ldcg(rec + kCorePcBeg), pe = __ldcg(rec + kCorePcEnd);
        uint32_t *row = rows + o * wpr;
        uint32_t *fw = fwin + o * kAccWords;
        for (unsigned pc = pb; pc < pe; ++pc) {
            const int4 pz = __ldcg(Q.pieces + pc);  // {vertex, pool offset, entries, flags}
            for (int32_t j0 = 0; j0 < pz.z; j0 += 8 * 32) {
                uint32_t u[8], fb[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int32_t j = j0 + lane + 32 * q;
                    u[q] = j < pz.z ? static_cast<uint32_t>(__ldcg(Q.pool + pz.y + j)) & ~kCoreSmaller : ~0u;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) fb[q] = u[q] != ~0u ? (__ldcg(Q.fbits + (u[q] >> 5)) >> (u[q] & 31)) & 1u : 0u;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (u[q] == ~0u) continue;
                    if (fb[q]) {
                        const int32_t c = __ldcg(cex_r1 + u[q]);
                        if (static_cast<unsigned>(c) < 32u * kAccWords) atomicOr(fw + (c >> 5), 1u << (c & 31));
                    } else {
                        const unsigned tu = __ldcg(core_rec(Q, u[q]) + kCoreTail);
                        atomicOr(row + (tu >> 5), 1u << (tu & 31));
                    }
                }
            }
        }
    }
    __syncthreads();
    TAIL_BUILD(5);
    cluster_sync();  // every block built before any block writes into another's colors
    TAIL_BUILD(6);

    const uint64_t *col_r0 = (R0 & 1) ? P.col0 : P.col1;  // the state words round R0 read
    const int32_t wk = ((k + 1023) >> 10) << 5;  // the row words that can hold bits: a multiple of 32
    unsigned *win = s_win[wib];
    unsigned *pw = &s_pw[0][threadIdx.x];  // word w of this lane's window: pw[w * kTailThreads]
#pragma unroll
    for (int w = 0; w < kAccWords; ++w) pw[w * kTailThreads] = 0u;
    int pass = R1;
    for (;;) {
        if (pass >= P.pass_end) {
            if (P.cap_is_error && rank == 0 && threadIdx.x == 0) set_error(P.err, GC_ERR_NO_CONVERGENCE, pass, 0);
            break;
        }
        const unsigned cur = static_cast<unsigned>(pass) & 1u, lc = static_cast<unsigned>(pass) % 3u,
                       ln = static_cast<unsigned>(pass + 1) % 3u;
        uint32_t *col_cur = col + cur * kt, *col_nxt = col + (cur ^ 1u) * kt;
        const int32_t *cex_cur = Q.cex + static_cast<size_t>(cur) * Q.max_v;
        int32_t *cex_nxt = Q.cex + static_cast<size_t>(cur ^ 1u) * Q.max_v;
        const unsigned nv = s_nlist[lc];
        // the list the next round appends to was read two rounds ago
        if (threadIdx.x == 0) s_nlist[(pass + 2) % 3] = 0u;
        unsigned st_deg = 0, st_cnt = 0, st_read = 0;
        if (threadIdx.x == 0) {
            TAIL_PROF(0, global_ns());
            TAIL_PROF(5, nv);
        }
#ifdef GC_TAIL_PROFILE
        unsigned long long pc_scan = 0, pc_merge = 0, pc_store = 0, pc0 = 0;
#endif
        for (unsigned idx = wib; idx < nv; idx += kTailWarps) {
#ifdef GC_TAIL_PROFILE
            pc0 = clock64();
#endif
            const int32_t o = s_list[lc * kTailOwned + idx];
            const int32_t t = o * static_cast<int32_t>(ncl) + static_cast<int32_t>(rank);
            const uint32_t cv = col_cur[t] & ~kTailFinal;
            uint32_t *row = rows + o * wpr;
            uint32_t *fw = fwin + o * kAccWords;
            unsigned conflict = 0, reads = 0;
            // a word of the row per lane, its bits four at a time in steps the whole warp takes
            // together (a loop whose trip count differs per lane lets the lanes drift apart); lane l
            // starts at bit l of its word, so the lanes' color reads fall in different banks; the
            // window words are the lane's own, updated without atomics (shared atomics of all lanes
            // run at about one a cycle per SM)
            for (int32_t i = lane; i < wk; i += 32) {
                const uint32_t x = row[i];
                uint32_t y = __funnelshift_r(x, x, lane), drop = 0;
                while (__any_sync(kFull, y != 0u)) {
                    int32_t tu[4];
                    uint32_t w[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        tu[q] = -1;
                        if (y != 0u) {
                            tu[q] = 32 * i + ((__ffs(static_cast<int>(y)) - 1 + lane) & 31);
                            y &= y - 1u;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) w[q] = tu[q] >= 0 ? col_cur[tu[q]] : 0u;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (tu[q] < 0) continue;
                        const uint32_t c = w[q] & ~kTailFinal;
                        conflict |= static_cast<unsigned>(c == cv && tu[q] < t);
                        if (c < 32u * kAccWords) {
                            pw[(c >> 5) * kTailThreads] |= 1u << (c & 31);
                            if (w[q] & kTailFinal) atomicOr(fw + (c >> 5), 1u << (c & 31));
                        }
                        if (w[q] & kTailFinal) drop |= 1u << (tu[q] & 31);
                        ++reads;
                    }
                }
                if (drop) row[i] = x & ~drop;
            }
            TAIL_CLK(pc_scan);
            // the warp's window: word w is the OR of the lanes' words w (and the lanes' are cleared)
            unsigned wsum = 0;
#pragma unroll
            for (int w = 0; w < kAccWords; ++w) {
                const unsigned x = __reduce_or_sync(kFull, pw[w * kTailThreads]);
                pw[w * kTailThreads] = 0u;
                if (lane == w) wsum = x;
            }
            __syncwarp();
            const bool lose = __any_sync(kFull, conflict != 0u);
            int32_t nc = static_cast<int32_t>(cv);
            if (lose) {
                const unsigned ww = lane < kAccWords ? (wsum | fw[lane]) : ~0u;
                const unsigned fm = __ballot_sync(kFull, ~ww != 0u);
                if (fm) {
                    const int l = __ffs(static_cast<int>(fm)) - 1;
                    nc = 32 * l + __ffs(static_cast<int>(~__shfl_sync(kFull, ww, l))) - 1;
                } else {
                    nc = core_mex_from<BATCH>(P, col_r0, s_gid[o], cex_cur, win, lane, 32 * kAccWords);
                }
            }
            TAIL_CLK(pc_merge);
            // C_{r+1} into every block's copy; a winner is FINAL in both copies
            if (static_cast<unsigned>(lane) < ncl) {
                cluster_st(cluster_addr(col_nxt + t, static_cast<unsigned>(lane)),
                           lose ? static_cast<uint32_t>(nc) : (cv | kTailFinal));
                if (!lose) cluster_st(cluster_addr(col_cur + t, static_cast<unsigned>(lane)), cv | kTailFinal);
            }
            if (lane == 0) {
                cex_nxt[s_core[o]] = nc;  // exact colors: the full-row rescan and the write-back read them
                if (lose) {
                    const unsigned pos = atomicAdd(&s_nlist[ln], 1u);
                    s_list[ln * kTailOwned + pos] = static_cast<uint16_t>(o);
                    if constexpr (BATCH) note_graph_round(P, s_g[o], pass + 1);
                }
                st_cnt += 1;
                st_deg += s_deg[o];
            }
            st_read += reads;
            __syncwarp();
            TAIL_CLK(pc_store);
        }
#ifdef GC_TAIL_PROFILE
        {
            const unsigned wr = __reduce_add_sync(kFull, st_read);
            if (rank == 0 && lane == 0 && pass - R1 < 4096) {
                atomicMax(g_tail_prof + 16 * (pass - R1) + 1, static_cast<unsigned long long>(global_ns()));
                atomicAdd(g_tail_prof + 16 * (pass - R1) + 6, static_cast<unsigned long long>(wr));
                atomicMax(g_tail_prof + 16 * (pass - R1) + 7, static_cast<unsigned long long>(wr));
                atomicAdd(g_tail_prof + 16 * (pass - R1) + 8, pc_scan);
                atomicAdd(g_tail_prof + 16 * (pass - R1) + 9, pc_merge);
                atomicAdd(g_tail_prof + 16 * (pass - R1) + 10, pc_store);
            }
        }
#endif
        __syncthreads();
        if (threadIdx.x == 0) TAIL_PROF(2, global_ns());
        // this block's losers into every block's count of the round's losers (a thread per block)
        if (threadIdx.x < ncl) cluster_add(cluster_addr(&s_total[ln], threadIdx.x), s_nlist[ln]);
        if (threadIdx.x == 0) {
            s_total[(pass + 2) % 3] = 0u;  // counted into next round; last read two rounds ago
            TAIL_PROF(3, global_ns());
        }
        if (P.stats) flush_stats(P, pass, st_deg, st_cnt, st_read);
        cluster_sync();
        if (threadIdx.x == 0) TAIL_PROF(4, global_ns());
        const unsigned total = *reinterpret_cast<volatile unsigned *>(&s_total[ln]);
        ++pass;
        if (total == 0u) break;
    }
    if (rank == 0 && threadIdx.x == 0) {
        P.passes[0] = pass;
        P.passes[1] = pass - 1;
    }
}

template <bool BATCH>
cudaError_t tail_config(int32_t ncl, cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at) {
    const void *fn = reinterpret_cast<const void *>(&tail_kernel<BATCH>);
    const size_t smem = tail_smem_bytes(kTailOwned * ncl);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess && ncl > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(static_cast<unsigned>(ncl));
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = smem;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = static_cast<unsigned>(ncl);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return e;
}

}  // namespace

int32_t tail_cluster_size() {
    for (int32_t ncl : {16, 8}) {
        bool ok = true;
        for (int b = 0; b < 2 && ok; ++b) {
            cudaLaunchConfig_t cfg;
            cudaLaunchAttribute at[1];
            int n = 0;
            if (b == 0) {
                ok = tail_config<false>(ncl, cfg, at) == cudaSuccess &&
                     cudaOccupancyMaxActiveClusters(&n, tail_kernel<false>, &cfg) == cudaSuccess && n >= 1;
            } else {
                ok = tail_config<true>(ncl, cfg, at) == cudaSuccess &&
                     cudaOccupancyMaxActiveClusters(&n, tail_kernel<true>, &cfg) == cudaSuccess && n >= 1;
            }
        }
        if (ok) return ncl;
        cudaGetLastError();
    }
    return 0;
}

cudaError_t launch_tail(const RoundParams &P, const CoreParams &Q, bool batch, cudaStream_t s) {
    if (Q.tail_max <= 0 || Q.tail_nc <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    cudaError_t e = batch ? tail_config<true>(Q.tail_nc, cfg, at) : tail_config<false>(Q.tail_nc, cfg, at);
    if (e != cudaSuccess) return e;
    cfg.stream = s;
#ifdef GC_TAIL_PROFILE
    static unsigned long long h_prof[16 * 4096], h_build[8];
    for (auto &x : h_prof) x = 0;
    cudaMemcpyToSymbolAsync(g_tail_prof, h_prof, sizeof h_prof, 0, cudaMemcpyHostToDevice, s);
#endif
    e = batch ? cudaLaunchKernelEx(&cfg, tail_kernel<true>, P, Q) : cudaLaunchKernelEx(&cfg, tail_kernel<false>, P, Q);
#ifdef GC_TAIL_PROFILE
    cudaMemcpyFromSymbolAsync(h_prof, g_tail_prof, sizeof h_prof, 0, cudaMemcpyDeviceToHost, s);
    cudaMemcpyFromSymbolAsync(h_build, g_tail_build, sizeof h_build, 0, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (const char *path = getenv("GC_TAIL_PROFILE_OUT")) {
        if (FILE *f = fopen(path, "w")) {
            for (int k = 0; k < 8; ++k) fprintf(f, "%llu ", h_build[k]);
            fprintf(f, "\n");
            for (int r = 0; r < 4096 && h_prof[16 * r] != 0; ++r) {
                for (int k = 0; k < 16; ++k) fprintf(f, "%llu ", h_prof[16 * r + k]);
                fprintf(f, "\n");
            }
            fclose(f);
        }
    }
#endif
    return e;
}

}  // namespace gc
