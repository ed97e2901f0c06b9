// C ABI of the coloring library: argument checks, per-device context with cached scratch, host
// array staging, and the launch sequence setup -> expand -> persistent round kernel -> counting.
// Declarations and the contract of every entry point are in include/gc.h.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gc_internal.h"

namespace gc {

// ------------------------------------------------------------------------------------------
// errors

static thread_local std::string t_error;

int set_last_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_error = buf;
    return code;
}

static int cuda_fail(cudaError_t e, const char *what) {
    return set_last_error(GC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GC_CUDA(call)                                                    \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);              \
    } while (0)

// ------------------------------------------------------------------------------------------
// device buffers and context

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes == 0) bytes = 16;
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        const size_t want = bytes + bytes / 8;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return e;
        }
        cap = want;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T>
    T *as() const {
        return static_cast<T *>(p);
    }
};

// Control block: one device allocation, fetched with one copy at the end of a run.
struct Ctl {
    int32_t err[4];
    int32_t passes[2];  // first round not executed, last round executed
    int32_t pad0[2];
    unsigned cnt[3 * kCnt];
    unsigned tmp[2];
    unsigned long long list_total, list_alloc;
    int32_t gmax1, gcount1, glast1, pad1;
    int32_t pad2[2];
    unsigned peel[4];  // smallest-last peeling: the two threshold words, the work items needed
    unsigned long long ecnt[3];  // list entries of each counter set's worklist (core hand-over)
    unsigned long long core_bump;
    int32_t core_go, pad3;
    alignas(16) unsigned core_cnt[12];  // three sets of four, each read with one 16-byte load
    unsigned core_m[4];
    unsigned tail_ctl[4];  // tail phase: handed over, first round
    GridBar bar;
};
static_assert(offsetof(Ctl, bar) % 128 == 0, "barrier alignment");
static_assert(offsetof(Ctl, core_cnt) % 16 == 0, "core counter alignment");

struct Context {
    int device = -1;
    std::mutex mu;
    cudaStream_t stream = nullptr;
    int sms = 0;
    int occ[2][2][2][2] = {};  // [wide][mode][batch][compact] blocks per SM of the round kernel
    int occ_part = 0;       // blocks per SM of the partition-mode round kernel
    int occ_ord[2] = {};    // blocks per SM of the ordered-mode round kernel [batch]
    int occ_peel = 0;       // blocks per SM of the peeling kernel
    Buf col0, col1, small0, small1, items, chunk0, chunk1, acc, lists, ctl, stats, bitmap, vg, hist;
    Buf gmax, gcount, glast, g_vbase, g_n, g_ebase, g_rbase, g_m;
    Buf st_rowptr, st_colidx, st_vtx, st_edge, st_colors, st_colors_in, mid0, mid1, rank;
    Buf core_rec, core_cex, core_c8, core_fbits, core_items, core_active, core_log, core_pool;
    Buf st_cur, st_work, st_next, st_lost;  // gc_det_round staging
    int32_t core_max_v = 0;  // largest core the round kernel's shared memory holds (-1: none)
    int32_t tail_nc = 0;     // blocks of the tail phase's cluster (-1: no cluster launch possible)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // host adjacency arrays are uploaded on copy_stream while the set-up runs on the call's stream;
    // ev_before orders the upload after earlier work, ev_colidx marks it done
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_before = nullptr, ev_colidx = nullptr;
    void release_all() {
        Buf *all[] = {&col0, &col1, &small0, &small1, &items, &chunk0, &chunk1, &acc, &lists, &ctl, &stats, &bitmap, &hist,
                      &vg, &gmax, &gcount, &glast, &g_vbase, &g_n, &g_ebase, &g_rbase, &g_m, &st_rowptr, &st_colidx, &st_vtx, &st_edge, &st_colors, &st_colors_in, &mid0, &mid1, &rank,
                      &core_rec, &core_cex, &core_c8, &core_fbits, &core_items, &core_active, &core_log, &core_pool,
                      &st_cur, &st_work, &st_next, &st_lost};
        for (Buf *b : all) b->release();
    }
};

static std::mutex g_ctx_mu;
static Context *g_ctx[128];

static int get_context(Context **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        cudaGetLastError();
        return set_last_error(GC_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    if (!g_ctx[dev]) {
        Context *c = new Context();
        c->device = dev;
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
        for (auto &ev : c->ev) cudaEventCreate(&ev);
        if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_before, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_colidx, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            c->copy_stream = nullptr;  // uploads then stay on the call's stream
        }
        g_ctx[dev] = c;
    }
    *out = g_ctx[dev];
    return GC_OK;
}

// Where a caller pointer lives: 1 = device memory of the current device (or managed), 0 = host.
static int locate(const void *p, int dev, int *on_device) {
    *on_device = 0;
    if (!p) return GC_OK;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GC_OK;
    }
    if (a.type == cudaMemoryTypeDevice) {
        if (a.device != dev)
            return set_last_error(GC_ERR_INVALID_ARG, "pointer %p is memory of device %d, current device is %d", p,
                                  a.device, dev);
        *on_device = 1;
    } else if (a.type == cudaMemoryTypeManaged) {
        *on_device = 1;
    }
    return GC_OK;
}

// Device view of a caller array: the array itself, or a staged copy of a host array.
static int device_view(const void *p, size_t bytes, int dev, Buf &stage, cudaStream_t s, const void **out) {
    int on_dev = 0;
    int st = locate(p, dev, &on_dev);
    if (st != GC_OK) return st;
    if (on_dev || bytes == 0) {
        *out = p;
        return GC_OK;
    }
    cudaError_t e = stage.ensure(bytes);
    if (e != cudaSuccess) return set_last_error(GC_ERR_OOM, "staging %zu bytes: %s", bytes, cudaGetErrorString(e));
    GC_CUDA(cudaMemcpyAsync(stage.p, p, bytes, cudaMemcpyHostToDevice, s));
    *out = stage.p;
    return GC_OK;
}


static int ensure(Buf &b, size_t bytes, const char *what) {
    cudaError_t e = b.ensure(bytes);
    if (e != cudaSuccess)
        return set_last_error(GC_ERR_OOM, "allocating %zu bytes for %s: %s", bytes, what, cudaGetErrorString(e));
    return GC_OK;
}

#define GC_TRY(call)                  \
    do {                              \
        int st_ = (call);             \
        if (st_ != GC_OK) return st_; \
    } while (0)

static int error_from_ctl(const Ctl &c) {
    const int64_t where = (static_cast<int64_t>(static_cast<uint32_t>(c.err[3])) << 32) | static_cast<uint32_t>(c.err[2]);
    switch (c.err[0]) {
        case GC_ERR_INVALID_GRAPH:
            if (c.err[1] < 0)
                return set_last_error(GC_ERR_INVALID_GRAPH, "invalid offset tables at graph %d", -1 - c.err[1]);
            return set_last_error(GC_ERR_INVALID_GRAPH,
                                  "invalid graph at vertex %d (row offset or adjacency entry %lld): row offsets must "
                                  "be non-decreasing from 0 to nnz, neighbours in [0, n) and no self-loops",
                                  c.err[1], static_cast<long long>(where));
        case GC_ERR_NO_CONVERGENCE:
            return set_last_error(GC_ERR_NO_CONVERGENCE, "worklist not empty after %d rounds", c.err[1] - 1);
        case GC_ERR_TIMEOUT:
            return set_last_error(GC_ERR_TIMEOUT, "grid barrier wait exceeded its limit (block %d)", c.err[1]);
        default:
            return set_last_error(c.err[0], "device error %d", c.err[0]);
    }
}

// ------------------------------------------------------------------------------------------
// the coloring run (single graph = batch of one)

struct Problem {
    bool batch;
    int32_t G;
    int32_t n;    // total vertices
    int64_t nnz;  // total entries
    const int32_t *rowptr;
    const int32_t *colidx;
    const int64_t *vtx_off;
    const int64_t *edge_off;
    cudaEvent_t colidx_ready = nullptr;  // recorded when a host colidx upload is done (else none)
    const int32_t *prio_rank = nullptr;  // recoloring pass: the given coloring (device view)
    int32_t priority_override = -1;        // >= 0: the priority to use instead of the options'
};

// Waits, when the call returns on any path, for an upload still running on the copy stream (the
// caller may free its host arrays as soon as the call returns).
struct UploadGuard {
    cudaStream_t s;
    ~UploadGuard() {
        if (s) cudaStreamSynchronize(s);
    }
};

// The call's stream waits for the adjacency upload before the first kernel that reads colidx.
static int wait_colidx(const Problem &pb, cudaStream_t s) {
    if (pb.colidx_ready) GC_CUDA(cudaStreamWaitEvent(s, pb.colidx_ready, 0));
    return GC_OK;
}

struct Outputs {
    int32_t *colors;   // caller array (device or host), total n
    int32_t *ncolors;  // single: host scalar; batch: caller array of G
    int32_t *rounds;
};

// Smallest-last levels of a single graph into C.rank (int32[n]): the peeling kernel with the
// ordered mode's lists; the residual degrees live in C.col1, which every mode rewrites afterwards.
// P holds the graph, the control block and the barrier; the counter sets must be zero.
// An NVTX range over a host-side phase of a call (visible in Nsight Systems; free when no tool is
// attached).  The device work of a phase runs asynchronously, so a range covers its launches and
// the host waits inside it, not the kernels' own time.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

static int peel_levels(Context &C, Ctl *ctl, RoundParams P, int32_t T1, int32_t CH, cudaStream_t s,
                       int32_t *nlevels, int32_t *degeneracy, int32_t blocks_per_sm) {
    NvtxRange range("gc: smallest-last peeling");
    const size_t n = static_cast<size_t>(P.n);
    GC_TRY(ensure(C.rank, 4 * n, "smallest-last levels"));
    GC_TRY(ensure(C.col0, 8 * n, "vertex state"));
    GC_TRY(ensure(C.col1, 8 * n, "vertex state"));
    GC_TRY(ensure(C.items, 4 * n, "worklist"));
    GC_TRY(ensure(C.small0, 4 * n, "worklist"));
    GC_TRY(ensure(C.small1, 4 * n, "worklist"));
    GC_TRY(ensure(C.mid0, 4 * n, "worklist"));
    GC_TRY(ensure(C.mid1, 4 * n, "worklist"));
    P.T1 = T1 < kOrdSmall ? T1 : kOrdSmall;
    P.CH = CH < kOrdChunk ? CH : kOrdChunk;
    P.pass_begin = 1;
    int32_t *res = reinterpret_cast<int32_t *>(C.col1.p);
    int32_t *level = C.rank.as<int32_t>();
    GC_CUDA(cudaMemsetAsync(ctl->peel, 0, sizeof(ctl->peel), s));
    GC_CUDA(launch_peel_init(P, res, level, ctl->peel, ctl->peel + 2, s));
    Ctl h{};
    GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    if (h.err[0] != 0) return error_from_ctl(h);
    const size_t n_items = h.peel[2];
    GC_TRY(ensure(C.chunk0, 16 * std::max<size_t>(n_items, 1), "work items"));
    GC_TRY(ensure(C.chunk1, 16 * std::max<size_t>(n_items, 1), "work items"));
    P.small0 = C.small0.as<int32_t>();
    P.small1 = C.small1.as<int32_t>();
    P.mid0 = C.mid0.as<int32_t>();
    P.mid1 = C.mid1.as<int32_t>();
    P.chunk0 = C.chunk0.as<int4>();
    P.chunk1 = C.chunk1.as<int4>();
    GC_CUDA(cudaMemsetAsync(ctl->cnt, 0, sizeof(ctl->cnt), s));
    int &occ = C.occ_peel;
    if (occ == 0) GC_CUDA(peel_kernel_occupancy(256, &occ));
    const int grid = (blocks_per_sm > 0 && blocks_per_sm < occ ? blocks_per_sm : occ) * C.sms;
    // the lists of vertices left by each threshold search: two scratch arrays that every mode
    // rewrites afterwards
    GC_CUDA(launch_peel(P, res, level, ctl->peel, C.items.as<int32_t>(), C.col0.as<int32_t>(), ctl->peel + 2, grid,
                        256, s));
    GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    if (h.err[0] != 0) return error_from_ctl(h);
    if (nlevels) *nlevels = h.passes[0];
    if (degeneracy) *degeneracy = h.passes[1];
    return GC_OK;
}

static int run(Context &C, const Problem &pb, int mode, uint64_t seed, const gc_options *opt, gc_stats *stats,
               const Outputs &out) {
    NvtxRange range(pb.batch ? "gc: batch coloring" : "gc: coloring");
    const int dev = C.device;
    cudaStream_t s = (opt && opt->stream) ? static_cast<cudaStream_t>(opt->stream) : C.stream;
    const uint32_t flags = opt ? opt->flags : 0u;
    const int32_t T1 = (opt && opt->small_max_degree) ? opt->small_max_degree : 127;
    const int32_t CH = (opt && opt->chunk) ? opt->chunk : 1024;
    const int32_t block = (opt && opt->block_size) ? opt->block_size : 256;
    if (T1 < 1 || T1 > 127) return set_last_error(GC_ERR_INVALID_ARG, "small_max_degree %d outside 1..127", T1);
    if (CH < 32 || CH > 8192 || CH % 32) return set_last_error(GC_ERR_INVALID_ARG, "chunk %d invalid", CH);
    if (block != 256) return set_last_error(GC_ERR_INVALID_ARG, "block_size %d unsupported (256)", block);
    const int32_t opt_priority = opt ? opt->priority : GC_PRIORITY_HASH;
    if (opt_priority != GC_PRIORITY_HASH && opt_priority != GC_PRIORITY_LARGEST_FIRST &&
        opt_priority != GC_PRIORITY_SMALLEST_LAST)
        return set_last_error(GC_ERR_INVALID_ARG, "unknown priority %d", opt_priority);
    if (opt_priority == GC_PRIORITY_SMALLEST_LAST && pb.priority_override < 0 && pb.batch)
        return set_last_error(GC_ERR_INVALID_ARG, "GC_PRIORITY_SMALLEST_LAST colors single graphs only");
    const int32_t priority = pb.priority_override >= 0 ? pb.priority_override : opt_priority;
    const int64_t n = pb.n;
    const int32_t G = pb.G;
    const int32_t max_rounds =
        (opt && opt->max_rounds > 0) ? opt->max_rounds : static_cast<int32_t>(n < INT32_MAX ? n + 1 : INT32_MAX);
    const int64_t spin_ns = (opt && opt->spin_limit_ns > 0) ? opt->spin_limit_ns : 1000000000LL;
    const int32_t stats_cap = (flags & GC_FLAG_STATS) ? (max_rounds < 65536 ? max_rounds : 65536) : 0;
    const size_t gz = static_cast<size_t>(G);

    // scratch sized by n; work-item buffers are sized after binning
    GC_TRY(ensure(C.col0, 8 * n, "vertex state"));
    GC_TRY(ensure(C.col1, 8 * n, "vertex state"));
    GC_TRY(ensure(C.items, 4 * n, "worklist"));
    GC_TRY(ensure(C.small0, 4 * n, "worklist"));
    GC_TRY(ensure(C.small1, 4 * n, "worklist"));
    GC_TRY(ensure(C.ctl, sizeof(Ctl), "control"));
    GC_TRY(ensure(C.bitmap, 4 * (n / 32 + 2), "color bitmap"));
    const int32_t shift = sort_shift(n);
    const size_t hist_words = 2 * static_cast<size_t>(sort_bins(static_cast<int32_t>(n), shift));
    GC_TRY(ensure(C.hist, 4 * hist_words, "worklist sort"));
    if (stats_cap) GC_TRY(ensure(C.stats, 8 * (4 * static_cast<size_t>(stats_cap) + 1), "statistics"));
    // compact sweep (larger vertices sweep lists of the neighbours that can still change): the
    // default of both modes; in-place mode keeps the plain kernel when no vertex is larger than T1
    // (it then has nothing to compact, and the plain kernel keeps more registers for the thread path)
    bool compact = (mode == GC_MODE_DETERMINISTIC || mode == GC_MODE_INPLACE) && !(flags & GC_FLAG_FULL_SWEEP);
    if (pb.batch) {
        GC_TRY(ensure(C.vg, 4 * n, "graph ids"));
        GC_TRY(ensure(C.gmax, 4 * gz, "per-graph max"));
        GC_TRY(ensure(C.gcount, 4 * gz, "per-graph counts"));
        GC_TRY(ensure(C.glast, 4 * gz, "per-graph rounds"));
        GC_TRY(ensure(C.g_vbase, 8 * gz, "graph table"));
        GC_TRY(ensure(C.g_n, 4 * gz, "graph table"));
        GC_TRY(ensure(C.g_ebase, 8 * gz, "graph table"));
        GC_TRY(ensure(C.g_rbase, 8 * gz, "graph table"));
        GC_TRY(ensure(C.g_m, 8 * gz, "graph table"));
    }
    Ctl *ctl = C.ctl.as<Ctl>();
    GC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    GC_CUDA(cudaMemsetAsync(&ctl->gmax1, 0xff, sizeof(int32_t), s));
    GC_CUDA(cudaMemsetAsync(C.bitmap.p, 0, 4 * (n / 32 + 2), s));
    GC_CUDA(cudaMemsetAsync(C.hist.p, 0, 4 * hist_words / 2, s));
    if (stats_cap) GC_CUDA(cudaMemsetAsync(C.stats.p, 0, 8 * (4 * static_cast<size_t>(stats_cap) + 1), s));

    if (pb.batch) GC_CUDA(cudaMemsetAsync(C.gmax.p, 0xff, 4 * gz, s));

    RoundParams P{};
    P.n = static_cast<int32_t>(n);
    P.G = G;
    P.nnz = pb.nnz;
    P.rowptr = pb.rowptr;
    P.colidx = pb.colidx;
    if (pb.batch) {
        P.g_vbase = C.g_vbase.as<int64_t>();
        P.g_n = C.g_n.as<int32_t>();
        P.g_ebase = C.g_ebase.as<int64_t>();
        P.g_rbase = C.g_rbase.as<int64_t>();
        P.g_m = C.g_m.as<int64_t>();
        P.vg = C.vg.as<int32_t>();
    }
    P.seed = seed;
    P.col0 = C.col0.as<uint64_t>();
    P.col1 = C.col1.as<uint64_t>();
    P.small0 = C.small0.as<int32_t>();
    P.small1 = C.small1.as<int32_t>();
    P.items = C.items.as<int32_t>();
    P.tmp = ctl->tmp;
    P.list_total = compact ? &ctl->list_total : nullptr;
    P.list_alloc = compact ? &ctl->list_alloc : nullptr;
    P.deg_hist = C.hist.as<unsigned>();
    P.sort_shift = shift;
    P.cnt = ctl->cnt;
    P.bar = &ctl->bar;
    P.err = ctl->err;
    P.passes = ctl->passes;
    P.graph_last = pb.batch ? C.glast.as<int32_t>() : &ctl->glast1;
    P.stats = stats_cap ? C.stats.as<unsigned long long>() : nullptr;
    P.stats_cap = stats_cap;
    P.pass_begin = 1;
    P.pass_end = max_rounds < INT32_MAX ? max_rounds + 1 : INT32_MAX;
    P.cap_is_error = 1;
    P.spin_ns = spin_ns;
    P.T1 = T1;
    P.CH = CH;
    P.priority = priority;
    P.prio_rank = pb.prio_rank;
    // (GC_FLAG_FULL_SWEEP reads every entry of every worklist row: no early stop either)
    P.early_exit = mode == GC_MODE_DETERMINISTIC && compact ? 1 : 0;
    // the entries of each worklist's lists are counted for the core hand-over from round 1 on, when
    // the graph has more entries than the core may take (else the worklist always fits)
    const int64_t core_E = std::min<int64_t>(
        pb.nnz, opt && opt->core_entries > 0 ? std::min<int64_t>(opt->core_entries, kCoreEntries) : kCoreEntries);
    if (mode == GC_MODE_DETERMINISTIC && compact && !(opt && opt->core_vertices < 0) && pb.nnz > core_E)
        P.ecnt = ctl->ecnt;

    const bool timing = (flags & GC_FLAG_TIMING) != 0;
    Ctl h{};
    if (pb.batch) {
        GC_CUDA(launch_batch_tables(P, pb.vtx_off, pb.edge_off, C.g_vbase.as<int64_t>(), C.g_n.as<int32_t>(),
                                    C.g_ebase.as<int64_t>(), C.g_rbase.as<int64_t>(), C.g_m.as<int64_t>(), s));
        GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
        if (h.err[0] != 0) return error_from_ctl(h);
    }
    if (timing) GC_CUDA(cudaEventRecord(C.ev[0], s));
    if (priority == GC_PRIORITY_SMALLEST_LAST && mode != GC_MODE_PARTITION && n > 0) {
        GC_TRY(wait_colidx(pb, s));
        int32_t nlev = 0, degen = 0;
        GC_TRY(peel_levels(C, ctl, P, T1, CH, s, &nlev, &degen, opt ? opt->blocks_per_sm : 0));
        P.prio_rank = C.rank.as<int32_t>();
        GC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
        GC_CUDA(cudaMemsetAsync(&ctl->gmax1, 0xff, sizeof(int32_t), s));
    }
    int64_t grid = 0;
    if (mode == GC_MODE_PARTITION) {
        // Algorithm 1 with p id-ordered blocks: its own set-up and round kernel
        GC_TRY(wait_colidx(pb, s));
        GC_CUDA(launch_partition_init(P, s));
        GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
        if (h.err[0] != 0) return error_from_ctl(h);
        if (timing) GC_CUDA(cudaEventRecord(C.ev[1], s));
        int &occ = C.occ_part;
        if (occ == 0) GC_CUDA(partition_kernel_occupancy(block, &occ));
        int per_sm = occ;
        if (opt && opt->blocks_per_sm > 0 && opt->blocks_per_sm < per_sm) per_sm = opt->blocks_per_sm;
        grid = static_cast<int64_t>(per_sm) * C.sms;
        int64_t p = (opt && opt->partitions > 0) ? opt->partitions : grid * (block / 32);
        if (p > n) p = n;
        if (p < 1) p = 1;
        const int64_t want = (p + block / 32 - 1) / (block / 32);  // one warp per block of ids
        if (want < grid) grid = want;
        if (grid < 1) grid = 1;
        if (n > 0) GC_CUDA(launch_partition_rounds(P, static_cast<int32_t>(p), static_cast<int>(grid), block, s));
    } else if (mode == GC_MODE_ORDERED) {
        // First Fit in key order: in-place set-up (vertices with neighbours uncolored, no worklist
        // sort; it also counts the larger vertices and their work items), pending counts of
        // smaller-key neighbours in the unused second state array, then rounds over the ready
        // vertices only
        P.deg_hist = nullptr;
        P.T1 = T1 < kOrdSmall ? T1 : kOrdSmall;
        // a single graph's rounds are a chain of short latency-bound steps: 64-entry work items and
        // one block per SM by default (R-MAT-22: 33.8 ms against 39.7 with 128 entries and three
        // blocks; the grid barrier is cheaper with fewer blocks)
        const int32_t ch_ord = (opt && opt->chunk) || pb.batch ? CH : kOrdSingleChunk;
        P.CH = ch_ord < kOrdChunk ? ch_ord : kOrdChunk;
        GC_CUDA(launch_setup(P, GC_MODE_INPLACE, pb.batch, 0, static_cast<int32_t>(n), -1, s));
        GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
        if (h.err[0] != 0) return error_from_ctl(h);
        // each vertex is listed once: the item lists hold at most all items; a vertex of several
        // items has at least two, so there are at most items - larger vertices of them
        const size_t n_big = h.tmp[0], n_items = h.tmp[1];
        const size_t slots = std::min(n_big, n_items - n_big);
        GC_TRY(ensure(C.chunk0, 16 * std::max<size_t>(n_items, 1), "work items"));
        GC_TRY(ensure(C.chunk1, 16 * std::max<size_t>(n_items, 1), "work items"));
        GC_TRY(ensure(C.acc, 4 * kOrdSlotWords * std::max<size_t>(slots, 1), "accumulators"));
        GC_TRY(ensure(C.mid0, 4 * static_cast<size_t>(n), "worklist"));
        GC_TRY(ensure(C.mid1, 4 * static_cast<size_t>(n), "worklist"));
        P.chunk0 = C.chunk0.as<int4>();
        P.chunk1 = C.chunk1.as<int4>();
        P.mid0 = C.mid0.as<int32_t>();
        P.mid1 = C.mid1.as<int32_t>();
        P.acc = C.acc.as<unsigned>();
        if (slots) GC_CUDA(cudaMemsetAsync(C.acc.p, 0, 4 * kOrdSlotWords * slots, s));
        GC_CUDA(cudaMemsetAsync(ctl->cnt, 0, sizeof(ctl->cnt), s));
        if (timing) GC_CUDA(cudaEventRecord(C.ev[1], s));
        int &occ = C.occ_ord[pb.batch ? 1 : 0];
        if (occ == 0) GC_CUDA(ordered_kernel_occupancy(pb.batch, block, &occ));
        int per_sm = pb.batch ? occ : 1;
        if (opt && opt->blocks_per_sm > 0) per_sm = opt->blocks_per_sm < occ ? opt->blocks_per_sm : occ;
        grid = static_cast<int64_t>(per_sm) * C.sms;
        GC_TRY(wait_colidx(pb, s));
        GC_CUDA(launch_ordered(P, pb.batch, reinterpret_cast<int32_t *>(C.col1.p), static_cast<int>(grid), block, s));
    } else {
    GC_CUDA(launch_setup(P, mode, pb.batch, 0, static_cast<int32_t>(n), -1, s));
    GC_CUDA(launch_sort_small(P, pb.batch, 0, static_cast<int32_t>(n), s));
    GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    if (h.err[0] != 0) return error_from_ctl(h);
    const unsigned n_small = h.cnt[kCnt * 1 + kCntSmall];  // round 1 uses counter set 1
    const unsigned n_items = h.tmp[0], n_chunks = h.tmp[1];
    GC_TRY(ensure(C.chunk0, kItemBytes * static_cast<size_t>(n_chunks), "work items"));
    GC_TRY(ensure(C.chunk1, kItemBytes * static_cast<size_t>(n_chunks), "work items"));
    GC_TRY(ensure(C.acc, 4 * kAccStride * static_cast<size_t>(n_items), "accumulators"));
    if (mode == GC_MODE_INPLACE && n_items == 0) compact = false;
    // single graphs only: a batch's state words stay in L2 only while its vertices are taken block
    // by block in the sorted order
    P.spread = mode == GC_MODE_INPLACE && n_items == 0 && !pb.batch ? 1 : 0;
    if (compact) GC_TRY(ensure(C.lists, 4 * static_cast<size_t>(h.list_total), "neighbour lists"));
    // core phase (deterministic compact mode): the last rounds with the worklist's colors in shared
    // memory once at most core_M vertices with at most core_E list entries remain
    const int32_t core_opt = opt ? opt->core_vertices : 0;
    CoreParams Q{};
    if (mode == GC_MODE_DETERMINISTIC && compact && core_opt >= 0 && pb.nnz > 0) {
        if (C.core_max_v == 0) {
            const int32_t cm = core_max_vertices();
            C.core_max_v = cm > 0 ? cm : -1;
        }
        // the shared colors hold the core and a sentinel entry after it, in a multiple of 16 entries
        // (local ids stay below 2^18: a warp's batch of finished vertices packs them into 18 bits)
        int64_t M = std::min<int64_t>({n, static_cast<int64_t>(C.core_max_v) - 16, (int64_t{1} << 18) - 32});
        if (core_opt > 0) M = std::min<int64_t>(M, core_opt);
        if (M > 0) {
            const int64_t E = core_E;
            const size_t Mp = (static_cast<size_t>(M) + 16) & ~size_t{15};
            Q.max_v = static_cast<int32_t>(Mp);
            Q.max_e = E;
            Q.max_pieces = E / kCorePiece + static_cast<int64_t>(Mp) + 32;
            GC_TRY(ensure(C.core_rec, 4 * kCoreRecWords * Mp, "core records"));
            GC_TRY(ensure(C.core_cex, 2 * 4 * Mp, "core colors"));
            GC_TRY(ensure(C.core_c8, 2 * Mp, "core colors"));
            GC_TRY(ensure(C.core_fbits, 4 * (Mp / 32 + 1), "core final bits"));
            GC_TRY(ensure(C.core_items, 16 * static_cast<size_t>(Q.max_pieces), "core pieces"));
            GC_TRY(ensure(C.core_active, 2 * 4 * static_cast<size_t>(Q.max_pieces), "core active pieces"));
            GC_TRY(ensure(C.core_log, 2 * 8 * Mp, "core change log"));
            GC_TRY(ensure(C.core_pool, 4 * static_cast<size_t>(E) + 16, "core rows"));  // + prefetch slack
            Q.rec = C.core_rec.as<unsigned>();
            Q.cex = C.core_cex.as<int32_t>();
            Q.c8 = C.core_c8.as<uint8_t>();
            Q.fbits = C.core_fbits.as<unsigned>();
            GC_CUDA(cudaMemsetAsync(Q.fbits, 0, 4 * (Mp / 32 + 1), s));
            Q.pieces = C.core_items.as<int4>();
            Q.active = C.core_active.as<int32_t>();
            Q.log = C.core_log.as<uint2>();
            Q.pool = C.core_pool.as<int32_t>();
            Q.bump = &ctl->core_bump;
            Q.cnt = ctl->core_cnt;
            Q.m = ctl->core_m;
            P.core_max = static_cast<int32_t>(M);
            P.core_emax = E;
            P.core_go = &ctl->core_go;
            // tail phase: the last rounds on one cluster once at most tail_max vertices remain
            Q.tail = ctl->tail_ctl;
            const int32_t tail_opt = opt ? opt->tail_vertices : 0;
            if (tail_opt >= 0) {
                if (C.tail_nc == 0) {
                    const int32_t t = tail_cluster_size();
                    C.tail_nc = t > 0 ? t : -1;
                }
                if (C.tail_nc > 0) {
                    Q.tail_nc = C.tail_nc;
                    Q.tail_max = std::min(kTailOwned * C.tail_nc, tail_opt > 0 ? tail_opt : kTailDefault);
                }
            }
        }
    }
    P.chunk0 = C.chunk0.as<int4>();
    P.chunk1 = C.chunk1.as<int4>();
    P.acc = C.acc.as<unsigned>();
    P.lists = compact ? C.lists.as<int32_t>() : nullptr;
    GC_CUDA(launch_expand(P, mode, pb.batch, compact, static_cast<int32_t>(n_items), s));
    if (timing) GC_CUDA(cudaEventRecord(C.ev[1], s));

    // kernel variant: the 80-register one (3 blocks per SM) when most adjacency entries belong to
    // larger vertices, whose warp sweep keeps more in registers; the 64-register one (4 blocks per
    // SM, more warps) when most are swept one thread per vertex.  blocks_per_sm = 3 or 4 picks one.
    const int bps_opt = opt ? opt->blocks_per_sm : 0;
    const bool wide = bps_opt == 3 || (bps_opt == 0 && 2 * static_cast<int64_t>(n_chunks) * CH >= pb.nnz &&
                                       n_chunks > 0);
    // persistent grid: every block resident; no more blocks than the first round can use
    int &occ = C.occ[wide ? 1 : 0][mode][pb.batch ? 1 : 0][compact ? 1 : 0];
    if (occ == 0) GC_CUDA(round_kernel_occupancy(mode, pb.batch, compact, block, &occ, wide));
    int per_sm = occ;
    if (bps_opt > 0 && bps_opt < per_sm) per_sm = bps_opt;
    grid = static_cast<int64_t>(per_sm) * C.sms;
    const int64_t want = (static_cast<int64_t>(n_small) + 32 * static_cast<int64_t>(n_chunks) + block - 1) / block;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    GC_TRY(wait_colidx(pb, s));
    GC_CUDA(launch_rounds(P, mode, pb.batch, compact, static_cast<int>(grid), block, s, wide));
    if (P.core_max > 0) GC_CUDA(launch_core(P, Q, pb.batch, s));
    }
    if (timing) GC_CUDA(cudaEventRecord(C.ev[2], s));

    // colors, per-graph counts; a device colors_out is written only if no error was posted, a host
    // one is staged through st_colors and copied after the status is known
    int out_dev = 0;
    GC_TRY(locate(out.colors, dev, &out_dev));
    if (!out_dev && out.colors) GC_TRY(ensure(C.st_colors, 4 * n, "color staging"));
    int32_t *colors_dev = out_dev ? out.colors : (out.colors ? C.st_colors.as<int32_t>() : nullptr);
    NvtxRange count_range("gc: color count and output");
    GC_CUDA(launch_count_colors(P, pb.batch, mode == GC_MODE_DETERMINISTIC ? &ctl->passes[1] : nullptr, 0,
                                static_cast<int32_t>(n), 0, G, C.bitmap.as<unsigned>(),
                                pb.batch ? C.gmax.as<int32_t>() : &ctl->gmax1,
                                pb.batch ? C.gcount.as<int32_t>() : &ctl->gcount1, colors_dev, s));
    std::vector<int64_t> st_host(4 * static_cast<size_t>(stats_cap) + 1);
    if (stats_cap)
        GC_CUDA(cudaMemcpyAsync(st_host.data(), C.stats.p, 8 * st_host.size(), cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> gmax_h, gcount_h, glast_h;
    if (pb.batch) {
        gmax_h.resize(gz);
        gcount_h.resize(gz);
        glast_h.resize(gz);
        GC_CUDA(cudaMemcpyAsync(gmax_h.data(), C.gmax.p, 4 * gz, cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaMemcpyAsync(gcount_h.data(), C.gcount.p, 4 * gz, cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaMemcpyAsync(glast_h.data(), C.glast.p, 4 * gz, cudaMemcpyDeviceToHost, s));
    }
    GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    if (h.err[0] != 0) return error_from_ctl(h);

    const int32_t last = h.passes[1];  // last round executed (0: every vertex isolated)
    if (!out_dev && out.colors)
        GC_CUDA(cudaMemcpyAsync(out.colors, colors_dev, 4 * static_cast<size_t>(n), cudaMemcpyDeviceToHost, s));
    const int32_t rounds_single = n > 0 ? (last > 0 ? last : 1) : 0;
    if (pb.batch) {
        int on_dev = 0;
        if (out.ncolors) {
            GC_TRY(locate(out.ncolors, dev, &on_dev));
            if (on_dev)
                GC_CUDA(cudaMemcpyAsync(out.ncolors, C.gcount.p, 4 * gz, cudaMemcpyDeviceToDevice, s));
            else
                std::memcpy(out.ncolors, gcount_h.data(), 4 * gz);
        }
        if (out.rounds) {
            GC_TRY(locate(out.rounds, dev, &on_dev));
            if (on_dev)
                GC_CUDA(cudaMemcpyAsync(out.rounds, C.glast.p, 4 * gz, cudaMemcpyDeviceToDevice, s));
            else
                std::memcpy(out.rounds, glast_h.data(), 4 * gz);
        }
    } else {
        if (out.ncolors) *out.ncolors = h.gcount1;
        if (out.rounds) *out.rounds = rounds_single;
    }
    GC_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        int32_t total_colors = 0, maxc = -1;
        if (pb.batch) {
            for (int32_t g = 0; g < G; ++g) {
                total_colors += gcount_h[g];
                if (gmax_h[g] > maxc) maxc = gmax_h[g];
            }
        } else {
            total_colors = h.gcount1;
            maxc = h.gmax1;
        }
        stats->rounds = rounds_single;
        stats->ncolors = total_colors;
        stats->max_color = maxc;
        stats->grid_blocks = static_cast<int32_t>(grid);
        stats->block_size = block;
        stats->worklist_total = 0;
        stats->entries_scanned = 0;
        if (stats_cap) {
            const int32_t R = last < stats_cap ? last : stats_cap;
            int64_t prev_t = st_host[4 * static_cast<size_t>(stats_cap)];
            for (int32_t r = 0; r < R; ++r) {
                int64_t w = st_host[4 * r], d = st_host[4 * r + 1];
                const int64_t t_end = st_host[4 * r + 2];
                stats->entries_scanned += st_host[4 * r + 3];
                if (stats->round_reads && r < stats->round_cap) stats->round_reads[r] = st_host[4 * r + 3];
                if (stats->round_ns && r < stats->round_cap) stats->round_ns[r] = t_end - prev_t;
                prev_t = t_end;
                if (r == 0 && mode != GC_MODE_ORDERED) {
                    w = n;  // W_1 = V; isolated vertices are final before the first sweep
                    d = pb.nnz;
                }
                stats->worklist_total += w;
                if (stats->wl_size && r < stats->round_cap) stats->wl_size[r] = w;
                if (stats->wl_degsum && r < stats->round_cap) stats->wl_degsum[r] = d;
            }
            if (last == 0 && n > 0) {
                stats->worklist_total = n;
                if (stats->wl_size && stats->round_cap > 0) stats->wl_size[0] = n;
                if (stats->wl_degsum && stats->round_cap > 0) stats->wl_degsum[0] = 0;
            }
        }
        stats->kernel_ms = 0.f;
        stats->setup_ms = 0.f;
        if (timing) {
            cudaEventElapsedTime(&stats->setup_ms, C.ev[0], C.ev[1]);
            cudaEventElapsedTime(&stats->kernel_ms, C.ev[1], C.ev[2]);
        }
    }
    return GC_OK;
}

// Device views of a single graph's CSR (host arrays staged), with GC_FLAG_VALIDATE applied.
static int single_problem(Context *C, int32_t n, const int32_t *rowptr, const int32_t *colidx, const gc_options *opt,
                          cudaStream_t s, Problem &pb) {
    int rp_dev = 0;
    GC_TRY(locate(rowptr, C->device, &rp_dev));
    int32_t nnz32 = 0;
    if (rp_dev) {
        GC_CUDA(cudaMemcpyAsync(&nnz32, rowptr + n, 4, cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
    } else {
        nnz32 = rowptr[n];
    }
    if (nnz32 < 0) return set_last_error(GC_ERR_INVALID_GRAPH, "rowptr[n] = %d is negative", nnz32);
    if (nnz32 > 0 && !colidx) return set_last_error(GC_ERR_INVALID_ARG, "NULL colidx with %d entries", nnz32);
    pb.batch = false;
    pb.G = 1;
    pb.n = n;
    pb.nnz = nnz32;
    const void *v = nullptr;
    GC_TRY(device_view(rowptr, 4 * (static_cast<size_t>(n) + 1), C->device, C->st_rowptr, s, &v));
    pb.rowptr = static_cast<const int32_t *>(v);
    int ci_dev = 0;
    GC_TRY(locate(colidx, C->device, &ci_dev));
    if (!ci_dev && nnz32 > 0 && C->copy_stream) {
        // the largest upload runs beside the set-up kernels, which read only the row offsets
        GC_CUDA(cudaEventRecord(C->ev_before, s));
        GC_CUDA(cudaStreamWaitEvent(C->copy_stream, C->ev_before, 0));
        GC_TRY(device_view(colidx, 4 * static_cast<size_t>(nnz32), C->device, C->st_colidx, C->copy_stream, &v));
        GC_CUDA(cudaEventRecord(C->ev_colidx, C->copy_stream));
        pb.colidx_ready = C->ev_colidx;
    } else {
        GC_TRY(device_view(colidx, 4 * static_cast<size_t>(nnz32), C->device, C->st_colidx, s, &v));
    }
    pb.colidx = static_cast<const int32_t *>(v);
    if (opt && (opt->flags & GC_FLAG_VALIDATE)) {
        GC_TRY(wait_colidx(pb, s));
        GC_TRY(ensure(C->ctl, sizeof(Ctl), "control"));
        Ctl *ctl = C->ctl.as<Ctl>();
        GC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
        GC_CUDA(launch_validate(n, pb.rowptr, pb.colidx ? pb.colidx : pb.rowptr, GC_VALIDATE_ALL, ctl->err, s));
        Ctl h{};
        GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
        if (h.err[0] != 0) return error_from_ctl(h);
    }
    if (!pb.colidx) pb.colidx = pb.rowptr;  // never dereferenced when nnz == 0
    return GC_OK;
}

static int color_single(int32_t n, const int32_t *rowptr, const int32_t *colidx, int mode, uint64_t seed,
                        int32_t *colors_out, int32_t *ncolors, int32_t *rounds, const gc_options *opt,
                        gc_stats *stats, const int32_t *colors_in = nullptr) {
    if (n < 0) return set_last_error(GC_ERR_INVALID_ARG, "n = %d is negative", n);
    if (mode != GC_MODE_DETERMINISTIC && mode != GC_MODE_INPLACE && mode != GC_MODE_PARTITION &&
        mode != GC_MODE_ORDERED)
        return set_last_error(GC_ERR_INVALID_ARG, "unknown mode %d", mode);
    if (n > 0 && (!rowptr || !colors_out)) return set_last_error(GC_ERR_INVALID_ARG, "NULL rowptr or colors_out");
    if (n == INT32_MAX) return set_last_error(GC_ERR_INVALID_ARG, "n too large");
    Context *C = nullptr;
    GC_TRY(get_context(&C));
    std::lock_guard<std::mutex> lk(C->mu);
    GC_CUDA(cudaSetDevice(C->device));
    if (n == 0) {
        if (ncolors) *ncolors = 0;
        if (rounds) *rounds = 0;
        if (stats) {
            int32_t cap = stats->round_cap;
            int64_t *a = stats->wl_size, *b = stats->wl_degsum, *t = stats->round_ns, *rr = stats->round_reads;
            std::memset(stats, 0, sizeof(*stats));
            stats->round_cap = cap;
            stats->wl_size = a;
            stats->wl_degsum = b;
            stats->round_ns = t;
            stats->round_reads = rr;
            stats->max_color = -1;
        }
        return GC_OK;
    }
    cudaStream_t s = (opt && opt->stream) ? static_cast<cudaStream_t>(opt->stream) : C->stream;
    Problem pb{};
    UploadGuard upload{C->copy_stream};
    GC_TRY(single_problem(C, n, rowptr, colidx, opt, s, pb));
    const void *v = nullptr;
    if (colors_in) {
        GC_TRY(device_view(colors_in, 4 * static_cast<size_t>(n), C->device, C->st_colors_in, s, &v));
        pb.prio_rank = static_cast<const int32_t *>(v);
        pb.priority_override = kPriorityRecolor;
    }
    Outputs o{colors_out, ncolors, rounds};
    return run(*C, pb, mode, seed, opt, stats, o);
}

static int color_batch(int32_t G, const int64_t *vtx_off, const int64_t *edge_off, const int32_t *rowptr,
                       const int32_t *colidx, int mode, uint64_t seed, int32_t *colors_out, int32_t *ncolors,
                       int32_t *rounds, const gc_options *opt, gc_stats *stats) {
    if (G < 0) return set_last_error(GC_ERR_INVALID_ARG, "G = %d is negative", G);
    if (mode != GC_MODE_DETERMINISTIC && mode != GC_MODE_INPLACE && mode != GC_MODE_ORDERED)
        return set_last_error(GC_ERR_INVALID_ARG, "unknown mode %d", mode);
    if (G > 0 && (!vtx_off || !edge_off)) return set_last_error(GC_ERR_INVALID_ARG, "NULL offset table");
    Context *C = nullptr;
    GC_TRY(get_context(&C));
    std::lock_guard<std::mutex> lk(C->mu);
    GC_CUDA(cudaSetDevice(C->device));
    if (G == 0) {
        if (stats) {
            std::memset(stats, 0, offsetof(gc_stats, round_cap));
            stats->max_color = -1;
        }
        return GC_OK;
    }
    cudaStream_t s = (opt && opt->stream) ? static_cast<cudaStream_t>(opt->stream) : C->stream;
    int vd = 0, ed = 0;
    GC_TRY(locate(vtx_off, C->device, &vd));
    GC_TRY(locate(edge_off, C->device, &ed));
    int64_t N = 0, NNZ = 0;
    if (vd)
        GC_CUDA(cudaMemcpyAsync(&N, vtx_off + G, 8, cudaMemcpyDeviceToHost, s));
    else
        N = vtx_off[G];
    if (ed)
        GC_CUDA(cudaMemcpyAsync(&NNZ, edge_off + G, 8, cudaMemcpyDeviceToHost, s));
    else
        NNZ = edge_off[G];
    GC_CUDA(cudaStreamSynchronize(s));
    if (N < 0 || NNZ < 0) return set_last_error(GC_ERR_INVALID_GRAPH, "negative totals in offset tables");
    if (N >= INT32_MAX - G) return set_last_error(GC_ERR_INVALID_ARG, "batch too large: %lld vertices", (long long)N);
    if (N > 0 && (!rowptr || !colors_out)) return set_last_error(GC_ERR_INVALID_ARG, "NULL rowptr or colors_out");
    if (NNZ > 0 && !colidx) return set_last_error(GC_ERR_INVALID_ARG, "NULL colidx");
    Problem pb{};
    pb.batch = true;
    pb.G = G;
    pb.n = static_cast<int32_t>(N);
    pb.nnz = NNZ;
    const void *v = nullptr;
    GC_TRY(device_view(vtx_off, 8 * (static_cast<size_t>(G) + 1), C->device, C->st_vtx, s, &v));
    pb.vtx_off = static_cast<const int64_t *>(v);
    GC_TRY(device_view(edge_off, 8 * (static_cast<size_t>(G) + 1), C->device, C->st_edge, s, &v));
    pb.edge_off = static_cast<const int64_t *>(v);
    GC_TRY(device_view(rowptr, 4 * (static_cast<size_t>(N) + G), C->device, C->st_rowptr, s, &v));
    pb.rowptr = static_cast<const int32_t *>(v);
    GC_TRY(device_view(colidx, 4 * static_cast<size_t>(NNZ), C->device, C->st_colidx, s, &v));
    pb.colidx = v ? static_cast<const int32_t *>(v) : pb.rowptr;
    Outputs o{colors_out, ncolors, rounds};
    return run(*C, pb, mode, seed, opt, stats, o);
}

}  // namespace gc

// ------------------------------------------------------------------------------------------
// exported entry points

extern "C" {

int gc_color(int32_t n, const int32_t *rowptr, const int32_t *colidx, int mode, uint64_t seed, int32_t *colors_out,
             int32_t *ncolors, int32_t *rounds) {
    return gc::color_single(n, rowptr, colidx, mode, seed, colors_out, ncolors, rounds, nullptr, nullptr);
}

int gc_color_ex(int32_t n, const int32_t *rowptr, const int32_t *colidx, int mode, uint64_t seed, int32_t *colors_out,
                int32_t *ncolors, int32_t *rounds, const gc_options *opt, gc_stats *stats) {
    return gc::color_single(n, rowptr, colidx, mode, seed, colors_out, ncolors, rounds, opt, stats);
}

int gc_smallest_last(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *level_out, int32_t *nlevels,
                     int32_t *degeneracy, const gc_options *opt) {
    using namespace gc;
    if (n < 0) return set_last_error(GC_ERR_INVALID_ARG, "n = %d is negative", n);
    if (n > 0 && (!rowptr || !level_out)) return set_last_error(GC_ERR_INVALID_ARG, "NULL rowptr or level_out");
    if (n == INT32_MAX) return set_last_error(GC_ERR_INVALID_ARG, "n too large");
    const int32_t T1 = (opt && opt->small_max_degree) ? opt->small_max_degree : 127;
    const int32_t CH = (opt && opt->chunk) ? opt->chunk : 1024;
    if (T1 < 1 || T1 > 127) return set_last_error(GC_ERR_INVALID_ARG, "small_max_degree %d outside 1..127", T1);
    if (CH < 32 || CH > 8192 || CH % 32) return set_last_error(GC_ERR_INVALID_ARG, "chunk %d invalid", CH);
    Context *C = nullptr;
    GC_TRY(get_context(&C));
    std::lock_guard<std::mutex> lk(C->mu);
    GC_CUDA(cudaSetDevice(C->device));
    if (n == 0) {
        if (nlevels) *nlevels = 0;
        if (degeneracy) *degeneracy = 0;
        return GC_OK;
    }
    cudaStream_t s = (opt && opt->stream) ? static_cast<cudaStream_t>(opt->stream) : C->stream;
    Problem pb{};
    UploadGuard upload{C->copy_stream};
    GC_TRY(single_problem(C, n, rowptr, colidx, opt, s, pb));
    GC_TRY(ensure(C->ctl, sizeof(Ctl), "control"));
    Ctl *ctl = C->ctl.as<Ctl>();
    GC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    RoundParams P{};
    P.n = n;
    P.G = 1;
    P.nnz = pb.nnz;
    P.rowptr = pb.rowptr;
    P.colidx = pb.colidx;
    P.cnt = ctl->cnt;
    P.bar = &ctl->bar;
    P.err = ctl->err;
    P.passes = ctl->passes;
    P.spin_ns = (opt && opt->spin_limit_ns > 0) ? opt->spin_limit_ns : 1000000000LL;
    int32_t nl = 0, dg = 0;
    GC_TRY(wait_colidx(pb, s));
    GC_TRY(peel_levels(*C, ctl, P, T1, CH, s, &nl, &dg, opt ? opt->blocks_per_sm : 0));
    int out_dev = 0;
    GC_TRY(locate(level_out, C->device, &out_dev));
    GC_CUDA(cudaMemcpyAsync(level_out, C->rank.p, 4 * static_cast<size_t>(n),
                            out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    if (nlevels) *nlevels = nl;
    if (degeneracy) *degeneracy = dg;
    return GC_OK;
}

int gc_recolor(int32_t n, const int32_t *rowptr, const int32_t *colidx, const int32_t *colors_in, uint64_t seed,
               int32_t *colors_out, int32_t *ncolors, int32_t *rounds, const gc_options *opt, gc_stats *stats) {
    if (n > 0 && !colors_in) return gc::set_last_error(GC_ERR_INVALID_ARG, "NULL colors_in");
    return gc::color_single(n, rowptr, colidx, GC_MODE_ORDERED, seed, colors_out, ncolors, rounds, opt, stats,
                            colors_in);
}

int gc_color_batch(int32_t G, const int64_t *vtx_off, const int64_t *edge_off, const int32_t *rowptr,
                   const int32_t *colidx, int mode, uint64_t seed, int32_t *colors_out, int32_t *ncolors,
                   int32_t *rounds) {
    return gc::color_batch(G, vtx_off, edge_off, rowptr, colidx, mode, seed, colors_out, ncolors, rounds, nullptr,
                           nullptr);
}

int gc_color_batch_ex(int32_t G, const int64_t *vtx_off, const int64_t *edge_off, const int32_t *rowptr,
                      const int32_t *colidx, int mode, uint64_t seed, int32_t *colors_out, int32_t *ncolors,
                      int32_t *rounds, const gc_options *opt, gc_stats *stats) {
    return gc::color_batch(G, vtx_off, edge_off, rowptr, colidx, mode, seed, colors_out, ncolors, rounds, opt, stats);
}

int gc_validate_graph(int32_t n, const int32_t *rowptr, const int32_t *colidx, int flags) {
    using namespace gc;
    if (n < 0) return set_last_error(GC_ERR_INVALID_ARG, "n = %d is negative", n);
    if (n > 0 && !rowptr) return set_last_error(GC_ERR_INVALID_ARG, "NULL rowptr");
    if ((flags & GC_VALIDATE_SYMMETRIC) && !(flags & GC_VALIDATE_SORTED))
        return set_last_error(GC_ERR_INVALID_ARG, "GC_VALIDATE_SYMMETRIC requires GC_VALIDATE_SORTED");
    Context *C = nullptr;
    GC_TRY(get_context(&C));
    std::lock_guard<std::mutex> lk(C->mu);
    GC_CUDA(cudaSetDevice(C->device));
    if (n == 0) return GC_OK;
    cudaStream_t s = C->stream;
    int rp_dev = 0;
    GC_TRY(locate(rowptr, C->device, &rp_dev));
    int32_t nnz = 0;
    if (rp_dev) {
        GC_CUDA(cudaMemcpyAsync(&nnz, rowptr + n, 4, cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
    } else {
        nnz = rowptr[n];
    }
    if (nnz < 0) return set_last_error(GC_ERR_INVALID_GRAPH, "rowptr[n] = %d is negative", nnz);
    if (nnz > 0 && !colidx) return set_last_error(GC_ERR_INVALID_ARG, "NULL colidx");
    const void *v = nullptr;
    GC_TRY(device_view(rowptr, 4 * (static_cast<size_t>(n) + 1), C->device, C->st_rowptr, s, &v));
    const int32_t *rp = static_cast<const int32_t *>(v);
    GC_TRY(device_view(colidx, 4 * static_cast<size_t>(nnz), C->device, C->st_colidx, s, &v));
    const int32_t *ci = v ? static_cast<const int32_t *>(v) : rp;
    GC_TRY(ensure(C->ctl, sizeof(Ctl), "control"));
    Ctl *ctl = C->ctl.as<Ctl>();
    GC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    GC_CUDA(launch_validate(n, rp, ci, flags, ctl->err, s));
    Ctl h{};
    GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    if (h.err[0] != 0) {
        const int64_t where =
            (static_cast<int64_t>(static_cast<uint32_t>(h.err[3])) << 32) | static_cast<uint32_t>(h.err[2]);
        return set_last_error(GC_ERR_INVALID_GRAPH,
                              "invalid graph at vertex %d, entry %lld (range, self-loop%s%s)", h.err[1],
                              static_cast<long long>(where), (flags & GC_VALIDATE_SORTED) ? ", order/duplicate" : "",
                              (flags & GC_VALIDATE_SYMMETRIC) ? ", missing reverse entry" : "");
    }
    return GC_OK;
}

const char *gc_last_error(void) { return gc::t_error.c_str(); }

int gc_version(void) { return 100; }

int gc_det_round(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed, const int32_t *colors_cur,
                 const int32_t *worklist, int32_t nwork, int32_t *colors_next, int32_t *lost) {
    using namespace gc;
    if (n < 0 || nwork < 0) return set_last_error(GC_ERR_INVALID_ARG, "negative n or nwork");
    if (nwork == 0) return GC_OK;
    if (!rowptr || !colors_cur || !worklist || !colors_next || !lost)
        return set_last_error(GC_ERR_INVALID_ARG, "NULL array");
    Context *C = nullptr;
    GC_TRY(get_context(&C));
    std::lock_guard<std::mutex> lk(C->mu);
    GC_CUDA(cudaSetDevice(C->device));
    cudaStream_t s = C->stream;
    int rp_dev = 0;
    GC_TRY(locate(rowptr, C->device, &rp_dev));
    int32_t nnz = 0;
    if (rp_dev) {
        GC_CUDA(cudaMemcpyAsync(&nnz, rowptr + n, 4, cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
    } else {
        nnz = rowptr[n];
    }
    if (nnz < 0) return set_last_error(GC_ERR_INVALID_GRAPH, "rowptr[n] = %d is negative", nnz);
    if (nnz > 0 && !colidx) return set_last_error(GC_ERR_INVALID_ARG, "NULL colidx");
    const void *v = nullptr;
    GC_TRY(device_view(rowptr, 4 * (static_cast<size_t>(n) + 1), C->device, C->st_rowptr, s, &v));
    const int32_t *rp = static_cast<const int32_t *>(v);
    GC_TRY(device_view(colidx, 4 * static_cast<size_t>(nnz), C->device, C->st_colidx, s, &v));
    const int32_t *ci = v ? static_cast<const int32_t *>(v) : rp;
    GC_TRY(device_view(colors_cur, 4 * static_cast<size_t>(n), C->device, C->st_cur, s, &v));
    const int32_t *cur = static_cast<const int32_t *>(v);
    GC_TRY(device_view(worklist, 4 * static_cast<size_t>(nwork), C->device, C->st_work, s, &v));
    const int32_t *work = static_cast<const int32_t *>(v);
    int next_dev = 0, lost_dev = 0;
    GC_TRY(locate(colors_next, C->device, &next_dev));
    GC_TRY(locate(lost, C->device, &lost_dev));
    if (!next_dev) GC_TRY(ensure(C->st_next, 4 * static_cast<size_t>(nwork), "round output"));
    if (!lost_dev) GC_TRY(ensure(C->st_lost, 4 * static_cast<size_t>(nwork), "round output"));
    int32_t *next_d = next_dev ? colors_next : C->st_next.as<int32_t>();
    int32_t *lost_d = lost_dev ? lost : C->st_lost.as<int32_t>();
    GC_TRY(ensure(C->ctl, sizeof(Ctl), "control"));
    Ctl *ctl = C->ctl.as<Ctl>();
    GC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    GC_CUDA(launch_det_round_block(n, rp, ci, seed, cur, work, nwork, next_d, lost_d, ctl->err, s));
    Ctl h{};
    GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    if (h.err[0] == GC_ERR_INVALID_ARG)
        return set_last_error(GC_ERR_INVALID_ARG, "worklist entry %d is not a vertex id", h.err[1]);
    if (h.err[0] != 0) return error_from_ctl(h);
    if (!next_dev)
        GC_CUDA(cudaMemcpyAsync(colors_next, next_d, 4 * static_cast<size_t>(nwork), cudaMemcpyDeviceToHost, s));
    if (!lost_dev) GC_CUDA(cudaMemcpyAsync(lost, lost_d, 4 * static_cast<size_t>(nwork), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    return GC_OK;
}

int gc_release_scratch(void) {
    using namespace gc;
    Context *C = nullptr;
    GC_TRY(get_context(&C));
    std::lock_guard<std::mutex> lk(C->mu);
    GC_CUDA(cudaStreamSynchronize(C->stream));
    C->release_all();
    return GC_OK;
}

}  // extern "C"
