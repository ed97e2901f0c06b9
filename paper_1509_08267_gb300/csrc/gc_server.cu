// Continuous-batching coloring server (gc_server_* in include/gc.h).
//
// A worker thread owns a resident device pool (CSR storage, color/priority/worklist state) and
// runs the batched round kernel a few rounds per launch over every resident request.  Between
// launches it (1) retires requests none of whose vertices is on the next round's worklist,
// (2) admits queued requests whose footprint fits the free pool space (first fit over vertex,
// entry and work-item ranges), joining them to the running batch at the next round: their first
// round is the batch's next round, and a request's own round count is measured from there.
// Because every graph's deterministic rounds read only its own previous colors, a request's
// colors do not depend on which other requests share the launch.  A request large enough to fill
// the GPU by itself (cfg.solo_entries) skips the pool: between launches the worker colors it alone
// the way gc_color_ex does, with the core and tail phases that the batch's shared rounds cannot run.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gc_internal.h"

namespace gc {
namespace {

constexpr int32_t kRoundsWhileQueued = 4;   // rounds per launch while requests wait for admission
constexpr int32_t kRoundsIdleQueue = 16;    // rounds per launch when nothing waits
constexpr int32_t kT1 = 127;
constexpr int32_t kCH = 1024;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, capacity) with coalescing of freed ranges.
class RangeAlloc {
  public:
    explicit RangeAlloc(int64_t cap = 0) { reset(cap); }
    void reset(int64_t cap) {
        free_.clear();
        if (cap > 0) free_[0] = cap;
        cap_ = cap;
    }
    bool alloc(int64_t len, int64_t *start) {
        if (len == 0) {
            *start = 0;
            return true;
        }
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *start = it->first;
                const int64_t rest = it->second - len, at = it->first + len;
                free_.erase(it);
                if (rest > 0) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(int64_t start, int64_t len) {
        if (len == 0) return;
        auto it = free_.emplace(start, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t capacity() const { return cap_; }

  private:
    std::map<int64_t, int64_t> free_;
    int64_t cap_ = 0;
};

enum ReqState { kQueued, kResident, kDone };

struct Engine;

struct Request {
    uint64_t id = 0;
    int32_t n = 0;
    int64_t m = 0;
    int32_t mode = GC_MODE_DETERMINISTIC;
    uint64_t seed = 0;
    Engine *eng = nullptr;
    int64_t n_large = 0, n_chunks = 0;
    std::vector<int32_t> rowptr, colidx, colors;
    ReqState state = kQueued;
    int status = GC_OK;
    int32_t ncolors = 0, rounds = 0;
    double t_submit = 0, t_done = 0;
    int32_t slot = -1, join = 0;
    int64_t vbase = 0, ebase = 0, rbase = 0;
    bool staged = false;  // its CSR was copied into the pool at submit
    void *dbuf = nullptr;  // colored alone: its row offsets, entries and colors on the device
};

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
    }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16); }
    template <class T>
    T *as() const {
        return static_cast<T *>(p);
    }
};

struct Ctl {
    int32_t err[4];
    int32_t passes[2];
    int32_t pad0[2];
    unsigned cnt[3 * kCnt];
    unsigned tmp[2];
    int32_t pad2[10];
    GridBar bar;
};

// One mode's resident pool: CSR storage, vertex state, worklists and the graph table of the
// batched round kernel, with first-fit allocators for vertex, entry and row-offset ranges and a
// work-item budget.
struct Engine {
    int mode = -1;  // -1: not allocated yet
    bool compact = false;  // deterministic mode: the compact sweep (slot and list space per pool vertex / entry)
    int grid = 0;
    int64_t PV = 0, PE = 0, PI = 0, PC = 0;  // capacities: vertices, entries, large vertices, work items
    int32_t S = 0;                           // slots
    DevBuf rowptr, colidx, col0, col1, outbuf, small0, small1, items, chunk0, chunk1, acc, lists, vg, ctl, bitmap;
    DevBuf g_vbase, g_n, g_ebase, g_rbase, g_m, glast, gmax, gcount, verr, gseed;
    std::vector<int64_t> h_vbase, h_ebase, h_rbase, h_m;
    std::vector<int32_t> h_n, h_glast;
    std::vector<uint64_t> h_seed;
    RangeAlloc va, ea, ra;
    int64_t used_items = 0, used_chunks = 0;
    std::vector<int32_t> free_slots;
    std::vector<Request *> resident;
    std::deque<Request *> queue;
    std::vector<Request *> staged;  // pool space reserved and CSR copied at submit
    int32_t next_pass = 1;
    bool busy() const { return mode >= 0 && (!queue.empty() || !resident.empty() || !staged.empty()); }
};

}  // namespace
}  // namespace gc

struct gc_server {
    gc_server_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;
    std::mutex copy_mu;
    std::mutex create_mu;  // engine allocation
    gc::Engine eng[2];     // [0] deterministic, [1] in-place
    std::deque<gc::Request *> solo;  // requests colored alone, in submission order
    int64_t solo_min = 0;            // adjacency entries from which a request is colored alone
    cudaMemPool_t solo_pool = nullptr;  // their device copies; freed memory stays in the pool
    std::unordered_map<uint64_t, std::unique_ptr<gc::Request>> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    // statistics
    int64_t submitted = 0, completed = 0, rejected = 0, failed = 0, rounds_run = 0, v_done = 0, e_done = 0;
    std::vector<double> latencies;
    double t_create = 0, busy = 0;
    int fatal = GC_OK;
    std::string fatal_msg;
};

namespace gc {
namespace {

int srv_fail(gc_server *s, int code, const char *what, cudaError_t e) {
    s->fatal = code;
    s->fatal_msg = std::string(what) + ": " + cudaGetErrorString(e);
    return code;
}

#define SRV_CUDA(call)                                                     \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return srv_fail(s, GC_ERR_CUDA, #call, e_); \
    } while (0)

int engine_index(int mode) { return mode == GC_MODE_INPLACE ? 1 : 0; }

// Allocates the pool of `mode` with the server's capacities (E.mode is left to the caller, which
// publishes the pool by setting it under the server lock).
int engine_create(gc_server *s, Engine &E, int mode) {
    const gc_server_config &cfg = s->cfg;
    E.S = cfg.max_requests > 0 ? cfg.max_requests : 4096;
    E.PV = cfg.pool_vertices;
    E.PE = cfg.pool_entries;
    E.PI = std::min<int64_t>(E.PV, E.PE / (kT1 + 1) + 1);
    E.PC = E.PE / kCH + E.PI + 1;
    // deterministic mode sweeps compact lists: a slot per pool vertex and two list regions per entry
    E.compact = mode == GC_MODE_DETERMINISTIC;
    const size_t slots = E.compact ? static_cast<size_t>(E.PV) : static_cast<size_t>(E.PI);
    const size_t V = static_cast<size_t>(E.PV), Sz = static_cast<size_t>(E.S);
    struct {
        DevBuf *b;
        size_t bytes;
    } plan[] = {
        {&E.rowptr, 4 * (V + Sz)}, {&E.colidx, 4 * static_cast<size_t>(E.PE)}, {&E.col0, 8 * V}, {&E.col1, 8 * V},
        {&E.outbuf, 4 * V}, {&E.small0, 4 * V}, {&E.small1, 4 * V}, {&E.items, 4 * V}, {&E.vg, 4 * V},
        {&E.chunk0, kItemBytes * static_cast<size_t>(E.PC)}, {&E.chunk1, kItemBytes * static_cast<size_t>(E.PC)},
        {&E.acc, 4 * kAccStride * slots}, {&E.lists, E.compact ? 8 * static_cast<size_t>(E.PE) : 0},
        {&E.ctl, sizeof(Ctl)}, {&E.bitmap, 4 * (V / 32 + 4)}, {&E.g_vbase, 8 * Sz}, {&E.g_n, 4 * Sz},
        {&E.g_ebase, 8 * Sz}, {&E.g_rbase, 8 * Sz}, {&E.g_m, 8 * Sz}, {&E.glast, 4 * Sz}, {&E.gmax, 4 * Sz},
        {&E.gcount, 4 * Sz}, {&E.verr, 16 * Sz}, {&E.gseed, 8 * Sz},
    };
    cudaError_t e = cudaSuccess;
    for (auto &a : plan) {
        if (e != cudaSuccess) break;
        e = a.b->alloc(a.bytes);
    }
    if (e == cudaSuccess) e = cudaMemset(E.ctl.p, 0, sizeof(Ctl));
    if (e == cudaSuccess) e = cudaMemset(E.acc.p, 0, 4 * kAccStride * slots);
    if (e == cudaSuccess) e = cudaMemset(E.g_n.p, 0, 4 * Sz);
    if (e == cudaSuccess) e = cudaMemset(E.glast.p, 0, 4 * Sz);
    if (e == cudaSuccess) e = cudaMemset(E.gseed.p, 0, 8 * Sz);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (auto &a : plan) a.b->release();
        return set_last_error(e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA, "server pool: %s",
                              cudaGetErrorString(e));
    }
    int per_sm = 0, sms = 0;
    round_kernel_occupancy(mode, true, E.compact, 256, &per_sm);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    E.grid = std::max(1, per_sm * sms);
    E.h_vbase.assign(Sz, 0);
    E.h_ebase.assign(Sz, 0);
    E.h_rbase.assign(Sz, 0);
    E.h_m.assign(Sz, 0);
    E.h_n.assign(Sz, 0);
    E.h_glast.assign(Sz, 0);
    E.h_seed.assign(Sz, 0);
    E.va.reset(E.PV);
    E.ea.reset(E.PE);
    E.ra.reset(E.PV + E.S);
    E.free_slots.clear();
    for (int32_t g = E.S - 1; g >= 0; --g) E.free_slots.push_back(g);
    E.next_pass = 1;
    return GC_OK;
}

RoundParams params(gc_server *s, Engine &E, int32_t rounds = kRoundsWhileQueued) {
    RoundParams P{};
    P.n = static_cast<int32_t>(E.PV);
    P.G = E.S;
    P.rowptr = E.rowptr.as<int32_t>();
    P.colidx = E.colidx.as<int32_t>();
    P.g_vbase = E.g_vbase.as<int64_t>();
    P.g_n = E.g_n.as<int32_t>();
    P.g_ebase = E.g_ebase.as<int64_t>();
    P.g_rbase = E.g_rbase.as<int64_t>();
    P.g_m = E.g_m.as<int64_t>();
    P.vg = E.vg.as<int32_t>();
    P.seed = 0;
    P.g_seed = E.gseed.as<uint64_t>();  // every request has its own seed
    P.col0 = E.col0.as<uint64_t>();
    P.col1 = E.col1.as<uint64_t>();
    P.small0 = E.small0.as<int32_t>();
    P.small1 = E.small1.as<int32_t>();
    P.chunk0 = E.chunk0.as<int4>();
    P.chunk1 = E.chunk1.as<int4>();
    P.items = E.items.as<int32_t>();
    if (E.compact) {
        P.lists = E.lists.as<int32_t>();
        P.slot_per_vertex = 1;
    }
    Ctl *c = E.ctl.as<Ctl>();
    P.tmp = c->tmp;
    P.cnt = c->cnt;
    P.acc = E.acc.as<unsigned>();
    P.bar = &c->bar;
    P.err = c->err;
    P.passes = c->passes;
    P.graph_last = E.glast.as<int32_t>();
    P.stats = nullptr;
    P.stats_cap = 0;
    P.pass_begin = E.next_pass;
    P.pass_end = E.next_pass + rounds;
    P.cap_is_error = 0;
    P.spin_ns = s->cfg.spin_limit_ns > 0 ? s->cfg.spin_limit_ns : 1000000000LL;
    P.T1 = kT1;
    P.CH = kCH;
    return P;
}

// Reserve pool space for r; false (nothing reserved) if it does not fit now.  Vertices, entries and
// row offsets need contiguous ranges; work-item capacity is a plain budget (slots and work items
// of a round are numbered afresh every round).
bool reserve(Engine &E, Request *r) {
    if (E.free_slots.empty()) return false;
    if (E.used_items + r->n_large > E.PI || E.used_chunks + r->n_chunks > E.PC) return false;
    int64_t vb, eb, rb;
    if (!E.va.alloc(r->n, &vb)) return false;
    if (!E.ea.alloc(r->m, &eb)) {
        E.va.release(vb, r->n);
        return false;
    }
    if (!E.ra.alloc(r->n + 1, &rb)) {
        E.va.release(vb, r->n);
        E.ea.release(eb, r->m);
        return false;
    }
    r->vbase = vb;
    r->ebase = eb;
    r->rbase = rb;
    E.used_items += r->n_large;
    E.used_chunks += r->n_chunks;
    r->slot = E.free_slots.back();
    E.free_slots.pop_back();
    return true;
}

void unreserve(Engine &E, Request *r) {
    E.va.release(r->vbase, r->n);
    E.ea.release(r->ebase, r->m);
    E.ra.release(r->rbase, r->n + 1);
    E.used_items -= r->n_large;
    E.used_chunks -= r->n_chunks;
    E.free_slots.push_back(r->slot);
    r->slot = -1;
}

// Copies admitted requests into the pool, checks their graph format on the device (each request
// has its own error slot, so a malformed request cannot disturb the batch) and appends the valid
// ones to the worklist of round next_pass.  Malformed requests are returned in `bad`.
int admit(gc_server *s, Engine &E, const std::vector<Request *> &adm, std::vector<Request *> &bad) {
    if (adm.empty()) return GC_OK;
    cudaStream_t st = s->stream;
    int32_t *verr = E.verr.as<int32_t>();
    for (Request *r : adm) {
        const int g = r->slot;
        if (!r->staged) {
            SRV_CUDA(cudaMemcpyAsync(E.rowptr.as<int32_t>() + r->rbase, r->rowptr.data(), 4 * (r->n + 1),
                                     cudaMemcpyHostToDevice, st));
            if (r->m)
                SRV_CUDA(cudaMemcpyAsync(E.colidx.as<int32_t>() + r->ebase, r->colidx.data(), 4 * r->m,
                                         cudaMemcpyHostToDevice, st));
        }
        SRV_CUDA(cudaMemsetAsync(verr + 4 * g, 0, 16, st));
        SRV_CUDA(launch_validate(r->n, E.rowptr.as<int32_t>() + r->rbase,
                                 r->m ? E.colidx.as<int32_t>() + r->ebase : E.rowptr.as<int32_t>() + r->rbase, 0,
                                 verr + 4 * g, st));
    }
    std::vector<int32_t> herr(adm.size());
    for (size_t i = 0; i < adm.size(); ++i)
        SRV_CUDA(cudaMemcpyAsync(&herr[i], verr + 4 * adm[i]->slot, 4, cudaMemcpyDeviceToHost, st));
    SRV_CUDA(cudaStreamSynchronize(st));
    std::vector<Request *> ok;
    for (size_t i = 0; i < adm.size(); ++i) {
        Request *r = adm[i];
        std::vector<int32_t>().swap(r->rowptr);  // the pool holds the graph now
        std::vector<int32_t>().swap(r->colidx);
        if (herr[i] != 0) {
            bad.push_back(r);
            continue;
        }
        ok.push_back(r);
        const int g = r->slot;
        E.h_vbase[g] = r->vbase;
        E.h_n[g] = r->n;
        E.h_ebase[g] = r->ebase;
        E.h_rbase[g] = r->rbase;
        E.h_m[g] = r->m;
        E.h_seed[g] = r->seed;
        E.h_glast[g] = E.next_pass - 1;  // raised to next_pass by setup if any vertex has a neighbour
        SRV_CUDA(cudaMemcpyAsync(E.g_vbase.as<int64_t>() + g, &E.h_vbase[g], 8, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(E.g_n.as<int32_t>() + g, &E.h_n[g], 4, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(E.g_ebase.as<int64_t>() + g, &E.h_ebase[g], 8, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(E.g_rbase.as<int64_t>() + g, &E.h_rbase[g], 8, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(E.g_m.as<int64_t>() + g, &E.h_m[g], 8, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(E.gseed.as<uint64_t>() + g, &E.h_seed[g], 8, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(E.glast.as<int32_t>() + g, &E.h_glast[g], 4, cudaMemcpyHostToDevice, st));
        r->join = E.next_pass;
    }
    if (ok.empty()) return GC_OK;
    RoundParams P = params(s, E);
    SRV_CUDA(cudaMemsetAsync(P.tmp, 0, 2 * sizeof(unsigned), st));
    for (Request *r : ok)
        SRV_CUDA(launch_setup(P, E.mode, true, static_cast<int32_t>(r->vbase), static_cast<int32_t>(r->vbase + r->n),
                              r->slot, st));
    SRV_CUDA(launch_expand(P, E.mode, true, E.compact, -1, st));
    return GC_OK;
}

// Colors, color count and rounds of finished requests; frees their pool space.
int retire(gc_server *s, Engine &E, const std::vector<Request *> &fin) {
    if (fin.empty()) return GC_OK;
    cudaStream_t st = s->stream;
    RoundParams P = params(s, E);
    std::vector<int32_t> sel(fin.size());
    for (size_t i = 0; i < fin.size(); ++i) {
        Request *r = fin[i];
        const int g = r->slot;
        // bits [vbase, vbase + n) of the bitmap hold this request's colors
        const int64_t w0 = r->vbase >> 5, w1 = (r->vbase + r->n + 31) >> 5;
        SRV_CUDA(cudaMemsetAsync(E.bitmap.as<unsigned>() + w0, 0, 4 * (w1 - w0 + 1), st));
        SRV_CUDA(cudaMemsetAsync(E.gmax.as<int32_t>() + g, 0xff, 4, st));
        SRV_CUDA(launch_count_colors(P, true, E.mode == GC_MODE_DETERMINISTIC ? E.glast.as<int32_t>() + g : nullptr,
                                     static_cast<int32_t>(r->vbase), static_cast<int32_t>(r->vbase + r->n), g, g + 1,
                                     E.bitmap.as<unsigned>(), E.gmax.as<int32_t>(), E.gcount.as<int32_t>(),
                                     E.outbuf.as<int32_t>() + r->vbase, st));
        r->colors.resize(r->n);
        if (r->n)
            SRV_CUDA(cudaMemcpyAsync(r->colors.data(), E.outbuf.as<int32_t>() + r->vbase, 4 * r->n,
                                     cudaMemcpyDeviceToHost, st));
        SRV_CUDA(cudaMemcpyAsync(&sel[i], E.gcount.as<int32_t>() + g, 4, cudaMemcpyDeviceToHost, st));
    }
    SRV_CUDA(cudaStreamSynchronize(st));
    const double t = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < fin.size(); ++i) {
        Request *r = fin[i];
        r->ncolors = r->n ? sel[i] : 0;
        const int32_t last = E.h_glast[r->slot];
        r->rounds = r->n ? std::max(1, last - r->join + 1) : 0;
        r->state = kDone;
        r->t_done = t;
        s->completed += 1;
        s->v_done += r->n;
        s->e_done += r->m / 2;
        s->latencies.push_back((r->t_done - r->t_submit) * 1e3);
        unreserve(E, r);
    }
    s->cv_done.notify_all();
    return GC_OK;
}

// A launch posted an error (a grid-barrier wait ran out, a malformed entry): the requests resident
// in this pool end with that status, the pool's control block and round count start over, and the
// queued requests stay queued.
int engine_reset(gc_server *s, Engine &E, int code) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const double t = now_s();
        for (Request *r : E.resident) {
            r->state = kDone;
            r->status = code;
            r->t_done = t;
            s->failed += 1;
            unreserve(E, r);
        }
        E.resident.clear();
        s->cv_done.notify_all();
    }
    SRV_CUDA(cudaMemsetAsync(E.ctl.p, 0, sizeof(Ctl), s->stream));
    SRV_CUDA(cudaStreamSynchronize(s->stream));
    E.next_pass = 1;
    return GC_OK;
}

void fail_all(gc_server *s, int code, const std::string &msg) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = code;
    s->fatal_msg = msg;
    for (Engine &E : s->eng) {
        for (auto *list : {&E.resident, &E.staged}) {
            for (Request *r : *list) {
                r->state = kDone;
                r->status = code;
            }
            list->clear();
        }
        for (Request *r : E.queue) {
            r->state = kDone;
            r->status = code;
        }
        E.queue.clear();
    }
    for (Request *r : s->solo) {
        if (r->dbuf) cudaFree(r->dbuf);
        r->dbuf = nullptr;
        r->state = kDone;
        r->status = code;
    }
    s->solo.clear();
    s->cv_done.notify_all();
}

// One pass of the worker over a pool: admission, a launch of a few rounds, retirement.  Returns
// false after an error the server cannot recover from (a failed CUDA call).
bool engine_step(gc_server *s, Engine &E, std::vector<Request *> &adm, bool queued) {
    const double t0 = now_s();
    std::vector<Request *> bad;
    if (admit(s, E, adm, bad) != GC_OK) return false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Request *r : bad) {
            E.resident.erase(std::find(E.resident.begin(), E.resident.end(), r));
            unreserve(E, r);
            r->status = GC_ERR_INVALID_GRAPH;
            r->state = kDone;
            s->rejected += 1;
        }
        if (!bad.empty()) s->cv_done.notify_all();
        if (E.resident.empty()) return true;
    }
    RoundParams P = params(s, E, queued ? kRoundsWhileQueued : kRoundsIdleQueue);
    cudaError_t e = launch_rounds(P, E.mode, true, E.compact, E.grid, 256, s->stream);
    Ctl h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, E.ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E.h_glast.data(), E.glast.p, 4 * E.S, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        srv_fail(s, GC_ERR_CUDA, "server round launch", e);
        return false;
    }
    if (h.err[0] != 0) {
        // the launch reported an error: fail what is resident in this pool, keep serving
        if (engine_reset(s, E, h.err[0]) != GC_OK) return false;
        s->busy += now_s() - t0;
        return true;
    }
    const int32_t ran = h.passes[0] - E.next_pass;
    E.next_pass = h.passes[0];
    std::vector<Request *> fin;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->rounds_run += ran;
        for (auto it = E.resident.begin(); it != E.resident.end();) {
            if (E.h_glast[(*it)->slot] < E.next_pass) {
                fin.push_back(*it);
                it = E.resident.erase(it);
            } else {
                ++it;
            }
        }
    }
    if (retire(s, E, fin) != GC_OK) return false;
    s->busy += now_s() - t0;
    return true;
}

// A request that fills the GPU by itself, colored alone as gc_color_ex colors it (core and tail
// phases included) on the server's stream, between launches of the batch.
// Its CSR waits on the device (copied at submit).
void color_solo(gc_server *s, Request *r) {
    gc_options o{};
    o.stream = s->stream;
    o.spin_limit_ns = s->cfg.spin_limit_ns;
    r->colors.resize(static_cast<size_t>(r->n));
    int32_t nc = 0, rd = 0;
    int32_t *d_rp = static_cast<int32_t *>(r->dbuf);
    int32_t *d_ci = d_rp + (r->n + 1);
    int32_t *d_col = d_ci + r->m;
    int st = gc_color_ex(r->n, d_rp, r->m ? d_ci : nullptr, r->mode, r->seed, r->n ? d_col : nullptr, &nc, &rd, &o,
                         nullptr);
    cudaError_t e = cudaSuccess;
    if (st == GC_OK && r->n)
        e = cudaMemcpyAsync(r->colors.data(), d_col, 4 * static_cast<size_t>(r->n), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaFreeAsync(r->dbuf, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (st == GC_OK) st = GC_ERR_CUDA;
    }
    r->dbuf = nullptr;
    const double t = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    r->status = st;
    r->ncolors = nc;
    r->rounds = rd;
    r->state = kDone;
    r->t_done = t;
    if (st == GC_OK) {
        s->completed += 1;
        s->v_done += r->n;
        s->e_done += r->m / 2;
        s->latencies.push_back((r->t_done - r->t_submit) * 1e3);
    } else if (st == GC_ERR_INVALID_GRAPH) {
        s->rejected += 1;
    } else {
        s->failed += 1;
    }
    s->cv_done.notify_all();
}

void worker_main(gc_server *s) {
    cudaSetDevice(s->device);
    while (true) {
        std::vector<Request *> adm[2];
        bool active[2] = {false, false}, queued[2] = {false, false};
        Request *solo = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->solo.empty() || s->eng[0].busy() || s->eng[1].busy(); });
            if (s->stop && s->solo.empty() && !s->eng[0].busy() && !s->eng[1].busy()) break;
            if (!s->solo.empty()) {
                solo = s->solo.front();
                s->solo.pop_front();
                solo->state = kResident;
            }
            for (int k = 0; k < 2; ++k) {
                Engine &E = s->eng[k];
                if (!E.busy()) continue;
                for (Request *r : E.staged) {
                    r->state = kResident;
                    adm[k].push_back(r);
                    E.resident.push_back(r);
                }
                E.staged.clear();
                for (auto it = E.queue.begin(); it != E.queue.end();) {
                    if (reserve(E, *it)) {
                        (*it)->state = kResident;
                        adm[k].push_back(*it);
                        E.resident.push_back(*it);
                        it = E.queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                active[k] = !E.resident.empty();
                queued[k] = !E.queue.empty();
            }
        }
        if (solo) {
            const double t0 = now_s();
            color_solo(s, solo);
            s->busy += now_s() - t0;
        }
        bool ok = true;
        for (int k = 0; k < 2 && ok; ++k)
            if (active[k]) ok = engine_step(s, s->eng[k], adm[k], queued[k]);
        if (!ok) {
            fail_all(s, s->fatal, s->fatal_msg);
            break;
        }
    }
}

}  // namespace
}  // namespace gc

using gc::set_last_error;

extern "C" {

int gc_server_create(const gc_server_config *cfg, gc_server **out) {
    if (!cfg || !out) return set_last_error(GC_ERR_INVALID_ARG, "NULL config or output");
    if (cfg->pool_vertices <= 0 || cfg->pool_entries <= 0 || cfg->pool_vertices >= INT32_MAX / 2)
        return set_last_error(GC_ERR_INVALID_ARG, "pool sizes must be positive (vertices < 2^30)");
    if (cfg->mode != GC_MODE_DETERMINISTIC && cfg->mode != GC_MODE_INPLACE)
        return set_last_error(GC_ERR_INVALID_ARG, "unknown mode %d", cfg->mode);
    if (cfg->spin_limit_ns < 0) return set_last_error(GC_ERR_INVALID_ARG, "negative spin_limit_ns");
    int dev = cfg->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return set_last_error(GC_ERR_CUDA, "no usable CUDA device");
    }
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return set_last_error(GC_ERR_CUDA, "cannot use device %d", dev);
    }
    auto s = std::make_unique<gc_server>();
    s->cfg = *cfg;
    s->device = dev;
    s->solo_min = cfg->solo_entries < 0 ? INT64_MAX : (cfg->solo_entries == 0 ? int64_t{1} << 24 : cfg->solo_entries);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        // the device copies of requests colored alone: memory freed by one stays for the next (a pool
        // that grew while the worker's kernels ran would stall the submitting thread)
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&s->solo_pool, &props);
        uint64_t keep = UINT64_MAX;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(s->solo_pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e == cudaSuccess) {
            // reserve the pool's size up front (a pool's worth of entries and vertices): requests
            // submitted together keep their copies alive together, and growing the pool while the
            // worker's kernels run stalls the submitting thread; a reservation that fails is skipped
            void *p = nullptr;
            const size_t want = 4 * static_cast<size_t>(cfg->pool_entries) + 12 * static_cast<size_t>(cfg->pool_vertices);
            if (cudaMallocFromPoolAsync(&p, want, s->solo_pool, s->copy_stream) == cudaSuccess) {
                cudaFreeAsync(p, s->copy_stream);
                cudaStreamSynchronize(s->copy_stream);
            }
            cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_last_error(GC_ERR_CUDA, "server streams: %s", cudaGetErrorString(e));
    }
    gc::Engine &E0 = s->eng[gc::engine_index(cfg->mode)];
    const int st = gc::engine_create(s.get(), E0, cfg->mode);
    E0.mode = cfg->mode;  // the worker thread does not exist yet
    if (st != GC_OK) {
        cudaStreamDestroy(s->stream);
        cudaStreamDestroy(s->copy_stream);
        cudaMemPoolDestroy(s->solo_pool);
        return st;
    }
    s->t_create = gc::now_s();
    gc_server *raw = s.release();
    raw->worker = std::thread(gc::worker_main, raw);
    *out = raw;
    return GC_OK;
}

int gc_server_submit(gc_server *s, int32_t n, const int32_t *rowptr, const int32_t *colidx, int mode, uint64_t seed,
                     uint64_t *req_id) {
    if (!s || !req_id) return set_last_error(GC_ERR_INVALID_ARG, "NULL server or request id");
    if (mode != GC_MODE_DETERMINISTIC && mode != GC_MODE_INPLACE)
        return set_last_error(GC_ERR_INVALID_ARG, "unknown mode %d (the server runs the deterministic and in-place "
                                                  "modes)", mode);
    if (n < 0 || (n > 0 && !rowptr)) return set_last_error(GC_ERR_INVALID_ARG, "bad n or NULL rowptr");
    gc::Engine &E = s->eng[gc::engine_index(mode)];
    {
        // the first request of a mode allocates that mode's pool
        std::lock_guard<std::mutex> ck(s->create_mu);
        bool created;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            created = E.mode >= 0;
        }
        if (!created) {
            // the worker ignores this pool until its mode is published under the server lock
            cudaSetDevice(s->device);
            const int st = gc::engine_create(s, E, mode);
            if (st != GC_OK) return st;
            std::lock_guard<std::mutex> lk(s->mu);
            E.mode = mode;
        }
    }
    auto r = std::make_unique<gc::Request>();
    r->n = n;
    r->mode = mode;
    r->seed = seed;
    r->eng = &E;
    r->rowptr.resize(static_cast<size_t>(n) + 1);
    cudaPointerAttributes a{};
    const bool rp_dev = cudaPointerGetAttributes(&a, rowptr) == cudaSuccess &&
                        (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (rp_dev) {
        if (cudaMemcpy(r->rowptr.data(), rowptr, 4 * (static_cast<size_t>(n) + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
            return set_last_error(GC_ERR_CUDA, "copying rowptr");
    } else if (n >= 0) {
        std::memcpy(r->rowptr.data(), rowptr ? rowptr : r->rowptr.data(), 4 * (static_cast<size_t>(n) + 1));
    }
    if (n == 0) r->rowptr[0] = 0;
    const int64_t m = r->rowptr[n];
    if (r->rowptr[0] != 0 || m < 0) return set_last_error(GC_ERR_INVALID_GRAPH, "rowptr must start at 0");
    if (m > 0 && !colidx) return set_last_error(GC_ERR_INVALID_ARG, "NULL colidx");
    r->m = m;
    // row offsets are checked here (they size the request's footprint); neighbour ids and self-loops
    // are checked on the device when the request is admitted
    for (int32_t v = 0; v < n; ++v) {
        const int64_t b = r->rowptr[v], e = r->rowptr[v + 1];
        if (e < b || e > m) return set_last_error(GC_ERR_INVALID_GRAPH, "rowptr not monotone at vertex %d", v);
        const int64_t d = e - b;
        if (d > gc::kT1) {
            r->n_large += 1;
            r->n_chunks += (d + gc::kCH - 1) / gc::kCH;
        }
    }
    const bool ci_dev = m > 0 && cudaPointerGetAttributes(&a, colidx) == cudaSuccess &&
                        (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    gc::Request *raw = r.get();
    const bool solo = m >= s->solo_min;  // fills the GPU by itself: colored alone
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal != GC_OK) return set_last_error(s->fatal, "server stopped: %s", s->fatal_msg.c_str());
        if (!solo && (n > E.va.capacity() || m > E.ea.capacity() || r->n_large > E.PI || r->n_chunks > E.PC)) {
            s->rejected += 1;
            return set_last_error(GC_ERR_OOM, "request (n=%d, nnz=%lld) exceeds the server pool", n,
                                  static_cast<long long>(m));
        }
        r->id = s->next_id++;
        r->t_submit = gc::now_s();
        *req_id = r->id;
        // with nothing queued ahead and room in the pool, the CSR goes straight into the pool (a
        // request colored alone never enters the pool)
        raw->staged = !solo && E.queue.empty() && gc::reserve(E, raw);
        s->reqs[raw->id] = std::move(r);
        s->submitted += 1;
    }
    cudaError_t e = cudaSuccess;
    if (solo) {
        // colored alone: its CSR goes to the device now (stream-ordered allocation) and waits there
        std::lock_guard<std::mutex> ck(s->copy_mu);
        const size_t bytes = 4 * (static_cast<size_t>(n) + 1) + 4 * static_cast<size_t>(m) + 4 * static_cast<size_t>(n);
        e = cudaMallocFromPoolAsync(&raw->dbuf, bytes, s->solo_pool, s->copy_stream);
        int32_t *d_rp = static_cast<int32_t *>(raw->dbuf);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_rp, raw->rowptr.data(), 4 * (static_cast<size_t>(n) + 1), cudaMemcpyHostToDevice,
                                s->copy_stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_rp + (n + 1), colidx, 4 * static_cast<size_t>(m),
                                ci_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->copy_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
        if (e != cudaSuccess && raw->dbuf) {
            cudaFreeAsync(raw->dbuf, s->copy_stream);
            cudaStreamSynchronize(s->copy_stream);
            raw->dbuf = nullptr;
        }
        std::vector<int32_t>().swap(raw->rowptr);
    } else if (raw->staged) {
        std::lock_guard<std::mutex> ck(s->copy_mu);
        e = cudaMemcpyAsync(E.rowptr.as<int32_t>() + raw->rbase, raw->rowptr.data(), 4 * (static_cast<size_t>(n) + 1),
                            cudaMemcpyHostToDevice, s->copy_stream);
        if (e == cudaSuccess && m)
            e = cudaMemcpyAsync(E.colidx.as<int32_t>() + raw->ebase, colidx, 4 * static_cast<size_t>(m),
                                ci_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->copy_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
        std::vector<int32_t>().swap(raw->rowptr);
    } else if (m) {
        raw->colidx.resize(static_cast<size_t>(m));
        if (ci_dev)
            e = cudaMemcpy(raw->colidx.data(), colidx, 4 * static_cast<size_t>(m), cudaMemcpyDeviceToHost);
        else
            std::memcpy(raw->colidx.data(), colidx, 4 * static_cast<size_t>(m));
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (raw->staged) gc::unreserve(E, raw);
        raw->state = gc::kDone;
        raw->status = e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA;
        return set_last_error(raw->status, "copying the request: %s", cudaGetErrorString(e));
    }
    if (raw->staged)
        E.staged.push_back(raw);
    else if (solo)
        s->solo.push_back(raw);
    else
        E.queue.push_back(raw);
    s->cv_work.notify_one();
    return GC_OK;
}

int gc_server_poll(gc_server *s, uint64_t req_id, int32_t timeout_ms, int32_t *colors_out, int32_t *ncolors,
                   int32_t *rounds) {
    if (!s) return set_last_error(GC_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return set_last_error(GC_ERR_INVALID_ARG, "unknown request %llu",
                                                   static_cast<unsigned long long>(req_id));
    gc::Request *r = it->second.get();
    auto done = [&] { return r->state == gc::kDone; };
    if (!done()) {
        if (timeout_ms < 0)
            s->cv_done.wait(lk, done);
        else if (timeout_ms > 0)
            s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
    }
    if (!done()) return set_last_error(GC_ERR_BUSY, "request %llu still running", static_cast<unsigned long long>(req_id));
    const int status = r->status;
    std::unique_ptr<gc::Request> keep = std::move(it->second);
    s->reqs.erase(it);
    const std::string fatal_msg = s->fatal_msg;
    lk.unlock();
    if (status == GC_ERR_INVALID_GRAPH)
        return set_last_error(status, "request %llu: invalid graph (neighbour id out of range or self-loop)",
                              static_cast<unsigned long long>(req_id));
    if (status == GC_ERR_TIMEOUT)
        return set_last_error(status, "request %llu: a grid-barrier wait of its launch exceeded the limit",
                              static_cast<unsigned long long>(req_id));
    if (status != GC_OK)
        return set_last_error(status, "request %llu failed (status %d)%s%s", static_cast<unsigned long long>(req_id),
                              status, fatal_msg.empty() ? "" : ": ", fatal_msg.c_str());
    if (colors_out && keep->n) {
        cudaPointerAttributes a{};
        const bool dev = cudaPointerGetAttributes(&a, colors_out) == cudaSuccess &&
                         (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        if (dev) {
            if (cudaMemcpy(colors_out, keep->colors.data(), 4 * static_cast<size_t>(keep->n), cudaMemcpyHostToDevice) !=
                cudaSuccess)
                return set_last_error(GC_ERR_CUDA, "copying colors");
        } else {
            std::memcpy(colors_out, keep->colors.data(), 4 * static_cast<size_t>(keep->n));
        }
    }
    if (ncolors) *ncolors = keep->ncolors;
    if (rounds) *rounds = keep->rounds;
    return GC_OK;
}

int gc_server_stats(gc_server *s, struct gc_server_stats *out) {
    if (!s || !out) return set_last_error(GC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->failed = s->failed;
    out->rounds_run = s->rounds_run;
    out->vertices_colored = s->v_done;
    out->edges_colored = s->e_done;
    if (!s->latencies.empty()) {
        std::vector<double> l = s->latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) { return l[std::min(l.size() - 1, static_cast<size_t>(q * (l.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
    }
    out->busy_s = s->busy;
    out->wall_s = gc::now_s() - s->t_create;
    for (const gc::Engine &E : s->eng) {
        out->resident += static_cast<int32_t>(E.resident.size());
        out->queued += static_cast<int32_t>(E.queue.size());
    }
    out->queued += static_cast<int32_t>(s->solo.size());
    return GC_OK;
}

int gc_server_stats_get(gc_server *s, struct gc_server_stats *out) { return gc_server_stats(s, out); }

void gc_server_destroy(gc_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    if (s->solo_pool) cudaMemPoolDestroy(s->solo_pool);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    delete s;
}

}  // extern "C"
