// Continuous-batching coloring server (gc_server_* in include/gc.h).
//
// A worker thread owns a resident device pool (CSR storage, color/priority/worklist state) and
// runs the batched round kernel a few rounds per launch over every resident request.  Between
// launches it (1) retires requests none of whose vertices is on the next round's worklist,
// (2) admits queued requests whose footprint fits the free pool space (first fit over vertex,
// entry and work-item ranges), joining them to the running batch at the next round: their first
// round is the batch's next round, and a request's own round count is measured from there.
// Because every graph's deterministic rounds read only its own previous colors, a request's
// colors do not depend on which other requests share the launch.
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

struct Request {
    uint64_t id = 0;
    int32_t n = 0;
    int64_t m = 0;
    int64_t n_large = 0, n_chunks = 0;
    std::vector<int32_t> rowptr, colidx, colors;
    ReqState state = kQueued;
    int status = GC_OK;
    int32_t ncolors = 0, rounds = 0;
    double t_submit = 0, t_done = 0;
    int32_t slot = -1, join = 0;
    int64_t vbase = 0, ebase = 0, rbase = 0;
    bool staged = false;  // its CSR was copied into the pool at submit
};

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
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

}  // namespace
}  // namespace gc

struct gc_server {
    gc_server_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    int grid = 0;
    int64_t PV = 0, PE = 0, PI = 0, PC = 0;  // pool capacities: vertices, entries, large vertices, work items
    int32_t S = 0;                           // slots
    bool compact = false;  // deterministic mode: the compact sweep (slot and list space per pool vertex / entry)
    gc::DevBuf rowptr, colidx, col0, col1, outbuf, small0, small1, items, chunk0, chunk1, acc, lists, vg, ctl, bitmap;
    gc::DevBuf g_vbase, g_n, g_ebase, g_rbase, g_m, glast, gmax, gcount, verr;
    std::vector<int64_t> h_vbase, h_ebase, h_rbase, h_m;
    std::vector<int32_t> h_n, h_glast;
    gc::RangeAlloc va, ea, ra;
    int64_t used_items = 0, used_chunks = 0;
    std::vector<int32_t> free_slots;
    std::vector<gc::Request *> resident;
    std::deque<gc::Request *> queue;
    std::vector<gc::Request *> staged;  // pool space reserved and CSR copied at submit
    std::mutex copy_mu;
    cudaStream_t copy_stream = nullptr;
    std::unordered_map<uint64_t, std::unique_ptr<gc::Request>> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    int32_t next_pass = 1;
    // statistics
    int64_t submitted = 0, completed = 0, rejected = 0, rounds_run = 0, v_done = 0, e_done = 0;
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

RoundParams params(gc_server *s, int32_t rounds = kRoundsWhileQueued) {
    RoundParams P{};
    P.n = static_cast<int32_t>(s->PV);
    P.G = s->S;
    P.rowptr = s->rowptr.as<int32_t>();
    P.colidx = s->colidx.as<int32_t>();
    P.g_vbase = s->g_vbase.as<int64_t>();
    P.g_n = s->g_n.as<int32_t>();
    P.g_ebase = s->g_ebase.as<int64_t>();
    P.g_rbase = s->g_rbase.as<int64_t>();
    P.g_m = s->g_m.as<int64_t>();
    P.vg = s->vg.as<int32_t>();
    P.seed = s->cfg.seed;
    P.col0 = s->col0.as<uint64_t>();
    P.col1 = s->col1.as<uint64_t>();
    P.small0 = s->small0.as<int32_t>();
    P.small1 = s->small1.as<int32_t>();
    P.chunk0 = s->chunk0.as<int4>();
    P.chunk1 = s->chunk1.as<int4>();
    P.items = s->items.as<int32_t>();
    if (s->compact) {
        P.lists = s->lists.as<int32_t>();
        P.slot_per_vertex = 1;
    }
    Ctl *c = s->ctl.as<Ctl>();
    P.tmp = c->tmp;
    P.cnt = c->cnt;
    P.acc = s->acc.as<unsigned>();
    P.bar = &c->bar;
    P.err = c->err;
    P.passes = c->passes;
    P.graph_last = s->glast.as<int32_t>();
    P.stats = nullptr;
    P.stats_cap = 0;
    P.pass_begin = s->next_pass;
    P.pass_end = s->next_pass + rounds;
    P.cap_is_error = 0;
    P.spin_ns = 1000000000LL;
    P.T1 = kT1;
    P.CH = kCH;
    return P;
}

// Reserve pool space for r; false (nothing reserved) if it does not fit now.  Vertices, entries and
// row offsets need contiguous ranges; work-item capacity is a plain budget (slots and work items
// of a round are numbered afresh every round).
bool reserve(gc_server *s, Request *r) {
    if (s->free_slots.empty()) return false;
    if (s->used_items + r->n_large > s->PI || s->used_chunks + r->n_chunks > s->PC) return false;
    int64_t vb, eb, rb;
    if (!s->va.alloc(r->n, &vb)) return false;
    if (!s->ea.alloc(r->m, &eb)) {
        s->va.release(vb, r->n);
        return false;
    }
    if (!s->ra.alloc(r->n + 1, &rb)) {
        s->va.release(vb, r->n);
        s->ea.release(eb, r->m);
        return false;
    }
    r->vbase = vb;
    r->ebase = eb;
    r->rbase = rb;
    s->used_items += r->n_large;
    s->used_chunks += r->n_chunks;
    r->slot = s->free_slots.back();
    s->free_slots.pop_back();
    return true;
}

void unreserve(gc_server *s, Request *r) {
    s->va.release(r->vbase, r->n);
    s->ea.release(r->ebase, r->m);
    s->ra.release(r->rbase, r->n + 1);
    s->used_items -= r->n_large;
    s->used_chunks -= r->n_chunks;
    s->free_slots.push_back(r->slot);
    r->slot = -1;
}

// Copies admitted requests into the pool, checks their graph format on the device (each request
// has its own error slot, so a malformed request cannot disturb the batch) and appends the valid
// ones to the worklist of round next_pass.  Malformed requests are returned in `bad`.
int admit(gc_server *s, const std::vector<Request *> &adm, std::vector<Request *> &bad) {
    if (adm.empty()) return GC_OK;
    cudaStream_t st = s->stream;
    int32_t *verr = s->verr.as<int32_t>();
    for (Request *r : adm) {
        const int g = r->slot;
        if (!r->staged) {
            SRV_CUDA(cudaMemcpyAsync(s->rowptr.as<int32_t>() + r->rbase, r->rowptr.data(), 4 * (r->n + 1),
                                     cudaMemcpyHostToDevice, st));
            if (r->m)
                SRV_CUDA(cudaMemcpyAsync(s->colidx.as<int32_t>() + r->ebase, r->colidx.data(), 4 * r->m,
                                         cudaMemcpyHostToDevice, st));
        }
        SRV_CUDA(cudaMemsetAsync(verr + 4 * g, 0, 16, st));
        SRV_CUDA(launch_validate(r->n, s->rowptr.as<int32_t>() + r->rbase,
                                 r->m ? s->colidx.as<int32_t>() + r->ebase : s->rowptr.as<int32_t>() + r->rbase, 0,
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
        s->h_vbase[g] = r->vbase;
        s->h_n[g] = r->n;
        s->h_ebase[g] = r->ebase;
        s->h_rbase[g] = r->rbase;
        s->h_m[g] = r->m;
        s->h_glast[g] = s->next_pass - 1;  // raised to next_pass by setup if any vertex has a neighbour
        SRV_CUDA(cudaMemcpyAsync(s->g_vbase.as<int64_t>() + g, &s->h_vbase[g], 8, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(s->g_n.as<int32_t>() + g, &s->h_n[g], 4, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(s->g_ebase.as<int64_t>() + g, &s->h_ebase[g], 8, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(s->g_rbase.as<int64_t>() + g, &s->h_rbase[g], 8, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(s->g_m.as<int64_t>() + g, &s->h_m[g], 8, cudaMemcpyHostToDevice, st));
        SRV_CUDA(cudaMemcpyAsync(s->glast.as<int32_t>() + g, &s->h_glast[g], 4, cudaMemcpyHostToDevice, st));
        r->join = s->next_pass;
    }
    if (ok.empty()) return GC_OK;
    RoundParams P = params(s);
    SRV_CUDA(cudaMemsetAsync(P.tmp, 0, 2 * sizeof(unsigned), st));
    for (Request *r : ok)
        SRV_CUDA(launch_setup(P, s->cfg.mode, true, static_cast<int32_t>(r->vbase),
                              static_cast<int32_t>(r->vbase + r->n), r->slot, st));
    SRV_CUDA(launch_expand(P, s->cfg.mode, true, s->compact, -1, st));
    return GC_OK;
}

// Colors, color count and rounds of finished requests; frees their pool space.
int retire(gc_server *s, const std::vector<Request *> &fin) {
    if (fin.empty()) return GC_OK;
    cudaStream_t st = s->stream;
    RoundParams P = params(s);
    std::vector<int32_t> sel(fin.size());
    for (size_t i = 0; i < fin.size(); ++i) {
        Request *r = fin[i];
        const int g = r->slot;
        // bits [vbase, vbase + n) of the bitmap hold this request's colors
        const int64_t w0 = r->vbase >> 5, w1 = (r->vbase + r->n + 31) >> 5;
        SRV_CUDA(cudaMemsetAsync(s->bitmap.as<unsigned>() + w0, 0, 4 * (w1 - w0 + 1), st));
        SRV_CUDA(cudaMemsetAsync(s->gmax.as<int32_t>() + g, 0xff, 4, st));
        SRV_CUDA(launch_count_colors(P, true, s->cfg.mode == GC_MODE_DETERMINISTIC ? s->glast.as<int32_t>() + g : nullptr,
                                     static_cast<int32_t>(r->vbase), static_cast<int32_t>(r->vbase + r->n), g, g + 1,
                                     s->bitmap.as<unsigned>(), s->gmax.as<int32_t>(), s->gcount.as<int32_t>(),
                                     s->outbuf.as<int32_t>() + r->vbase, st));
        r->colors.resize(r->n);
        if (r->n)
            SRV_CUDA(cudaMemcpyAsync(r->colors.data(), s->outbuf.as<int32_t>() + r->vbase, 4 * r->n,
                                     cudaMemcpyDeviceToHost, st));
        SRV_CUDA(cudaMemcpyAsync(&sel[i], s->gcount.as<int32_t>() + g, 4, cudaMemcpyDeviceToHost, st));
    }
    SRV_CUDA(cudaStreamSynchronize(st));
    const double t = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < fin.size(); ++i) {
        Request *r = fin[i];
        r->ncolors = r->n ? sel[i] : 0;
        const int32_t last = s->h_glast[r->slot];
        r->rounds = r->n ? std::max(1, last - r->join + 1) : 0;
        r->state = kDone;
        r->t_done = t;
        s->completed += 1;
        s->v_done += r->n;
        s->e_done += r->m / 2;
        s->latencies.push_back((r->t_done - r->t_submit) * 1e3);
        unreserve(s, r);
    }
    s->cv_done.notify_all();
    return GC_OK;
}

void fail_all(gc_server *s, int code, const std::string &msg) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = code;
    s->fatal_msg = msg;
    for (Request *r : s->resident) {
        r->state = kDone;
        r->status = code;
    }
    s->resident.clear();
    for (Request *r : s->queue) {
        r->state = kDone;
        r->status = code;
    }
    s->queue.clear();
    for (Request *r : s->staged) {
        r->state = kDone;
        r->status = code;
    }
    s->staged.clear();
    s->cv_done.notify_all();
}

void worker_main(gc_server *s) {
    cudaSetDevice(s->device);
    while (true) {
        std::vector<Request *> adm;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                return s->stop || !s->queue.empty() || !s->resident.empty() || !s->staged.empty();
            });
            if (s->stop && s->queue.empty() && s->resident.empty() && s->staged.empty()) break;
            for (Request *r : s->staged) {
                r->state = kResident;
                adm.push_back(r);
                s->resident.push_back(r);
            }
            s->staged.clear();
            for (auto it = s->queue.begin(); it != s->queue.end();) {
                if (reserve(s, *it)) {
                    (*it)->state = kResident;
                    adm.push_back(*it);
                    s->resident.push_back(*it);
                    it = s->queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        const double t0 = now_s();
        std::vector<Request *> bad;
        if (admit(s, adm, bad) != GC_OK) {
            fail_all(s, s->fatal, s->fatal_msg);
            break;
        }
        bool queued = false;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (Request *r : bad) {
                s->resident.erase(std::find(s->resident.begin(), s->resident.end(), r));
                unreserve(s, r);
                r->status = GC_ERR_INVALID_GRAPH;
                r->state = kDone;
                s->rejected += 1;
            }
            if (!bad.empty()) s->cv_done.notify_all();
            queued = !s->queue.empty();
            if (s->resident.empty()) continue;
        }
        RoundParams P = params(s, queued ? kRoundsWhileQueued : kRoundsIdleQueue);
        cudaError_t e = launch_rounds(P, s->cfg.mode, true, s->compact, s->grid, 256, s->stream);
        Ctl h{};
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, s->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->h_glast.data(), s->glast.p, 4 * s->S, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) {
            fail_all(s, GC_ERR_CUDA, std::string("server round launch: ") + cudaGetErrorString(e));
            break;
        }
        if (h.err[0] != 0) {
            fail_all(s, h.err[0], "device error in the batched round kernel");
            break;
        }
        const int32_t ran = h.passes[0] - s->next_pass;
        s->next_pass = h.passes[0];
        std::vector<Request *> fin;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->rounds_run += ran;
            for (auto it = s->resident.begin(); it != s->resident.end();) {
                if (s->h_glast[(*it)->slot] < s->next_pass) {
                    fin.push_back(*it);
                    it = s->resident.erase(it);
                } else {
                    ++it;
                }
            }
        }
        if (retire(s, fin) != GC_OK) {
            fail_all(s, s->fatal, s->fatal_msg);
            break;
        }
        s->busy += now_s() - t0;
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
    s->S = cfg->max_requests > 0 ? cfg->max_requests : 4096;
    s->PV = cfg->pool_vertices;
    s->PE = cfg->pool_entries;
    s->PI = std::min<int64_t>(s->PV, s->PE / (gc::kT1 + 1) + 1);
    s->PC = s->PE / gc::kCH + s->PI + 1;
    // deterministic mode sweeps compact lists: a slot per pool vertex and two list regions per entry
    s->compact = cfg->mode == GC_MODE_DETERMINISTIC;
    const size_t slots = s->compact ? static_cast<size_t>(s->PV) : static_cast<size_t>(s->PI);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    const size_t V = static_cast<size_t>(s->PV), Sz = static_cast<size_t>(s->S);
    struct {
        gc::DevBuf *b;
        size_t bytes;
    } plan[] = {
        {&s->rowptr, 4 * (V + Sz)}, {&s->colidx, 4 * static_cast<size_t>(s->PE)}, {&s->col0, 8 * V}, {&s->col1, 8 * V},
        {&s->outbuf, 4 * V}, {&s->small0, 4 * V}, {&s->small1, 4 * V}, {&s->items, 4 * V}, {&s->vg, 4 * V},
        {&s->chunk0, gc::kItemBytes * static_cast<size_t>(s->PC)}, {&s->chunk1, gc::kItemBytes * static_cast<size_t>(s->PC)},
        {&s->acc, 4 * gc::kAccStride * slots}, {&s->lists, s->compact ? 8 * static_cast<size_t>(s->PE) : 0},
        {&s->ctl, sizeof(gc::Ctl)},
        {&s->bitmap, 4 * (V / 32 + 4)}, {&s->g_vbase, 8 * Sz}, {&s->g_n, 4 * Sz}, {&s->g_ebase, 8 * Sz},
        {&s->g_rbase, 8 * Sz}, {&s->g_m, 8 * Sz}, {&s->glast, 4 * Sz}, {&s->gmax, 4 * Sz}, {&s->gcount, 4 * Sz},
        {&s->verr, 16 * Sz},
    };
    for (auto &a : plan) {
        if (e != cudaSuccess) break;
        e = a.b->alloc(a.bytes);
    }
    if (e == cudaSuccess) e = cudaMemset(s->ctl.p, 0, sizeof(gc::Ctl));
    if (e == cudaSuccess) e = cudaMemset(s->acc.p, 0, 4 * gc::kAccStride * slots);
    if (e == cudaSuccess) e = cudaMemset(s->g_n.p, 0, 4 * Sz);
    if (e == cudaSuccess) e = cudaMemset(s->glast.p, 0, 4 * Sz);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (s->stream) cudaStreamDestroy(s->stream);
        return set_last_error(e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA, "server pool: %s",
                              cudaGetErrorString(e));
    }
    int per_sm = 0, sms = 0;
    gc::round_kernel_occupancy(cfg->mode, true, s->compact, 256, &per_sm);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s->grid = std::max(1, per_sm * sms);
    s->h_vbase.assign(Sz, 0);
    s->h_ebase.assign(Sz, 0);
    s->h_rbase.assign(Sz, 0);
    s->h_m.assign(Sz, 0);
    s->h_n.assign(Sz, 0);
    s->h_glast.assign(Sz, 0);
    s->va.reset(s->PV);
    s->ea.reset(s->PE);
    s->ra.reset(s->PV + s->S);
    for (int32_t g = s->S - 1; g >= 0; --g) s->free_slots.push_back(g);
    s->t_create = gc::now_s();
    gc_server *raw = s.release();
    raw->worker = std::thread(gc::worker_main, raw);
    *out = raw;
    return GC_OK;
}

int gc_server_submit(gc_server *s, int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t *req_id) {
    if (!s || !req_id) return set_last_error(GC_ERR_INVALID_ARG, "NULL server or request id");
    if (n < 0 || (n > 0 && !rowptr)) return set_last_error(GC_ERR_INVALID_ARG, "bad n or NULL rowptr");
    auto r = std::make_unique<gc::Request>();
    r->n = n;
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
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal != GC_OK) return set_last_error(s->fatal, "server stopped: %s", s->fatal_msg.c_str());
        if (n > s->va.capacity() || m > s->ea.capacity() || r->n_large > s->PI || r->n_chunks > s->PC) {
            s->rejected += 1;
            return set_last_error(GC_ERR_OOM, "request (n=%d, nnz=%lld) exceeds the server pool", n,
                                  static_cast<long long>(m));
        }
        r->id = s->next_id++;
        r->t_submit = gc::now_s();
        *req_id = r->id;
        // with nothing queued ahead and room in the pool, the CSR goes straight into the pool
        raw->staged = s->queue.empty() && gc::reserve(s, raw);
        s->reqs[raw->id] = std::move(r);
        s->submitted += 1;
    }
    cudaError_t e = cudaSuccess;
    if (raw->staged) {
        std::lock_guard<std::mutex> ck(s->copy_mu);
        e = cudaMemcpyAsync(s->rowptr.as<int32_t>() + raw->rbase, raw->rowptr.data(), 4 * (static_cast<size_t>(n) + 1),
                            cudaMemcpyHostToDevice, s->copy_stream);
        if (e == cudaSuccess && m)
            e = cudaMemcpyAsync(s->colidx.as<int32_t>() + raw->ebase, colidx, 4 * static_cast<size_t>(m),
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
        if (raw->staged) gc::unreserve(s, raw);
        raw->state = gc::kDone;
        raw->status = GC_ERR_CUDA;
        return set_last_error(GC_ERR_CUDA, "copying the request: %s", cudaGetErrorString(e));
    }
    if (raw->staged)
        s->staged.push_back(raw);
    else
        s->queue.push_back(raw);
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
    lk.unlock();
    if (status == GC_ERR_INVALID_GRAPH)
        return set_last_error(status, "request %llu: invalid graph (neighbour id out of range or self-loop)",
                              static_cast<unsigned long long>(req_id));
    if (status != GC_OK) return set_last_error(status, "request failed: %s", s->fatal_msg.c_str());
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

int gc_server_stats_get(gc_server *s, gc_server_stats *out) {
    if (!s || !out) return set_last_error(GC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
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
    out->resident = static_cast<int32_t>(s->resident.size());
    out->queued = static_cast<int32_t>(s->queue.size());
    return GC_OK;
}

void gc_server_destroy(gc_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    delete s;
}

}  // extern "C"
