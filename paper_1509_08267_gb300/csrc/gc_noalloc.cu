// gc_color_noalloc: deterministic coloring of one graph without allocating device memory.
//
// Some callers cannot call cudaMalloc: code that runs where allocation is not allowed or not safe
// (inside a custom allocator or a memory-pool callback, under a host framework that owns all device
// memory and forbids side allocations, or in a process that must not grow its footprint after
// start-up).  For them this entry point works entirely in a fixed scratch array that is part of the
// library image: a file-scope __device__ array that every GPU which loads the library holds until the
// process exits.  The caller passes only its own inputs and outputs (device memory).
//
// The kernels are the library's regular ones (setup, work-item expansion, the persistent round
// kernel and color counting); only the placement of their scratch differs from gc_color.
#include <cstring>
#include <mutex>

#include "gc_internal.h"

namespace gc {
namespace {

// Limits of the scratch-free path.
constexpr int32_t kNaMaxVertices = 16384;
constexpr int64_t kNaMaxEntries = int64_t{1} << 20;
constexpr int32_t kNaT1 = 32;     // vertices up to this degree take one thread
constexpr int32_t kNaCH = 1024;   // adjacency entries per warp work item
// A vertex of degree d > T1 has ceil(d / CH) <= d / CH + 1 work items, so all of them together have
// at most nnz / CH + n items; at most n vertices need an accumulator slot.
constexpr int64_t kNaMaxItems = kNaMaxEntries / kNaCH + kNaMaxVertices;

// Control block, laid out like the one gc_color uses (the kernels only see pointers into it).
struct NaCtl {
    int32_t err[4];
    int32_t passes[2];
    int32_t pad0[2];
    unsigned cnt[3 * kCnt];
    unsigned tmp[2];
    int32_t gmax1, gcount1, glast1, pad1;
    int32_t pad2[6];
    GridBar bar;
};
static_assert(offsetof(NaCtl, bar) % 128 == 0, "barrier alignment");

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t{255}; }
constexpr size_t kOffCtl = 0;
constexpr size_t kOffCol0 = align256(kOffCtl + sizeof(NaCtl));
constexpr size_t kOffCol1 = align256(kOffCol0 + 8 * size_t{kNaMaxVertices});
constexpr size_t kOffSmall0 = align256(kOffCol1 + 8 * size_t{kNaMaxVertices});
constexpr size_t kOffSmall1 = align256(kOffSmall0 + 4 * size_t{kNaMaxVertices});
constexpr size_t kOffItems = align256(kOffSmall1 + 4 * size_t{kNaMaxVertices});
constexpr size_t kOffChunk0 = align256(kOffItems + 4 * size_t{kNaMaxVertices});
constexpr size_t kOffChunk1 = align256(kOffChunk0 + kItemBytes * size_t{kNaMaxItems});
constexpr size_t kOffAcc = align256(kOffChunk1 + kItemBytes * size_t{kNaMaxItems});
constexpr size_t kOffBitmap = align256(kOffAcc + 4 * size_t{kAccStride} * size_t{kNaMaxVertices});
constexpr size_t kBitmapWords = kNaMaxVertices / 32 + 2;
constexpr size_t kScratchBytes = align256(kOffBitmap + 4 * kBitmapWords);  // about 5.8 MB

// The scratch itself.  Host code must not use the name as an address: it looks up the device
// address with cudaGetSymbolAddress (once per device, again if that context went away) and hands
// that to the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_na_mu;
void *g_na_base[128];  // device address of the scratch, per device (looked up on first use)

int na_fail(int code, const char *what, cudaError_t e) {
    return set_last_error(code, "%s: %s", what, cudaGetErrorString(e));
}

// Still a device address of the current context?  (After cudaDeviceReset, or under another
// context, a cached address is stale.)  cudaPointerGetAttributes allocates nothing.
bool still_mapped(void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Device address of the scratch on the current device.  The first call on a device looks it up
// with that device current; later calls reuse it after checking that it still belongs to the
// current context, and look it up again if not.
int scratch_base(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (g_na_base[dev] && !still_mapped(g_na_base[dev], dev)) g_na_base[dev] = nullptr;
    if (!g_na_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return na_fail(GC_ERR_CUDA, "cudaGetSymbolAddress(scratch)", e);
        }
        g_na_base[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_na_base[dev]);
    return GC_OK;
}

bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace gc

extern "C" int gc_color_noalloc(int32_t n, const int32_t *rowptr, const int32_t *colidx, uint64_t seed,
                                int32_t *colors_out, int32_t *ncolors, int32_t *rounds, void *stream) {
    using namespace gc;
    if (n < 0) return set_last_error(GC_ERR_INVALID_ARG, "n = %d is negative", n);
    if (n > kNaMaxVertices)
        return set_last_error(GC_ERR_INVALID_ARG, "n = %d exceeds the scratch-free limit of %d vertices", n,
                              kNaMaxVertices);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        cudaGetLastError();
        return set_last_error(GC_ERR_CUDA, "no usable CUDA device");
    }
    if (n == 0) {
        if (ncolors) *ncolors = 0;
        if (rounds) *rounds = 0;
        return GC_OK;
    }
    if (!rowptr || !colors_out || !on_device(rowptr, dev) || !on_device(colors_out, dev))
        return set_last_error(GC_ERR_INVALID_ARG, "rowptr and colors_out must be device memory of the current device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *base = nullptr;
    int st = scratch_base(dev, &base);
    if (st != GC_OK) return st;

    int32_t nnz = 0;
    e = cudaMemcpyAsync(&nnz, rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(GC_ERR_CUDA, "reading rowptr[n]", e);
    if (nnz < 0) return set_last_error(GC_ERR_INVALID_GRAPH, "rowptr[n] = %d is negative", nnz);
    if (nnz > kNaMaxEntries)
        return set_last_error(GC_ERR_INVALID_ARG, "%d adjacency entries exceed the scratch-free limit of %lld", nnz,
                              static_cast<long long>(kNaMaxEntries));
    if (nnz > 0 && (!colidx || !on_device(colidx, dev)))
        return set_last_error(GC_ERR_INVALID_ARG, "colidx must be device memory of the current device");

    NaCtl *ctl = reinterpret_cast<NaCtl *>(base + kOffCtl);
    RoundParams P{};
    P.n = n;
    P.G = 1;
    P.nnz = nnz;
    P.rowptr = rowptr;
    P.colidx = nnz > 0 ? colidx : rowptr;  // never dereferenced when there are no entries
    P.seed = seed;
    P.col0 = reinterpret_cast<uint64_t *>(base + kOffCol0);
    P.col1 = reinterpret_cast<uint64_t *>(base + kOffCol1);
    P.small0 = reinterpret_cast<int32_t *>(base + kOffSmall0);
    P.small1 = reinterpret_cast<int32_t *>(base + kOffSmall1);
    P.items = reinterpret_cast<int32_t *>(base + kOffItems);
    P.chunk0 = reinterpret_cast<int4 *>(base + kOffChunk0);
    P.chunk1 = reinterpret_cast<int4 *>(base + kOffChunk1);
    P.acc = reinterpret_cast<unsigned *>(base + kOffAcc);
    P.tmp = ctl->tmp;
    P.cnt = ctl->cnt;
    P.bar = &ctl->bar;
    P.err = ctl->err;
    P.passes = ctl->passes;
    P.graph_last = &ctl->glast1;
    P.pass_begin = 1;
    P.pass_end = n + 2;  // a worklist shrinks every round, so n + 1 rounds always suffice
    P.cap_is_error = 1;
    P.spin_ns = 1000000000LL;
    P.T1 = kNaT1;
    P.CH = kNaCH;

    // every call starts from a cleared control block and color bitmap (the array keeps the last
    // call's contents)
    unsigned *bitmap = reinterpret_cast<unsigned *>(base + kOffBitmap);
    e = cudaMemsetAsync(ctl, 0, sizeof(NaCtl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&ctl->gmax1, 0xff, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bitmap, 0, 4 * kBitmapWords, s);
    if (e == cudaSuccess) e = launch_setup(P, GC_MODE_DETERMINISTIC, false, 0, n, -1, s);
    NaCtl h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl, sizeof(NaCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(GC_ERR_CUDA, "setup", e);
    if (h.err[0] != 0)
        return set_last_error(GC_ERR_INVALID_GRAPH, "invalid graph at vertex %d (row offsets must be non-decreasing "
                                                    "from 0 to nnz)", h.err[1]);
    const unsigned n_small = h.cnt[kCnt * 1 + kCntSmall], n_items = h.tmp[0], n_chunks = h.tmp[1];
    if (n_items > static_cast<unsigned>(kNaMaxVertices) || n_chunks > static_cast<unsigned>(kNaMaxItems))
        return set_last_error(GC_ERR_INVALID_GRAPH, "work-item count outside the scratch bounds");
    e = launch_expand(P, GC_MODE_DETERMINISTIC, false, false, static_cast<int32_t>(n_items), s);
    if (e != cudaSuccess) return na_fail(GC_ERR_CUDA, "expand", e);

    int per_sm = 0, sms = 0;
    e = round_kernel_occupancy(GC_MODE_DETERMINISTIC, false, false, 256, &per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return na_fail(GC_ERR_CUDA, "occupancy", e);
    int64_t grid = static_cast<int64_t>(per_sm) * sms;
    const int64_t want = (static_cast<int64_t>(n_small) + 32 * static_cast<int64_t>(n_chunks) + 255) / 256;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    e = launch_rounds(P, GC_MODE_DETERMINISTIC, false, false, static_cast<int>(grid), 256, s);
    // colors go straight to colors_out (the counting kernel skips the copy if an error was posted)
    if (e == cudaSuccess)
        e = launch_count_colors(P, false, &ctl->passes[1], 0, n, 0, 1, bitmap, &ctl->gmax1, &ctl->gcount1, colors_out, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctl, sizeof(NaCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(GC_ERR_CUDA, "round kernel", e);
    switch (h.err[0]) {
        case 0:
            break;
        case GC_ERR_INVALID_GRAPH:
            return set_last_error(GC_ERR_INVALID_GRAPH, "invalid adjacency entry at vertex %d", h.err[1]);
        case GC_ERR_TIMEOUT:
            return set_last_error(GC_ERR_TIMEOUT, "grid barrier wait exceeded its limit");
        case GC_ERR_NO_CONVERGENCE:
            return set_last_error(GC_ERR_NO_CONVERGENCE, "worklist not empty after %d rounds", h.err[1] - 1);
        default:
            return set_last_error(h.err[0], "device error %d", h.err[0]);
    }
    if (ncolors) *ncolors = h.gcount1;
    if (rounds) *rounds = h.passes[1] > 0 ? h.passes[1] : 1;
    return GC_OK;
}
