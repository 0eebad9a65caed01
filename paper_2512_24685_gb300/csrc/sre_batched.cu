// sre_batched.cu -- M2 of many states of uneven N in one submission.
//
// States are grouped in classes of equal N (largest first).  Each class is
// one persistent launch that walks the concatenated work list of all its
// states (the single-tile kernel for N <= 12; for N > 12 the two-pass
// kernel, once for shifts below 4096 and once for the halved shifts).  A norm
// launch covers all states and a finalize launch turns each state's
// fixed-order partial sums into M2, so every result is bitwise the same as
// for that state alone in a batch of equal composition.
//
// The whole submission is captured once into a CUDA graph per distinct
// batch (same state pointers, sizes, output and mode) and replayed from the
// graph afterwards.  The first submission of a batch runs eagerly (it also
// sets kernel attributes, which must not happen during capture) and is then
// captured for later replays; a stream that cannot be captured (the legacy
// default stream) simply runs eagerly every time.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "sre_batched.h"

namespace sre {

namespace {

template <typename T>
cudaError_t grow(T **p, size_t *cap, size_t need) {
    if (*p && *cap >= need) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, sizeof(T) * std::max<size_t>(need, 1));
    if (e == cudaSuccess) *cap = need;
    return e;
}

struct GraphEntry {
    std::vector<const void *> ptrs;  // submission order
    std::vector<int> Ns;
    sre_mode_t mode;
    double *out;
    int *status_out = nullptr;
    // per-entry device tables (stable for replays)
    const void **d_ptrs = nullptr;
    int *d_Ns = nullptr;
    int *d_out = nullptr;
    longlong4 *d_seg = nullptr;
    void *conv = nullptr;  // converted copies (dtype differs from the mode)
    cudaGraphExec_t exec = nullptr;
    unsigned long long generation = 0;  // shared-buffer generation it was built for
    unsigned long long launches = 0;    // kernels one submission launches
};

}  // namespace

struct BatchedContext {
    DeviceInfo dev;
    double *parts = nullptr;
    size_t parts_cap = 0;
    double *npart = nullptr;
    size_t npart_cap = 0;
    int *flags = nullptr;
    size_t flags_cap = 0;
    unsigned *counters = nullptr;
    size_t counters_cap = 0;  // 3 * chunk capacity
    int *tc_e = nullptr;      // split modes: per-state scale tables of a class
    double *tc_bn = nullptr;
    size_t tc_e_cap = 0, tc_bn_cap = 0;
    unsigned long long generation = 1;
    std::vector<GraphEntry> graphs;  // most recent last
};

static void free_entry(GraphEntry &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    cudaFree(g.d_ptrs);
    cudaFree(g.d_Ns);
    cudaFree(g.d_out);
    cudaFree(g.d_seg);
    cudaFree(g.conv);
    g = GraphEntry();
}

BatchedContext *batched_create(const DeviceInfo &dev) {
    BatchedContext *c = new (std::nothrow) BatchedContext();
    if (c) c->dev = dev;
    return c;
}

void batched_destroy(BatchedContext *ctx) {
    if (!ctx) return;
    for (GraphEntry &g : ctx->graphs) free_entry(g);
    cudaFree(ctx->parts);
    cudaFree(ctx->npart);
    cudaFree(ctx->flags);
    cudaFree(ctx->counters);
    cudaFree(ctx->tc_e);
    cudaFree(ctx->tc_bn);
    delete ctx;
}

// Enqueue the whole batch (norm, classes, finalize) for entry g.
static cudaError_t enqueue_entry(BatchedContext *ctx, const Workspace &ws, const DeviceInfo &dev,
                                 GraphEntry &g, const std::vector<BatchClass> &classes,
                                 const std::vector<int> &order, sre_dtype_t dtype, size_t chunk_cap,
                                 cudaStream_t st, long long wait_ns) {
    cudaError_t e;
    const int count = (int)g.ptrs.size();
    const bool fp64 = g.mode == SRE_MODE_FP64;
    if ((int)dtype != (fp64 ? SRE_C128 : SRE_C64)) {
        // converted copies, in class order, at the offsets baked into d_ptrs
        size_t off = 0;
        const size_t eb = fp64 ? 16 : 8;
        for (int k = 0; k < count; ++k) {
            const int i = order[k];
            void *dst = (char *)g.conv + off;
            if ((e = enqueue_convert(g.ptrs[i], dtype, dst, g.Ns[i], st)) != cudaSuccess) return e;
            ws.launches += 1;
            off += eb << g.Ns[i];
        }
    }
    if ((e = enqueue_batch_norm(ws, g.d_ptrs, g.d_Ns, count, ctx->npart, ctx->flags, g.mode, st)) !=
        cudaSuccess)
        return e;
    size_t first = 0;
    for (const BatchClass &L : classes) {
        if ((e = enqueue_batch_class(ws, dev, L, g.d_ptrs + first, ctx->parts, ctx->counters, chunk_cap,
                                     g.mode, st, wait_ns, ctx->tc_e, ctx->tc_bn,
                                     std::min(ctx->tc_e_cap, ctx->tc_bn_cap))) != cudaSuccess)
            return e;
        first += (size_t)L.S;
    }
    return enqueue_batch_finalize(ws, g.d_seg, ctx->parts, ctx->npart, ctx->flags, g.d_Ns, g.d_out,
                                  count, g.out, g.status_out, st);
}

cudaError_t batched_run(BatchedContext *ctx, const Workspace &ws, const DeviceInfo &dev,
                        const void *const *d_states, const int *Ns, int count, sre_dtype_t dtype,
                        sre_mode_t mode, cudaStream_t stream, double *d_m2_out, long long wait_ns,
                        const LargeCfg *const *tuned_half, bool capture, int *d_status_out) {
    cudaError_t e;
    // ---- replay an existing graph for an identical batch
    for (size_t k = 0; k < ctx->graphs.size(); ++k) {
        GraphEntry &g = ctx->graphs[k];
        if (g.mode != mode || g.out != d_m2_out || g.status_out != d_status_out || (int)g.ptrs.size() != count)
            continue;
        if (!std::equal(g.ptrs.begin(), g.ptrs.end(), d_states) || !std::equal(g.Ns.begin(), g.Ns.end(), Ns))
            continue;
        if (g.exec && g.generation == ctx->generation) {
            e = cudaGraphLaunch(g.exec, stream);
            if (e == cudaSuccess) ws.launches += g.launches;
            return e;
        }
    }

    // ---- layout: classes of equal N, largest first (stable in submission order)
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return Ns[a] > Ns[b]; });
    std::vector<BatchClass> classes;
    for (int k = 0; k < count;) {
        int j = k;
        while (j < count && Ns[order[j]] == Ns[order[k]]) ++j;
        const int N = Ns[order[k]];
        classes.push_back(batch_class_layout(dev, ws, N, j - k, mode, tuned_half ? tuned_half[N] : nullptr));
        k = j;
    }
    size_t parts_total = 0, chunk_cap = 1;
    for (BatchClass &L : classes) {
        L.parts_off = parts_total;
        parts_total += L.parts_n;
        chunk_cap = std::max(chunk_cap, L.chunks_max);
    }
    std::vector<longlong4> seg(count);
    std::vector<int> sNs(count), sout(count);
    {
        int k = 0;
        for (const BatchClass &L : classes) {
            for (int s = 0; s < L.S; ++s, ++k) {
                longlong4 v;
                if (L.N <= kTileBits) {
                    v = make_longlong4((long long)L.parts_off + s * L.cps_full, L.cps_full, 0, 0);
                } else {
                    const long long offB = (long long)L.parts_off + (long long)L.S * L.cps_full;
                    v = make_longlong4((long long)L.parts_off + s * L.cps_full, L.cps_full,
                                       offB + s * L.cps_half, L.cps_half);
                }
                seg[k] = v;
                sNs[k] = Ns[order[k]];
                sout[k] = order[k];
            }
        }
    }

    // ---- shared buffers (a reallocation invalidates every captured graph)
    const size_t gen0 = ctx->parts_cap + ctx->npart_cap + ctx->flags_cap + ctx->counters_cap;
    if ((e = grow(&ctx->parts, &ctx->parts_cap, parts_total)) != cudaSuccess) return e;
    if ((e = grow(&ctx->npart, &ctx->npart_cap, (size_t)count * kNormBlocks)) != cudaSuccess) return e;
    if ((e = grow(&ctx->flags, &ctx->flags_cap, (size_t)count)) != cudaSuccess) return e;
    if ((e = grow(&ctx->counters, &ctx->counters_cap, 3 * chunk_cap)) != cudaSuccess) return e;
    chunk_cap = ctx->counters_cap / 3;
    if (ctx->parts_cap + ctx->npart_cap + ctx->flags_cap + ctx->counters_cap != gen0) ++ctx->generation;

    // ---- the entry with its own device tables
    if (ctx->graphs.size() >= 8) {
        free_entry(ctx->graphs.front());
        ctx->graphs.erase(ctx->graphs.begin());
    }
    ctx->graphs.emplace_back();
    GraphEntry &g = ctx->graphs.back();
    g.ptrs.assign(d_states, d_states + count);
    g.Ns.assign(Ns, Ns + count);
    g.mode = mode;
    g.out = d_m2_out;
    g.status_out = d_status_out;
    g.generation = ctx->generation;
    const bool fp64 = mode == SRE_MODE_FP64;
    const bool convert = (int)dtype != (fp64 ? SRE_C128 : SRE_C64);
    std::vector<const void *> sptr(count);
    size_t conv_total = 0;
    for (int k = 0; k < count; ++k) conv_total += (size_t)(fp64 ? 16 : 8) << sNs[k];
    if (convert && (e = cudaMalloc(&g.conv, conv_total)) != cudaSuccess) {
        free_entry(g);
        ctx->graphs.pop_back();
        return e;
    }
    size_t off = 0;
    for (int k = 0; k < count; ++k) {
        sptr[k] = convert ? (const void *)((char *)g.conv + off) : d_states[order[k]];
        if (convert) off += (size_t)(fp64 ? 16 : 8) << sNs[k];
    }
    // split modes: a class whose halved shifts fit the tensor-core kernel
    // (16 <= N <= 20) and whose states are all 16-byte aligned takes it
    {
        size_t tc_need = 0;
        int k = 0;
        for (BatchClass &L : classes) {
            L.tc_kind = 0;
            if (tc_mode_available(mode) && L.N > kTileBits && tc_applies(L.N, 1, 2, sptr[k])) {
                bool aligned = true;
                for (int q = 0; q < L.S; ++q) aligned &= ((uintptr_t)sptr[k + q] & 15) == 0;
                if (aligned) {
                    L.tc_kind = mode == SRE_MODE_BF16_SPLIT ? 1 : 2;
                    tc_need = std::max(tc_need, (size_t)L.S << (L.N - kTileBits));
                }
            }
            k += L.S;
        }
        const size_t tc0 = ctx->tc_e_cap + ctx->tc_bn_cap;
        if (tc_need && ((e = grow(&ctx->tc_e, &ctx->tc_e_cap, tc_need)) != cudaSuccess ||
                        (e = grow(&ctx->tc_bn, &ctx->tc_bn_cap, tc_need)) != cudaSuccess)) {
            free_entry(g);
            ctx->graphs.pop_back();
            return e;
        }
        if (ctx->tc_e_cap + ctx->tc_bn_cap != tc0) {
            ++ctx->generation;  // graphs captured before hold the old tables
            g.generation = ctx->generation;
        }
    }
    size_t tmp = 0;
    if ((e = grow(&g.d_ptrs, &tmp, (size_t)count)) != cudaSuccess ||
        (e = grow(&g.d_Ns, &(tmp = 0), (size_t)count)) != cudaSuccess ||
        (e = grow(&g.d_out, &(tmp = 0), (size_t)count)) != cudaSuccess ||
        (e = grow(&g.d_seg, &(tmp = 0), (size_t)count)) != cudaSuccess) {
        free_entry(g);
        ctx->graphs.pop_back();
        return e;
    }
    // the tables are copied synchronously: they must be in place before any
    // (captured or eager) work reads them
    if ((e = cudaMemcpy(g.d_ptrs, sptr.data(), sizeof(void *) * count, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(g.d_Ns, sNs.data(), sizeof(int) * count, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(g.d_out, sout.data(), sizeof(int) * count, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(g.d_seg, seg.data(), sizeof(longlong4) * count, cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;

    // ---- eager run now, then capture for later replays
    const unsigned long long l0 = ws.launches;
    if ((e = enqueue_entry(ctx, ws, dev, g, classes, order, dtype, chunk_cap, stream, wait_ns)) != cudaSuccess)
        return e;
    g.launches = ws.launches - l0;
    if (!capture) {
        // one-off batch (e.g. a server unit): keep no entry around
        free_entry(g);
        ctx->graphs.pop_back();
        return cudaSuccess;
    }
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return cudaSuccess;
    if (stream == 0 || stream == cudaStreamLegacy) return cudaSuccess;  // not capturable
    const unsigned long long launches = ws.launches;
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;
    }
    e = enqueue_entry(ctx, ws, dev, g, classes, order, dtype, chunk_cap, stream, wait_ns);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(stream, &graph);
    ws.launches = launches;
    if (e == cudaSuccess && e2 == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) g.exec = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();  // a failed capture leaves the eager result valid
    return cudaSuccess;
}

}  // namespace sre
