// sre_server.cu -- continuous-batching M2 server of libsre.
//
// Requests of mixed N arrive through sre_server_submit, which copies the
// state into device memory owned by the server and admits it only if the
// bytes resident on the device (queued + in-flight states, plus the slots'
// scratch) stay within the HBM budget (SRE_EBUSY otherwise).  A host
// scheduler thread owns `max_inflight` slots; each slot has its own stream,
// scratch workspace and batched-evaluation context, so the work of different
// slots overlaps on the device.  Whenever a slot is free the scheduler takes
// the oldest queued request and, if it is small (N <= kBatchMaxN), also
// the next queued small requests up to a work cap, and launches them as one
// batched evaluation; a large request gets a slot of its own.  Completion is
// detected with CUDA events; latencies (submit -> result on the host) feed
// p50/p99.  Device-side waits inside the kernels are bounded by the
// configured wait limit; every request carries the status its evaluation
// recorded on the device (a merged batch whose wait expired marks all of
// its requests SRE_ETIMEDOUT).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "sre_batched.h"
#include "sre_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kBatchMaxN = 16;                  // requests up to this N may share a launch
constexpr double kBatchWorkCap = 4.0e10;        // Pauli terms per merged launch
constexpr int kBatchMaxCount = 256;

struct Request {
    uint64_t ticket = 0;
    int N = 0;
    void *d_state = nullptr;  // server-owned copy, compute dtype
    size_t bytes = 0;
    Clock::time_point t_submit;
    double m2 = 0.0;
    int status = 0;
    bool done = false;
    // shift-range units (chunked requests have parts > 1)
    int parts = 1, next_part = 0, parts_done = 0;
    std::vector<double> S_part;  // partial S of each range
    double n2 = 0.0;
    int unit_status = 0;         // first non-zero status of a unit
};

struct Slot {
    cudaStream_t stream = nullptr;
    sre::Workspace ws;
    sre::BatchedContext *batched = nullptr;
    cudaEvent_t ev = nullptr;
    double *d_out = nullptr;   // kBatchMaxCount
    double *h_out = nullptr;   // pinned
    int *d_st = nullptr;       // kBatchMaxCount per-request statuses
    int *h_st = nullptr;       // pinned
    sre::Result *h_res = nullptr;  // pinned (single-request path)
    std::vector<uint64_t> tickets;  // in flight
    bool single = false;
    int part = 0;                   // single path: the unit (shift range) in flight
    bool busy = false;
};

}  // namespace

struct sre_server_s {
    sre_server_cfg_t cfg;
    sre::DeviceInfo dev;
    std::vector<Slot> slots;
    size_t slot_bytes = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Request> reqs;
    std::atomic<bool> stop{false};
    std::thread worker;
    uint64_t next_ticket = 1;
    uint64_t resident = 0, peak_resident = 0;
    uint64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, failed = 0;
    double terms_done = 0.0;
    std::vector<double> latencies_ms;
    Clock::time_point t_first;
    bool have_first = false;
    Clock::time_point t_last_done;
    std::map<size_t, std::vector<void *>> pool;  // device buffers by size
    cudaStream_t copy_stream = nullptr;          // submit-side copies / conversions
    std::mutex copy_mu;
    sre::LargeCfg tuned[SRE_MAX_QUBITS + 1];     // sre_server_set_tuning, per N
    bool has_tuned[SRE_MAX_QUBITS + 1] = {};
};

namespace {

// Shift ranges of a request: 2^k ranges of at most chunk_terms Pauli terms
// each (and at least 4096 shifts) for N > kBatchMaxN, else one.
int server_parts(const sre_server_cfg_t &cfg, int N) {
    if (!cfg.chunk_terms || N <= kBatchMaxN) return 1;
    const double terms = std::ldexp(1.0, 2 * N);
    int k = 0;
    while (terms / std::ldexp(1.0, k) > (double)cfg.chunk_terms && N - k > sre::kTileBits) ++k;
    return 1 << k;
}

void *pool_get(sre_server_s *s, size_t bytes) {
    auto it = s->pool.find(bytes);
    if (it != s->pool.end() && !it->second.empty()) {
        void *p = it->second.back();
        it->second.pop_back();
        return p;
    }
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pool_put(sre_server_s *s, void *p, size_t bytes) { s->pool[bytes].push_back(p); }

void finish(sre_server_s *s, Request &r, double m2, int status) {
    r.m2 = m2;
    r.status = status;
    r.done = true;
    const Clock::time_point now = Clock::now();
    s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
    s->completed += 1;
    if (status) s->failed += 1;
    s->terms_done += std::ldexp(1.0, 2 * r.N);
    s->t_last_done = now;
    pool_put(s, r.d_state, r.bytes);
    r.d_state = nullptr;
    s->resident -= r.bytes;
}

// A unit of a chunked request has finished (or failed to launch): record
// its partial sum and finish the request after its last unit, adding the
// partial sums in range order (Eq. (final1) on their total).
void unit_done(sre_server_s *s, Request &r, int part, double S, double n2, int status) {
    if (status && !r.unit_status) r.unit_status = status;
    if (status == SRE_ECUDA || status == SRE_ETIMEDOUT) {
        // drop the units not launched yet
        r.parts_done += r.parts - r.next_part;
        r.next_part = r.parts;
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
            if (*it == r.ticket) {
                s->queue.erase(it);
                break;
            }
    }
    if (part >= 0) {
        r.S_part[(size_t)part] = S;
        r.n2 = n2;
    }
    r.parts_done += 1;
    if (r.parts_done < r.parts) return;
    double St = 0.0;
    for (double v : r.S_part) St += v;
    const int st = r.unit_status;
    const double m2 = (st || !(St > 0.0) || !(r.n2 > 0.0)) ? std::nan("")
                                                           : -(std::log2(St) - (double)r.N - 4.0 * std::log2(r.n2));
    finish(s, r, m2, st);
}

// Launch the next unit of work on slot sl (mutex held): the oldest queued
// request, merged with later small requests, or one shift range of a large
// (possibly chunked) request, which then goes to the back of the queue if
// it has more ranges.
void launch_unit(sre_server_s *s, Slot &sl) {
    if (s->queue.empty()) return;
    std::vector<uint64_t> take;
    const uint64_t head = s->queue.front();
    Request &h = s->reqs[head];
    s->queue.pop_front();
    take.push_back(head);
    const bool single = h.N > kBatchMaxN;
    if (!single) {
        double work = std::ldexp(1.0, 2 * h.N);
        for (auto it = s->queue.begin(); it != s->queue.end() && (int)take.size() < kBatchMaxCount;) {
            const Request &q = s->reqs[*it];
            const double w = std::ldexp(1.0, 2 * q.N);
            if (q.N <= kBatchMaxN && work + w <= kBatchWorkCap) {
                work += w;
                take.push_back(*it);
                it = s->queue.erase(it);
            } else {
                ++it;
            }
        }
    }
    const sre_dtype_t dt = s->cfg.mode == SRE_MODE_FP64 ? SRE_C128 : SRE_C64;
    cudaError_t e;
    sl.single = single;
    if (single) {
        const int part = h.next_part++;
        if (h.next_part < h.parts) s->queue.push_back(head);  // round robin over ranges
        const uint64_t d = 1ull << h.N, span = d / (uint64_t)h.parts;
        sre::LargeCfg c;
        sre::LargeCfg *cp = nullptr;
        if (s->has_tuned[h.N]) {
            c = s->tuned[h.N];
            cp = &c;
        }
        sl.part = part;
        e = sre::enqueue_m2(sl.ws, s->dev, h.d_state, dt, h.N, span * (uint64_t)part, span * (uint64_t)(part + 1),
                            s->cfg.mode, sl.stream, nullptr, nullptr, (long long)s->cfg.wait_limit_ns, cp);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.h_res, sl.ws.result, sizeof(sre::Result), cudaMemcpyDeviceToHost, sl.stream);
    } else {
        std::vector<const void *> ptrs;
        std::vector<int> Ns;
        for (uint64_t t : take) {
            ptrs.push_back(s->reqs[t].d_state);
            Ns.push_back(s->reqs[t].N);
        }
        e = sre::batched_run(sl.batched, sl.ws, s->dev, ptrs.data(), Ns.data(), (int)take.size(), dt,
                             s->cfg.mode, sl.stream, sl.d_out, (long long)s->cfg.wait_limit_ns, nullptr,
                             /*capture=*/false, sl.d_st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.h_out, sl.d_out, sizeof(double) * take.size(), cudaMemcpyDeviceToHost,
                                sl.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.h_st, sl.d_st, sizeof(int) * take.size(), cudaMemcpyDeviceToHost, sl.stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (single)
            unit_done(s, h, -1, 0.0, 0.0, SRE_ECUDA);
        else
            for (uint64_t t : take) finish(s, s->reqs[t], std::nan(""), SRE_ECUDA);
        return;
    }
    if (!single || sl.part == 0) s->admitted += take.size();
    sl.tickets = take;
    sl.busy = true;
}

void collect(sre_server_s *s, Slot &sl) {
    const cudaError_t q = cudaEventQuery(sl.ev);
    if (q == cudaErrorNotReady) return;
    if (q != cudaSuccess) cudaGetLastError();
    for (size_t i = 0; i < sl.tickets.size(); ++i) {
        Request &r = s->reqs[sl.tickets[i]];
        if (sl.single) {
            if (q != cudaSuccess)
                unit_done(s, r, -1, 0.0, 0.0, SRE_ECUDA);
            else if (r.parts == 1)
                finish(s, r, sl.h_res->m2, sl.h_res->status);  // the device's own M2, as alone
            else
                unit_done(s, r, sl.part, sl.h_res->S, sl.h_res->n2, sl.h_res->status);
        } else if (q != cudaSuccess) {
            finish(s, r, std::nan(""), SRE_ECUDA);
        } else {
            finish(s, r, sl.h_out[i], sl.h_st[i]);
        }
    }
    sl.tickets.clear();
    sl.busy = false;
}

void worker_main(sre_server_s *s) {
    cudaSetDevice(s->cfg.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop.load()) {
        bool any_busy = false;
        for (Slot &sl : s->slots) {
            if (sl.busy) collect(s, sl);
            if (!sl.busy) launch_unit(s, sl);
            any_busy |= sl.busy;
        }
        s->cv.notify_all();
        if (any_busy)
            s->cv.wait_for(lk, std::chrono::microseconds(20));
        else
            s->cv.wait_for(lk, std::chrono::milliseconds(2),
                           [&] { return s->stop.load() || !s->queue.empty(); });
    }
    // drain in-flight work
    for (Slot &sl : s->slots) {
        if (sl.busy) {
            cudaEventSynchronize(sl.ev);
            collect(s, sl);
        }
    }
}

void destroy_slots(sre_server_s *s) {
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        sre::batched_destroy(sl.batched);
        sre::workspace_free(&sl.ws);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        cudaFree(sl.d_out);
        cudaFreeHost(sl.h_out);
        cudaFree(sl.d_st);
        cudaFreeHost(sl.h_st);
        cudaFreeHost(sl.h_res);
    }
    s->slots.clear();
}

}  // namespace

extern "C" {

void sre_server_cfg_default(sre_server_cfg_t *cfg) {
    if (!cfg) return;
    cfg->hbm_budget_bytes = 8ull << 30;
    cfg->max_inflight = 4;
    cfg->max_queue = 4096;
    cfg->max_N = 20;
    cfg->mode = SRE_MODE_FP32;
    cfg->wait_limit_ns = 5000000000ull;
    cfg->device = 0;
    cfg->slot_scratch_bytes = 0;
    cfg->chunk_terms = 0;
}

sre_status_t sre_server_create(const sre_server_cfg_t *cfg, sre_server_t *out) {
    if (!cfg || !out) return SRE_EINVAL;
    if (cfg->max_N < 1 || cfg->max_N > SRE_MAX_QUBITS || cfg->max_inflight < 1 || cfg->max_inflight > 64 ||
        cfg->max_queue < 1 ||
        (cfg->mode != SRE_MODE_FP32 && cfg->mode != SRE_MODE_FP64 && !sre::tc_mode_available(cfg->mode)))
        return SRE_EINVAL;
    if (cfg->slot_scratch_bytes > (64ull << 30)) return SRE_EINVAL;
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        cudaGetLastError();
        return SRE_ECUDA;
    }
    sre_server_s *s = new (std::nothrow) sre_server_s();
    if (!s) return SRE_ENOMEM;
    s->cfg = *cfg;
    if (sre::query_device(&s->dev) != cudaSuccess) {
        delete s;
        return SRE_ECUDA;
    }
    const int eb = cfg->mode == SRE_MODE_FP64 ? 16 : 8;
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return SRE_ECUDA;
    }
    s->slots.resize(cfg->max_inflight);
    for (Slot &sl : s->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        const size_t scratch = cfg->slot_scratch_bytes ? (size_t)cfg->slot_scratch_bytes : sre::kSlotScratch;
        if (e == cudaSuccess) e = sre::workspace_alloc(&sl.ws, s->dev, cfg->max_N, eb, cfg->mode, scratch);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_out, sizeof(double) * kBatchMaxCount);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_out, sizeof(double) * kBatchMaxCount);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_st, sizeof(int) * kBatchMaxCount);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_st, sizeof(int) * kBatchMaxCount);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_res, sizeof(sre::Result));
        sl.batched = sre::batched_create(s->dev);
        if (e != cudaSuccess || !sl.batched) {
            cudaGetLastError();
            destroy_slots(s);
            cudaStreamDestroy(s->copy_stream);
            delete s;
            return e == cudaErrorMemoryAllocation ? SRE_ENOMEM : SRE_ECUDA;
        }
        s->slot_bytes += sl.ws.scratch_bytes + sizeof(double) * (sl.ws.item_part_cap + sl.ws.chunk_cap) +
                         sizeof(unsigned) * 3 * sl.ws.chunk_cap;
    }
    s->resident = s->slot_bytes;
    s->peak_resident = s->resident;
    if (s->resident > cfg->hbm_budget_bytes) {
        destroy_slots(s);
        cudaStreamDestroy(s->copy_stream);
        delete s;
        return SRE_EINVAL;  // the budget does not even cover the slots' scratch
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return SRE_OK;
}

sre_status_t sre_server_set_tuning(sre_server_t s, int N, const sre_tuning_t *t) {
    if (!s || !t || N <= sre::kTileBits || N > s->cfg.max_N) return SRE_EINVAL;
    const int eb = s->cfg.mode == SRE_MODE_FP64 ? 16 : 8;
    sre::LargeCfg c = sre::choose_large_cfg(s->dev, N, eb, 1);
    if (t->x_batch_log >= 0) c.C_log = t->x_batch_log;
    if (t->ring_slots >= 0) c.R = t->ring_slots;
    if (t->lag >= 0) c.D = t->lag;
    if (t->pass2_tiles_log >= 0) c.G2_log = t->pass2_tiles_log;
    if (t->pass1_blocks_log >= 0) c.B1_log = t->pass1_blocks_log;
    if (t->pass1_staged >= 0) c.stage1 = t->pass1_staged;
    if (t->pass2_staged >= 0) c.stage2 = t->pass2_staged;
    c.G2_log = std::min(c.G2_log, N - sre::kTileBits - 1);
    c.B1_log = std::min(c.B1_log, N - sre::kTileBits - 1);
    std::lock_guard<std::mutex> lk(s->mu);
    for (const Slot &sl : s->slots)
        if (!sre::large_cfg_fits(sl.ws, c, N, 1)) return SRE_EINVAL;
    s->tuned[N] = c;
    s->has_tuned[N] = true;
    return SRE_OK;
}

sre_status_t sre_server_submit(sre_server_t s, const void *state, int on_device, int N, sre_dtype_t dtype,
                               uint64_t *ticket) {
    if (!s || !state || !ticket || N < 1 || N > s->cfg.max_N) return SRE_EINVAL;
    if (dtype != SRE_C64 && dtype != SRE_C128) return SRE_EINVAL;
    const bool fp64 = s->cfg.mode == SRE_MODE_FP64;
    const size_t in_eb = dtype == SRE_C128 ? 16 : 8, eb = fp64 ? 16 : 8;
    const size_t bytes = eb << N;
    std::unique_lock<std::mutex> lk(s->mu);
    s->submitted += 1;
    if ((int)s->queue.size() >= s->cfg.max_queue || s->resident + bytes > s->cfg.hbm_budget_bytes) {
        s->rejected += 1;
        return SRE_EBUSY;
    }
    void *d = pool_get(s, bytes);
    if (!d) {
        s->rejected += 1;
        return SRE_ENOMEM;
    }
    s->resident += bytes;
    s->peak_resident = std::max(s->peak_resident, s->resident);
    lk.unlock();
    // copy (and convert) into the server's buffer; synchronous, so the caller
    // may reuse its buffer when this returns
    cudaError_t e;
    cudaSetDevice(s->cfg.device);
    {
        std::lock_guard<std::mutex> ck(s->copy_mu);
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (in_eb == eb) {
            e = cudaMemcpyAsync(d, state, bytes, kind, s->copy_stream);
        } else {
            void *tmp = nullptr;
            e = cudaMalloc(&tmp, in_eb << N);
            if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, state, in_eb << N, kind, s->copy_stream);
            if (e == cudaSuccess) e = sre::enqueue_convert(tmp, dtype, d, N, s->copy_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
            cudaFree(tmp);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
    }
    lk.lock();
    if (e != cudaSuccess) {
        cudaGetLastError();
        pool_put(s, d, bytes);
        s->resident -= bytes;
        s->rejected += 1;
        return SRE_ECUDA;
    }
    Request r;
    r.ticket = s->next_ticket++;
    r.N = N;
    r.d_state = d;
    r.bytes = bytes;
    r.parts = server_parts(s->cfg, N);
    r.S_part.assign((size_t)r.parts, 0.0);
    r.t_submit = Clock::now();
    if (!s->have_first) {
        s->t_first = r.t_submit;
        s->have_first = true;
    }
    s->reqs[r.ticket] = r;
    s->queue.push_back(r.ticket);
    *ticket = r.ticket;
    s->cv.notify_all();
    return SRE_OK;
}

sre_status_t sre_server_poll(sre_server_t s, uint64_t ticket, int *done, double *m2) {
    if (!s || !done) return SRE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return SRE_ENOTFOUND;
    if (!it->second.done) {
        *done = 0;
        return SRE_OK;
    }
    *done = 1;
    if (m2) *m2 = it->second.m2;
    const int st = it->second.status;
    s->reqs.erase(it);
    return st == SRE_ETIMEDOUT || st == SRE_ECUDA ? (sre_status_t)st : SRE_OK;
}

sre_status_t sre_server_wait(sre_server_t s, uint64_t ticket, double timeout_ms, double *m2) {
    if (!s) return SRE_EINVAL;
    const Clock::time_point end = Clock::now() + std::chrono::microseconds((long long)(timeout_ms * 1000.0));
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return SRE_ENOTFOUND;
        if (it->second.done) {
            if (m2) *m2 = it->second.m2;
            const int st = it->second.status;
            s->reqs.erase(it);
            return st == SRE_ETIMEDOUT || st == SRE_ECUDA ? (sre_status_t)st : SRE_OK;
        }
        if (s->cv.wait_until(lk, end) == std::cv_status::timeout && Clock::now() >= end) return SRE_ETIMEDOUT;
    }
}

sre_status_t sre_server_stats(sre_server_t s, sre_server_stats_t *st) {
    if (!s || !st) return SRE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *st = sre_server_stats_t();
    st->submitted = s->submitted;
    st->admitted = s->admitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->failed = s->failed;
    st->queued = s->queue.size();
    uint64_t inflight = 0;
    for (const Slot &sl : s->slots) inflight += sl.tickets.size();
    st->inflight = inflight;
    if (!s->latencies_ms.empty()) {
        std::vector<double> v = s->latencies_ms;
        auto pct = [&](double q) {
            const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return v[k];
        };
        st->p50_latency_ms = pct(0.50);
        st->p99_latency_ms = pct(0.99);
        double sum = 0.0;
        for (double x : s->latencies_ms) sum += x;
        st->mean_latency_ms = sum / (double)s->latencies_ms.size();
    }
    if (s->have_first && s->completed) {
        const double secs = std::chrono::duration<double>(s->t_last_done - s->t_first).count();
        if (secs > 0) {
            st->states_per_s = (double)s->completed / secs;
            st->pauli_terms_per_s = s->terms_done / secs;
        }
    }
    st->resident_bytes = s->resident;
    st->peak_resident_bytes = s->peak_resident;
    return SRE_OK;
}

sre_status_t sre_server_destroy(sre_server_t s) {
    if (!s) return SRE_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop.store(true);
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    destroy_slots(s);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    for (auto &kv : s->pool)
        for (void *p : kv.second) cudaFree(p);
    for (auto &kv : s->reqs)
        if (kv.second.d_state) cudaFree(kv.second.d_state);
    delete s;
    return SRE_OK;
}

}  // extern "C"
