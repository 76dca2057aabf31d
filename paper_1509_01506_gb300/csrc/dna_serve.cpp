// dna_serve.cpp -- the request loop: scans of mixed sizes against resident automata,
// admitted continuously as device slots and memory free up.
//
// A server owns S slots (one CUDA stream each), a device memory pool and a dispatcher
// thread. Requests (a host sequence, an automaton index, an arrival time) wait in
// arrival order; the dispatcher admits the head of the queue as soon as its arrival
// time has passed, a slot is free and the device memory the request needs fits under
// the admission cap. An admitted request is queued on its slot's stream as: copy the
// sequence to the device, the chunked scan of Sec. III-A (the same kernels as dna_scan,
// count only), copy the count back, record an event. Different slots' copies and
// kernels overlap on the device. The dispatcher polls the slots' events; a finished
// request is stamped, its memory returns to the pool and its slot takes the next
// request. The paper scans one input at a time; this loop is the serving form of the
// same scan.

#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/dna_dfa.h"
#include "dna_runtime.h"

using namespace dnalib;

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t id;
    const uint8_t *host;
    uint64_t len;
    uint32_t dfa;
    uint64_t arrival_ns;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_h2d = nullptr, ev_end = nullptr;
    uint64_t *d_count = nullptr;      // device result
    uint64_t *h_count = nullptr;      // pinned host copy of the result
    void *d_seq = nullptr;            // the request's sequence (from the pool)
    uint64_t need = 0;                // admitted bytes
    bool busy = false;
    Request req{};
    uint64_t admit_ns = 0;
    int status = DNA_OK;
};

// Device bytes a request is charged for: its sequence (16-byte padded) and the scan's
// stream-ordered scratch (chunk bookkeeping, about 32 bytes per 2 KiB chunk; 1 MiB
// covers it for any request the cap admits).
uint64_t request_bytes(uint64_t len) { return ((len + 4095) & ~4095ull) + (1ull << 20); }

}  // namespace

struct dna_server {
    int device = 0;
    std::vector<const dna_dfa *> dfas;
    uint64_t cap = 0;
    std::vector<Slot> slots;
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv_submit, cv_done;
    std::deque<Request> queue;
    std::deque<dna_completion> done;
    uint64_t in_use = 0;
    int64_t next_id = 0;
    uint64_t submitted = 0, completed = 0;
    bool stop = false;
    std::thread worker;
    std::atomic<int> fatal{DNA_OK};
};

namespace {

// Queues one request on a free slot (dispatcher thread, lock not held).
int admit(dna_server &s, Slot &sl, const Request &r) {
    sl.req = r;
    sl.busy = true;
    sl.admit_ns = now_ns();
    sl.need = request_bytes(r.len);
    sl.status = DNA_OK;
    cudaError_t e = cudaEventRecord(sl.ev_start, sl.stream);
    if (e == cudaSuccess && r.len)
        e = pool_alloc(&sl.d_seq, r.len + 16, s.pool, sl.stream);
    if (e == cudaSuccess && r.len)
        e = cudaMemcpyAsync(sl.d_seq, r.host, r.len, cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev_h2d, sl.stream);
    int rc = cuda_status(e);
    if (rc == DNA_OK)
        rc = scan_impl(s.dfas[r.dfa], (const uint8_t *)sl.d_seq, r.len, sl.stream, sl.d_count, nullptr, 0, nullptr);
    if (rc == DNA_OK)
        rc = cuda_status(cudaMemcpyAsync(sl.h_count, sl.d_count, 8, cudaMemcpyDeviceToHost, sl.stream));
    if (sl.d_seq) {
        cudaFreeAsync(sl.d_seq, sl.stream);
        sl.d_seq = nullptr;
    }
    cudaEventRecord(sl.ev_end, sl.stream);
    sl.status = rc;
    return rc;
}

void dispatcher(dna_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool progress = false;
        // completions
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            lk.unlock();
            const cudaError_t q = cudaEventQuery(sl.ev_end);
            const uint64_t t = now_ns();
            lk.lock();
            if (q == cudaErrorNotReady) continue;
            dna_completion c;
            c.id = sl.req.id;
            c.dfa = sl.req.dfa;
            c.len = sl.req.len;
            c.arrival_ns = sl.req.arrival_ns;
            c.admit_ns = sl.admit_ns;
            c.done_ns = t;
            c.status = sl.status != DNA_OK ? sl.status : cuda_status(q);
            c.count = c.status == DNA_OK ? *sl.h_count : 0;
            float h2d = 0.f, all = 0.f;
            cudaEventElapsedTime(&h2d, sl.ev_start, sl.ev_h2d);
            cudaEventElapsedTime(&all, sl.ev_start, sl.ev_end);
            c.h2d_us = h2d * 1e3f;
            c.device_us = all * 1e3f;
            s->in_use -= sl.need;
            sl.busy = false;
            s->done.push_back(c);
            ++s->completed;
            progress = true;
        }
        if (progress) s->cv_done.notify_all();
        // admissions, in arrival order
        const uint64_t t = now_ns();
        while (!s->queue.empty()) {
            const Request &r = s->queue.front();
            if (r.arrival_ns > t) break;
            const uint64_t need = request_bytes(r.len);
            if (need > s->cap) {   // can never fit: fail it instead of blocking the queue
                dna_completion c{};
                c.id = r.id; c.dfa = r.dfa; c.len = r.len; c.arrival_ns = r.arrival_ns;
                c.admit_ns = c.done_ns = t; c.status = DNA_ERR_CAPACITY;
                s->done.push_back(c);
                ++s->completed;
                s->queue.pop_front();
                s->cv_done.notify_all();
                continue;
            }
            if (s->in_use + need > s->cap) break;
            Slot *free_slot = nullptr;
            for (Slot &sl : s->slots)
                if (!sl.busy) { free_slot = &sl; break; }
            if (!free_slot) break;
            Request req = r;
            s->queue.pop_front();
            s->in_use += need;
            free_slot->busy = true;
            lk.unlock();
            admit(*s, *free_slot, req);
            lk.lock();
            progress = true;
        }
        bool any_busy = false;
        for (Slot &sl : s->slots) any_busy |= sl.busy;
        if (s->stop && !any_busy && s->queue.empty()) break;
        if (progress) continue;
        if (any_busy) {
            // work in flight: poll again at once (a sleep would delay completion stamps by
            // the timer slack, tens of microseconds)
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else if (!s->queue.empty()) {
            // idle until the head request arrives (or a new submit)
            const uint64_t head = s->queue.front().arrival_ns, t2 = now_ns();
            if (head > t2 + 200000)
                s->cv_submit.wait_for(lk, std::chrono::nanoseconds(head - t2 - 100000));
            else {
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            }
        } else {
            s->cv_submit.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
}

void destroy(dna_server *s) {
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_submit.notify_all();
        s->worker.join();
    }
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ev_start) cudaEventDestroy(sl.ev_start);
        if (sl.ev_h2d) cudaEventDestroy(sl.ev_h2d);
        if (sl.ev_end) cudaEventDestroy(sl.ev_end);
        if (sl.d_count) cudaFree(sl.d_count);
        if (sl.h_count) cudaFreeHost(sl.h_count);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
}

}  // namespace

// ========================================================================= C ABI

extern "C" uint64_t dna_server_now_ns(void) { return now_ns(); }

extern "C" int dna_server_create(const dna_dfa *const *dfas, uint32_t n_dfas, const dna_server_opts *opts,
                                 dna_server **out) {
    if (!dfas || !out || n_dfas == 0) return DNA_ERR_INVALID_ARG;
    int dev = -1;
    DNA_CUDA(cudaGetDevice(&dev));
    for (uint32_t k = 0; k < n_dfas; ++k)
        if (!dfas[k] || dfas[k]->device != dev) return DNA_ERR_INVALID_ARG;
    const uint32_t n_slots = opts && opts->slots ? opts->slots : 8;
    if (n_slots > 256) return DNA_ERR_INVALID_ARG;
    dna_server *s = new (std::nothrow) dna_server;
    if (!s) return DNA_ERR_NOMEM;
    s->device = dev;
    s->dfas.assign(dfas, dfas + n_dfas);
    s->cap = opts && opts->mem_cap_bytes ? opts->mem_cap_bytes : (40ull << 30);
    s->slots.resize(n_slots);
    cudaError_t e = cudaSuccess;
    for (Slot &sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&sl.ev_start);
        if (e == cudaSuccess) e = cudaEventCreate(&sl.ev_h2d);
        if (e == cudaSuccess) e = cudaEventCreate(&sl.ev_end);
        if (e == cudaSuccess) e = device_alloc((void **)&sl.d_count, 8);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_count, 8);
    }
    if (e == cudaSuccess) {
        // the server's own pool keeps up to the cap reserved between requests
        cudaMemPoolProps pp = {};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.handleTypes = cudaMemHandleTypeNone;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = dev;
        e = cudaMemPoolCreate(&s->pool, &pp);
        if (e == cudaSuccess) {
            uint64_t thr = s->cap;
            e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    if (e != cudaSuccess) {
        destroy(s);
        return cuda_status(e);
    }
    try {
        s->worker = std::thread(dispatcher, s);
    } catch (...) {
        destroy(s);
        return DNA_ERR_NOMEM;
    }
    *out = s;
    return DNA_OK;
}

extern "C" int64_t dna_server_submit(dna_server *s, const uint8_t *host_seq, uint64_t len, uint32_t dfa,
                                     uint64_t arrival_ns) {
    if (!s || (len && !host_seq) || dfa >= s->dfas.size() || len > (1ull << 40)) return DNA_ERR_INVALID_ARG;
    if (s->fatal.load() != DNA_OK) return s->fatal.load();
    Request r;
    r.host = host_seq;
    r.len = len;
    r.dfa = dfa;
    r.arrival_ns = arrival_ns ? arrival_ns : now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return DNA_ERR_INVALID_ARG;
        r.id = s->next_id++;
        // arrival order: a request scheduled before the tail is inserted in place
        auto it = s->queue.end();
        while (it != s->queue.begin() && (it - 1)->arrival_ns > r.arrival_ns) --it;
        s->queue.insert(it, r);
        ++s->submitted;
    }
    s->cv_submit.notify_all();
    return r.id;
}

extern "C" int dna_server_poll(dna_server *s, dna_completion *out, uint32_t max, int32_t timeout_ms) {
    if (!s || (!out && max)) return DNA_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_ms != 0) {
        auto pred = [&] { return !s->done.empty(); };
        if (timeout_ms < 0) s->cv_done.wait(lk, pred);
        else s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
    }
    uint32_t n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return (int)n;
}

extern "C" int dna_server_drain(dna_server *s, int32_t timeout_ms) {
    if (!s) return DNA_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto pred = [&] { return s->completed == s->submitted; };
    if (timeout_ms < 0) s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return DNA_ERR_TIMEOUT;
    return DNA_OK;
}

extern "C" int dna_server_stats(dna_server *s, dna_server_stats_t *out) {
    if (!s || !out) return DNA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->queued = s->queue.size();
    uint32_t busy = 0;
    for (const Slot &sl : s->slots) busy += sl.busy ? 1u : 0u;
    out->in_flight = busy;
    out->mem_in_use = s->in_use;
    out->mem_cap = s->cap;
    out->slots = (uint32_t)s->slots.size();
    return DNA_OK;
}

extern "C" void dna_server_free(dna_server *s) { destroy(s); }
