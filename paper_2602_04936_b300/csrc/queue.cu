// Work queue feeding one persistent search kernel (host side; the worker is
// k_queue_worker in search.cu).
//
// Requests against any resident indexes -- uneven N, L and k -- are cut into
// tasks of up to `chunk` queries.  The request record and its task records
// are written to pinned memory and copied to device memory on a copy stream,
// and the new task count is copied after them on the same stream, so the
// count never lands before the records it covers.  The worker reads device
// memory only (a running kernel does not reliably observe host writes to
// mapped memory it has read before); its warps claim tasks with a
// compare-and-swap on a device counter, so one launch serves every request
// that arrives while it runs.  Completion travels back the other way: the
// request's ticket is written into mapped host memory after a system-scope
// fence.  A warp that finds no work for idle_ms exits; when the last one has
// exited the host relaunches the worker on the next submit or poll that
// finds work outstanding, so no device wait is unbounded and no work is lost
// between an exit and a publish.
#include <cuda/atomic>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <vector>
#include <mutex>
#include <new>
#include <thread>

#include "search.cuh"

struct QueueInflight {
    uint64_t ticket;
    int32_t slot;
    int32_t ntasks;
};

struct lcp_queue_s {
    int device = 0;
    int rcap = 0, tcap = 0, ctas = 0;
    double idle_ms = 0;
    // pinned host staging (stable until the request that wrote it completes)
    lcpk::QReq* h_reqs = nullptr;
    lcpk::QTask* h_tasks = nullptr;
    int64_t* h_pub = nullptr;  // [rcap] task count after each slot's request
    int32_t* h_stop = nullptr;
    uint64_t* done = nullptr;  // mapped: written by the device
    void* pinned = nullptr;
    void* dev = nullptr;       // device: ctl, reqs, tasks, claimed, done_count
    lcpk::QueueArgs args;
    cudaStream_t ws = nullptr;  // the worker's stream
    cudaStream_t cs = nullptr;  // record and count copies
    cudaEvent_t ev = nullptr;
    bool launched = false;
    int64_t published = 0;
    uint64_t next_ticket = 1;
    int64_t inflight_tasks = 0;
    std::deque<QueueInflight> inflight;
    std::deque<int32_t> free_slots;
    int64_t launches = 0;
    std::mutex mu;
};

namespace {

bool worker_running(lcp_queue_s* q) {
    return q->launched && cudaEventQuery(q->ev) == cudaErrorNotReady;
}

int ensure_worker(lcp_queue_s* q) {  // caller holds mu
    if (q->inflight.empty() || worker_running(q)) return LCP_OK;
    cudaGetLastError();  // a completed event query leaves no error, a not-ready one is expected
    lcph::launch_queue_worker(q->args, (unsigned)q->ctas, q->ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lcph::cuda_status(e);
    cudaEventRecord(q->ev, q->ws);
    q->launched = true;
    q->launches++;
    return LCP_OK;
}

// Retires completed requests at the front of the in-flight list (their
// slots and task room become free).  Caller holds mu.
void reap(lcp_queue_s* q) {
    while (!q->inflight.empty()) {
        const QueueInflight& f = q->inflight.front();
        const uint64_t seen = cuda::atomic_ref<uint64_t, cuda::thread_scope_system>(q->done[f.slot]).load(cuda::memory_order_acquire);
        if (seen != f.ticket) break;
        q->free_slots.push_back(f.slot);
        q->inflight_tasks -= f.ntasks;
        q->inflight.pop_front();
    }
}

bool is_done(lcp_queue_s* q, uint64_t ticket) {  // caller holds mu
    if (ticket == 0 || ticket >= q->next_ticket) return false;
    // in-flight tickets are ascending: binary search
    auto it = std::lower_bound(q->inflight.begin(), q->inflight.end(), ticket,
                               [](const QueueInflight& f, uint64_t t) { return f.ticket < t; });
    if (it == q->inflight.end() || it->ticket != ticket) return true;  // retired (or answered at submit)
    return cuda::atomic_ref<uint64_t, cuda::thread_scope_system>(q->done[it->slot]).load(cuda::memory_order_acquire) ==
           ticket;
}

}  // namespace

extern "C" {

int lcp_queue_create(const lcp_queue_cfg_t* cfg, lcp_queue_t* out) {
    if (!cfg || !out || cfg->max_requests < 1 || cfg->max_requests > (1 << 16) || cfg->max_tasks < 1 ||
        cfg->max_tasks > (1 << 24) || cfg->idle_ms <= 0 || cfg->ctas_per_sm < 1 || cfg->ctas_per_sm > 32)
        return LCP_ERR_INVALID;
    *out = nullptr;
    lcp_queue_s* q = new (std::nothrow) lcp_queue_s();
    if (!q) return LCP_ERR_OOM;
    cudaGetDevice(&q->device);
    q->rcap = cfg->max_requests;
    q->tcap = cfg->max_tasks;
    q->idle_ms = cfg->idle_ms;
    q->ctas = lcph::sm_count() * cfg->ctas_per_sm;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_reqs = up(sizeof(lcpk::QReq) * q->rcap), b_tasks = up(sizeof(lcpk::QTask) * q->tcap);
    const size_t b_pub = up(sizeof(int64_t) * q->rcap), b_done = up(sizeof(uint64_t) * q->rcap);
    const size_t pinned_bytes = b_reqs + b_tasks + b_pub + 256 + b_done;
    const size_t b_ctl = up(sizeof(lcpk::QCtl)), b_claim = 256, b_cnt = up(sizeof(int32_t) * q->rcap);
    const size_t b_taken = up(sizeof(int64_t) * q->tcap);
    const size_t dev_bytes = b_ctl + b_reqs + b_tasks + b_claim + b_cnt + b_taken;
    cudaError_t e = cudaHostAlloc(&q->pinned, pinned_bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaMalloc(&q->dev, dev_bytes);
    if (e == cudaSuccess) e = cudaMemset(q->dev, 0, dev_bytes - b_taken);
    if (e == cudaSuccess) e = cudaMemset(static_cast<char*>(q->dev) + dev_bytes - b_taken, 0xFF, b_taken);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->ws, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (q->pinned) cudaFreeHost(q->pinned);
        cudaFree(q->dev);
        if (q->ws) cudaStreamDestroy(q->ws);
        if (q->cs) cudaStreamDestroy(q->cs);
        delete q;
        return lcph::cuda_status(e);
    }
    memset(q->pinned, 0, pinned_bytes);
    {
        const int64_t none = INT64_MAX;  // no id abandoned yet
        e = cudaMemcpy(static_cast<char*>(q->dev) + b_ctl + b_reqs + b_tasks + 128, &none, sizeof(none),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFreeHost(q->pinned);
            cudaFree(q->dev);
            cudaStreamDestroy(q->ws);
            cudaStreamDestroy(q->cs);
            cudaEventDestroy(q->ev);
            delete q;
            return lcph::cuda_status(e);
        }
    }
    char* h = static_cast<char*>(q->pinned);
    q->h_reqs = reinterpret_cast<lcpk::QReq*>(h);
    q->h_tasks = reinterpret_cast<lcpk::QTask*>(h + b_reqs);
    q->h_pub = reinterpret_cast<int64_t*>(h + b_reqs + b_tasks);
    q->h_stop = reinterpret_cast<int32_t*>(h + b_reqs + b_tasks + b_pub);
    q->done = reinterpret_cast<uint64_t*>(h + b_reqs + b_tasks + b_pub + 256);
    char* dd = nullptr;
    cudaHostGetDevicePointer((void**)&dd, q->done, 0);
    char* d = static_cast<char*>(q->dev);
    lcpk::QueueArgs& a = q->args;
    a.ctl = reinterpret_cast<const lcpk::QCtl*>(d);
    a.reqs = reinterpret_cast<const lcpk::QReq*>(d + b_ctl);
    a.tasks = reinterpret_cast<const lcpk::QTask*>(d + b_ctl + b_reqs);
    a.claimed = reinterpret_cast<int64_t*>(d + b_ctl + b_reqs + b_tasks);
    a.min_abandoned = reinterpret_cast<int64_t*>(d + b_ctl + b_reqs + b_tasks + 128);  // own cache line
    a.exited = reinterpret_cast<unsigned*>(d + b_ctl + b_reqs + b_tasks + 192);
    a.taken = reinterpret_cast<int64_t*>(d + dev_bytes - b_taken);
    a.done_count = reinterpret_cast<int32_t*>(d + b_ctl + b_reqs + b_tasks + b_claim);
    a.done = reinterpret_cast<uint64_t*>(dd);
    a.rcap = q->rcap;
    a.tcap = q->tcap;
    a.idle_ns = (long long)(cfg->idle_ms * 1e6);
    a.status = lcph::lib_status_word();
    for (int s = 0; s < q->rcap; ++s) q->free_slots.push_back(s);
    *out = q;
    return LCP_OK;
}

int lcp_queue_submit(lcp_queue_t q, lcp_index_t x, const void* d_queries, int64_t Q, int32_t k,
                     int32_t* d_out_ids, uint8_t* d_out_lcp, uint64_t* ticket) {
    if (!q || !x || !ticket || Q < 0 || k < 1 || k > x->max_k || lcph::index_is_wide(x)) return LCP_ERR_INVALID;
    if (Q > 0 && (!d_queries || !d_out_ids || !d_out_lcp)) return LCP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(q->mu);
    x->shared = true;  // read by the persistent worker from now on
    if (Q == 0 || x->N == 0) {  // nothing to search: answered here (padding)
        if (Q > 0) {
            cudaMemsetAsync(d_out_ids, 0xFF, sizeof(int32_t) * (size_t)Q * k, q->ws);
            cudaMemsetAsync(d_out_lcp, 0, (size_t)Q * k, q->ws);
            cudaStreamSynchronize(q->ws);
        }
        *ticket = q->next_ticket++;
        return LCP_OK;
    }
    // tasks small enough to spread one request over every worker warp (a
    // warp answers its task's queries one after another), at most 32
    // queries, and larger for huge requests so a request never needs more
    // than a quarter of the ring
    const int64_t warps = (int64_t)q->ctas * lcpk::kSearchWarps;
    int64_t chunk = (Q + warps - 1) / warps;
    chunk = chunk < 1 ? 1 : (chunk > 32 ? 32 : chunk);
    while ((Q + chunk - 1) / chunk > q->tcap / 4 && chunk < (1ll << 30)) chunk <<= 1;
    const int64_t ntasks = (Q + chunk - 1) / chunk;
    reap(q);
    if (q->free_slots.empty() || q->inflight_tasks + ntasks > q->tcap) return LCP_ERR_CAPACITY;
    const int32_t slot = q->free_slots.front();
    q->free_slots.pop_front();
    lcpk::QReq& r = q->h_reqs[slot];
    r.ix = lcph::dev_view(x);
    r.queries = reinterpret_cast<const uint8_t*>(d_queries);
    r.qf = lcpk::make_fmt(x->tb, x->L, d_queries);
    r.k = k;
    r.ntasks = (int32_t)ntasks;
    r.out_ids = d_out_ids;
    r.out_lcp = d_out_lcp;
    r.ticket = q->next_ticket++;
    const int64_t t0 = q->published % q->tcap;
    for (int64_t j = 0; j < ntasks; ++j) {
        lcpk::QTask& t = q->h_tasks[(t0 + j) % q->tcap];
        t.q0 = j * chunk;
        t.q1 = (j + 1) * chunk < Q ? (j + 1) * chunk : Q;
        t.slot = slot;
    }
    // records first, then the count that covers them (one stream: in order)
    cudaError_t e = cudaMemcpyAsync(const_cast<lcpk::QReq*>(q->args.reqs) + slot, &r, sizeof(lcpk::QReq),
                                    cudaMemcpyHostToDevice, q->cs);
    const int64_t first = ntasks < q->tcap - t0 ? ntasks : q->tcap - t0;
    lcpk::QTask* dt = const_cast<lcpk::QTask*>(q->args.tasks);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dt + t0, q->h_tasks + t0, sizeof(lcpk::QTask) * first, cudaMemcpyHostToDevice, q->cs);
    if (e == cudaSuccess && ntasks > first)
        e = cudaMemcpyAsync(dt, q->h_tasks, sizeof(lcpk::QTask) * (ntasks - first), cudaMemcpyHostToDevice, q->cs);
    q->published += ntasks;
    q->h_pub[slot] = q->published;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<int64_t*>(&q->args.ctl->published), &q->h_pub[slot], sizeof(int64_t),
                            cudaMemcpyHostToDevice, q->cs);
    if (e != cudaSuccess) return lcph::cuda_status(e);
    q->inflight.push_back({r.ticket, slot, (int32_t)ntasks});
    q->inflight_tasks += ntasks;
    *ticket = r.ticket;
    return ensure_worker(q);
}

int lcp_queue_poll(lcp_queue_t q, uint64_t ticket, int32_t timeout_ms) {
    if (!q || ticket == 0) return LCP_ERR_INVALID;
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms > 0 ? timeout_ms : 0);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(q->mu);
            if (ticket >= q->next_ticket) return LCP_ERR_INVALID;
            if (is_done(q, ticket)) {
                reap(q);
                return LCP_OK;
            }
            int rc = ensure_worker(q);  // (no device-wide sync here: the worker may be running)
            if (rc != LCP_OK) return rc;
        }
        if (std::chrono::steady_clock::now() >= t_end) return LCP_PENDING;
        std::this_thread::yield();
    }
}

int lcp_queue_stats(lcp_queue_t q, int64_t* inflight, int64_t* worker_launches) {
    if (!q) return LCP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(q->mu);
    reap(q);
    if (inflight) *inflight = (int64_t)q->inflight.size();
    if (worker_launches) *worker_launches = q->launches;
    return LCP_OK;
}

int lcp_queue_replay(lcp_queue_t q, const lcp_queue_replay_req_t* reqs, int64_t n, double timeout_s,
                     double* latency_s, double* wall_s) {
    if (!q || n < 0 || (n > 0 && (!reqs || !latency_s)) || timeout_s <= 0) return LCP_ERR_INVALID;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    struct Out {
        uint64_t ticket;
        int64_t req;
        int32_t slot;
    };
    std::vector<Out> out;
    int64_t next = 0;
    int rc_all = LCP_OK;
    double last_done = 0.0;
    while (next < n || !out.empty()) {
        const double now = now_s();
        if (now > timeout_s) {
            rc_all = LCP_ERR_TIMEOUT;
            break;
        }
        // completions first (a completed request's slot may be reused by a
        // submission below; is_done also answers for retired tickets)
        {
            std::lock_guard<std::mutex> lk(q->mu);
            for (size_t i = 0; i < out.size();) {
                if (is_done(q, out[i].ticket)) {
                    const double t = now_s();
                    latency_s[out[i].req] = t - reqs[out[i].req].arrival_s;
                    last_done = t;
                    out[i] = out.back();
                    out.pop_back();
                } else {
                    ++i;
                }
            }
        }
        // submit every request whose arrival time has come (FIFO: a request
        // the queue has no room for waits, and so do the ones behind it)
        while (next < n && reqs[next].arrival_s <= now) {
            const lcp_queue_replay_req_t& r = reqs[next];
            uint64_t t = 0;
            const int rc = lcp_queue_submit(q, r.index, r.d_queries, r.Q, r.k, r.d_out_ids, r.d_out_lcp, &t);
            if (rc == LCP_ERR_CAPACITY) break;
            if (rc != LCP_OK) {
                latency_s[next] = -1.0;
            } else {
                int32_t slot = -1;
                {
                    std::lock_guard<std::mutex> lk(q->mu);
                    if (!q->inflight.empty() && q->inflight.back().ticket == t) slot = q->inflight.back().slot;
                }
                if (slot < 0) latency_s[next] = now_s() - r.arrival_s;  // answered at submit
                else out.push_back({t, next, slot});
            }
            ++next;
        }
        {
            std::lock_guard<std::mutex> lk(q->mu);
            reap(q);
            const int rc = ensure_worker(q);
            if (rc != LCP_OK) {
                rc_all = rc;
                break;
            }
        }
    }
    for (const auto& o : out) latency_s[o.req] = -1.0;
    if (wall_s) *wall_s = last_done;
    return rc_all;
}

int lcp_queue_destroy(lcp_queue_t q) {
    if (!q) return LCP_OK;
    int rc = LCP_OK;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        reap(q);
        if (!q->inflight.empty()) rc = LCP_ERR_STATE;  // outstanding work is waited for below
    }
    // outstanding requests finish (the worker is relaunched if needed; at
    // most 30 s), then stop makes idle warps leave at once
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::seconds(30);
    while (rc == LCP_ERR_STATE && std::chrono::steady_clock::now() < t_end) {
        uint64_t last;
        {
            std::lock_guard<std::mutex> lk(q->mu);
            if (q->inflight.empty()) break;
            last = q->inflight.back().ticket;
        }
        int p = lcp_queue_poll(q, last, 1000);
        if (p != LCP_OK && p != LCP_PENDING) break;
    }
    *q->h_stop = 1;
    cudaMemcpyAsync(const_cast<int32_t*>(&q->args.ctl->stop), q->h_stop, sizeof(int32_t), cudaMemcpyHostToDevice,
                    q->cs);
    cudaStreamSynchronize(q->cs);
    cudaStreamSynchronize(q->ws);
    cudaEventDestroy(q->ev);
    cudaStreamDestroy(q->ws);
    cudaStreamDestroy(q->cs);
    cudaFree(q->dev);
    cudaFreeHost(q->pinned);
    delete q;
    return LCP_OK;
}

}  // extern "C"
