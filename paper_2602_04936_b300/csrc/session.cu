// Serving session: resident indexes, memory-budget admission, requests on
// several CUDA streams.
//
// A request moves pending -> in flight -> done.  Admission is first come,
// first served: the oldest waiting request is admitted as soon as fewer than
// max_inflight requests are on the GPU and its device memory fits what the
// budget has left; requests behind it wait (no overtaking, so a large request
// is not starved by a stream of small ones).  Admitted requests go round-robin
// to the session's streams, where their host-to-device copy, search kernels
// and device-to-host copy are ordered; different streams overlap.  Retiring a
// request (its completion event has fired) returns its memory and may admit
// the next ones; this happens inside every submit and poll, so the session
// needs no thread of its own.
//
// Request memory is the session's own: the budget is allocated once, at
// creation, and each admitted request's query, id and LCP buffers are carved
// from it (first fit over a free list that merges neighbours), to be returned
// when the request retires.  No request allocates device memory, so a
// long-running session's latency does not depend on the state of the
// device's shared stream-ordered pool.
#include <chrono>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "index.cuh"

namespace {

enum ReqState { kPending = 0, kInflight = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

struct Req {
    int slot = 0;
    const void* hq = nullptr;
    int64_t Q = 0;
    int k = 0;
    int32_t* hid = nullptr;
    uint8_t* hlcp = nullptr;
    int64_t bytes = 0;   // accounted against the budget
    int64_t blk = 0;     // bytes of its block in the slab
    int64_t off = -1;    // the block's offset (-1: none held)
    int state = kPending;
    int rc = LCP_OK;
    int stream = 0;
    cudaEvent_t ev = nullptr;
};

}  // namespace

// A slot answered by the full scan: resident tokens instead of an index.
struct ScanSlot {
    const void* tokens = nullptr;  // null: an index slot
    int64_t N = 0;
    int tb = 0, L = 0;
};

struct lcp_session_s {
    lcp_session_cfg_t cfg{};
    int device = 0;
    std::mutex mu;
    std::vector<lcp_index_t> idx;
    std::vector<ScanSlot> scan;  // per slot
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> spare_events;
    std::deque<uint64_t> pending;
    std::vector<uint64_t> inflight;  // tickets on the GPU (at most max_inflight)
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_ticket = 1;
    int rr = 0;
    lcp_session_stats_t st{};
    char* slab = nullptr;                 // mem_budget + kSlabSlack bytes of device memory
    std::map<int64_t, int64_t> free_blk;  // offset -> bytes of the free blocks, merged
};

namespace {

int64_t request_bytes(const lcp_index_s* x, int64_t Q, int k) {
    // queries + ids + lcps + the search's per-query position record
    return Q * ((int64_t)x->L * x->tb + 16 + 5 * (int64_t)k);
}

constexpr int64_t round256(int64_t b) { return (b + 255) & ~(int64_t)255; }

// The slab holds the budget plus this much, so that any request within the
// budget (whose three buffers are rounded up to 256 bytes each) fits an empty
// slab.
constexpr int64_t kSlabSlack = 1024;

int64_t slab_block(int64_t row_bytes, int64_t Q, int k) {
    return round256(Q * row_bytes) + round256(Q * 4 * (int64_t)k) + round256(Q * (int64_t)k);
}

// First fit; -1 when no free block is large enough.
int64_t slab_take(lcp_session_s* s, int64_t bytes) {
    for (auto it = s->free_blk.begin(); it != s->free_blk.end(); ++it) {
        if (it->second < bytes) continue;
        const int64_t off = it->first, rest = it->second - bytes;
        s->free_blk.erase(it);
        if (rest > 0) s->free_blk.emplace(off + bytes, rest);
        return off;
    }
    return -1;
}

void slab_give(lcp_session_s* s, int64_t off, int64_t bytes) {
    auto it = s->free_blk.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != s->free_blk.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_blk.erase(nx);
    }
    if (it != s->free_blk.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_blk.erase(it);
        }
    }
}

// Enqueues the request's copies and kernels on its stream (lock held).
int launch(lcp_session_s* s, Req& r) {
    if (s->cfg.dry_run) return LCP_OK;
    lcp_index_s* x = s->idx[r.slot];
    const ScanSlot& sc = s->scan[r.slot];
    cudaStream_t st = s->streams[r.stream];
    const size_t qb = (size_t)r.Q * (x ? x->L * x->tb : sc.L * sc.tb);
    const size_t ib = (size_t)r.Q * r.k * sizeof(int32_t), lb = (size_t)r.Q * r.k;
    if (r.Q > 0) {
        char* base = s->slab + r.off;
        void* dq = base;
        int32_t* did = reinterpret_cast<int32_t*>(base + round256((int64_t)qb));
        uint8_t* dl = reinterpret_cast<uint8_t*>(base + round256((int64_t)qb) + round256((int64_t)ib));
        // queries and outputs may be host or device memory: unified
        // addressing tells the copy engine which
        LCP_CUDA_TRY(cudaMemcpyAsync(dq, r.hq, qb, cudaMemcpyDefault, st));
        int rc = x ? lcp_topk_batch(x, dq, r.Q, r.k, did, dl, st)
                   : lcph::scan_topk_device(sc.tokens, sc.N, sc.tb, sc.L, dq, r.Q, r.k, did, dl, st);
        if (rc != LCP_OK) return rc;
        LCP_CUDA_TRY(cudaMemcpyAsync(r.hid, did, ib, cudaMemcpyDefault, st));
        LCP_CUDA_TRY(cudaMemcpyAsync(r.hlcp, dl, lb, cudaMemcpyDefault, st));
    }
    if (s->spare_events.empty()) {
        LCP_CUDA_TRY(cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming));
    } else {
        r.ev = s->spare_events.back();
        s->spare_events.pop_back();
    }
    LCP_CUDA_TRY(cudaEventRecord(r.ev, st));
    return LCP_OK;
}

void finish(lcp_session_s* s, Req& r, int state, int rc) {
    r.state = state;
    r.rc = rc;
    s->st.inflight--;
    s->st.mem_in_use -= r.bytes;
    if (r.off >= 0) {
        slab_give(s, r.off, r.blk);
        r.off = -1;
    }
    if (state == kDone) s->st.completed++;
    if (r.ev) {
        s->spare_events.push_back(r.ev);
        r.ev = nullptr;
    }
}

// Retires finished requests (if `retire`) and admits waiting ones (lock held).
// Only the requests on the GPU are looked at (one event query each), so a
// pump costs at most max_inflight queries however many requests wait or
// await their poll.  Dry-run requests finish when retired, i.e. on the next
// poll.
void pump(lcp_session_s* s, bool retire = true) {
    for (size_t i = 0; retire && i < s->inflight.size();) {
        Req& r = s->reqs[s->inflight[i]];
        bool gone = true;
        if (s->cfg.dry_run) {
            finish(s, r, kDone, LCP_OK);
        } else {
            cudaError_t e = cudaEventQuery(r.ev);
            if (e == cudaSuccess) finish(s, r, kDone, LCP_OK);
            else if (e != cudaErrorNotReady) finish(s, r, kFailed, lcph::cuda_status(e));
            else gone = false;
        }
        if (gone) {
            s->inflight[i] = s->inflight.back();
            s->inflight.pop_back();
        } else {
            ++i;
        }
    }
    while (!s->pending.empty()) {
        auto it = s->reqs.find(s->pending.front());
        if (it == s->reqs.end() || it->second.state != kPending) {
            s->pending.pop_front();
            continue;
        }
        Req& r = it->second;
        if (s->st.inflight >= s->cfg.max_inflight || s->st.mem_in_use + r.bytes > s->cfg.mem_budget) break;
        if (!s->cfg.dry_run && r.Q > 0) {
            // a block of the slab, or wait for retirements (an empty slab
            // always fits a request within the budget)
            r.off = slab_take(s, r.blk);
            if (r.off < 0) break;
        }
        const uint64_t ticket = s->pending.front();
        s->pending.pop_front();
        s->st.pending--;
        r.state = kInflight;
        r.stream = s->rr;
        s->rr = (s->rr + 1) % (int)s->cfg.streams;
        s->st.inflight++;
        s->st.admitted++;
        s->st.mem_in_use += r.bytes;
        if (s->st.mem_in_use > s->st.mem_peak) s->st.mem_peak = s->st.mem_in_use;
        int rc = launch(s, r);
        if (rc != LCP_OK) {
            // copies already enqueued may still use the block
            cudaStreamSynchronize(s->streams[r.stream]);
            finish(s, r, kFailed, rc);
        } else {
            s->inflight.push_back(ticket);
        }
    }
}

}  // namespace

extern "C" {

int lcp_session_create(const lcp_session_cfg_t* cfg, lcp_session_t* out) {
    if (!cfg || !out) return LCP_ERR_INVALID;
    *out = nullptr;
    if (cfg->mem_budget <= 0 || cfg->max_inflight < 1 || cfg->streams < 1 || cfg->streams > 64)
        return LCP_ERR_INVALID;
    lcp_session_s* s = new (std::nothrow) lcp_session_s();
    if (!s) return LCP_ERR_OOM;
    s->cfg = *cfg;
    if (!cfg->dry_run) {
        cudaGetDevice(&s->device);
        for (int i = 0; i < cfg->streams; ++i) {
            cudaStream_t st;
            cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
                delete s;
                return lcph::cuda_status(e);
            }
            s->streams.push_back(st);
        }
        // the requests' memory, once
        const int64_t slab_bytes = cfg->mem_budget + kSlabSlack;
        cudaError_t e = cudaMalloc((void**)&s->slab, (size_t)slab_bytes);
        if (e != cudaSuccess) {
            for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
            delete s;
            return lcph::cuda_status(e);
        }
        s->free_blk.emplace(0, slab_bytes);
    }
    *out = s;
    return LCP_OK;
}

int lcp_session_add_index(lcp_session_t s, lcp_index_t index, int32_t* slot) {
    if (!s || (!index && !s->cfg.dry_run) || !slot || (index && lcph::index_is_wide(index)))
        return LCP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    if (index) index->shared = true;  // used on the session's streams from now on
    s->idx.push_back(index);
    s->scan.push_back(ScanSlot());
    *slot = (int32_t)s->idx.size() - 1;
    return LCP_OK;
}

int lcp_session_add_scan(lcp_session_t s, const void* d_tokens, int64_t N, lcp_format_t fmt, int32_t* slot) {
    if (!s || !slot || N < 1 || N >= (1ll << 30) || !d_tokens || (fmt.token_bytes != 1 && fmt.token_bytes != 2) ||
        fmt.L < 1 || fmt.L > LCP_MAX_L)
        return LCP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    ScanSlot sc;
    sc.tokens = d_tokens;
    sc.N = N;
    sc.tb = fmt.token_bytes;
    sc.L = fmt.L;
    s->idx.push_back(nullptr);
    s->scan.push_back(sc);
    *slot = (int32_t)s->idx.size() - 1;
    return LCP_OK;
}

int lcp_session_submit(lcp_session_t s, int32_t slot, const void* h_queries, int64_t Q, int32_t k,
                       int32_t* h_out_ids, uint8_t* h_out_lcp, uint64_t* ticket) {
    if (!s || !ticket || Q < 0 || k < 1) return LCP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    if (slot < 0 || slot >= (int32_t)s->idx.size()) return LCP_ERR_INVALID;
    lcp_index_s* x = s->idx[slot];
    const ScanSlot& sc = s->scan[slot];
    int64_t bytes;
    int64_t blk = 0;
    if (x) {
        if (k > x->max_k) return LCP_ERR_INVALID;
        bytes = request_bytes(x, Q, k);
        blk = slab_block((int64_t)x->L * x->tb, Q, k);
    } else if (sc.tokens) {
        if (k > LCP_SCAN_MAX_K) return LCP_ERR_INVALID;
        bytes = Q * ((int64_t)sc.L * sc.tb + 5 * (int64_t)k);  // queries + results
        blk = slab_block((int64_t)sc.L * sc.tb, Q, k);
    } else {
        bytes = Q * (16 + 5 * (int64_t)k);  // dry run without an index
    }
    if (Q > 0 && (!h_queries || !h_out_ids || !h_out_lcp)) return LCP_ERR_INVALID;
    s->st.submitted++;
    if (bytes > s->cfg.mem_budget) {
        s->st.rejected++;
        return LCP_ERR_BUDGET;
    }
    Req r;
    r.slot = slot;
    r.hq = h_queries;
    r.Q = Q;
    r.k = k;
    r.hid = h_out_ids;
    r.hlcp = h_out_lcp;
    r.bytes = bytes;
    r.blk = blk;
    const uint64_t t = s->next_ticket++;
    s->reqs.emplace(t, r);
    s->pending.push_back(t);
    s->st.pending++;
    *ticket = t;
    if (!s->cfg.dry_run) cudaSetDevice(s->device);
    pump(s, !s->cfg.dry_run);
    return LCP_OK;
}

int lcp_session_poll(lcp_session_t s, uint64_t ticket, int32_t timeout_ms) {
    if (!s) return LCP_ERR_INVALID;
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms > 0 ? timeout_ms : 0);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (!s->cfg.dry_run) cudaSetDevice(s->device);
            pump(s);
            auto it = s->reqs.find(ticket);
            if (it == s->reqs.end()) return LCP_ERR_INVALID;
            const int state = it->second.state;
            if (state == kDone || state == kFailed || state == kCancelled) {
                const int rc = state == kDone ? LCP_OK : (state == kCancelled ? LCP_ERR_STATE : it->second.rc);
                s->reqs.erase(it);
                return rc;
            }
        }
        if (std::chrono::steady_clock::now() >= t_end) return LCP_PENDING;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int lcp_session_stats(lcp_session_t s, lcp_session_stats_t* stats) {
    if (!s || !stats) return LCP_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    *stats = s->st;
    return LCP_OK;
}

int lcp_session_destroy(lcp_session_t s) {
    if (!s) return LCP_OK;
    int rc = LCP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (uint64_t t : s->pending) {
            auto it = s->reqs.find(t);
            if (it != s->reqs.end() && it->second.state == kPending) it->second.state = kCancelled;
        }
        s->pending.clear();
    }
    // wait for the requests on the GPU, bounded
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::seconds(10);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (!s->cfg.dry_run) cudaSetDevice(s->device);
            pump(s);
            if (s->st.inflight == 0) break;
        }
        if (std::chrono::steady_clock::now() >= t_end) {
            rc = LCP_ERR_TIMEOUT;
            break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    if (!s->cfg.dry_run) {
        for (auto& kv : s->reqs)
            if (kv.second.ev) cudaEventDestroy(kv.second.ev);
        for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
        if (rc == LCP_OK) {  // (after a timeout, memory the GPU may still use is kept)
            for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
            cudaFree(s->slab);
        }
    }
    delete s;
    return rc;
}

int lcp_session_replay(lcp_session_t s, const lcp_replay_req_t* reqs, int64_t n, double timeout_s,
                       double* latency_s, double* wall_s) {
    if (!s || n < 0 || (n > 0 && (!reqs || !latency_s)) || timeout_s <= 0) return LCP_ERR_INVALID;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    std::deque<std::pair<uint64_t, int64_t>> out;  // (ticket, request) in submission order
    int64_t next = 0;
    int rc_all = LCP_OK;
    double last_done = 0.0;
    while (next < n || !out.empty()) {
        const double now = now_s();
        if (now > timeout_s) {
            rc_all = LCP_ERR_TIMEOUT;
            break;
        }
        bool progress = false;
        while (next < n && reqs[next].arrival_s <= now) {
            const lcp_replay_req_t& r = reqs[next];
            uint64_t t = 0;
            const int rc = lcp_session_submit(s, r.slot, r.h_queries, r.Q, r.k, r.h_out_ids, r.h_out_lcp, &t);
            if (rc == LCP_OK) out.emplace_back(t, next);
            else latency_s[next] = -1.0;
            ++next;
            progress = true;
        }
        // one pump, then the outstanding requests' states (a poll per
        // request would pump once each)
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (!s->cfg.dry_run) cudaSetDevice(s->device);
            pump(s);
            double t = -1.0;
            for (auto it = out.begin(); it != out.end();) {
                auto rit = s->reqs.find(it->first);
                int rc = LCP_ERR_INVALID;
                if (rit != s->reqs.end()) {
                    const int state = rit->second.state;
                    if (state != kDone && state != kFailed && state != kCancelled) {
                        ++it;
                        continue;
                    }
                    rc = state == kDone ? LCP_OK : (state == kCancelled ? LCP_ERR_STATE : rit->second.rc);
                    s->reqs.erase(rit);
                }
                if (t < 0) t = now_s();
                latency_s[it->second] = rc == LCP_OK ? t - reqs[it->second].arrival_s : -1.0;
                if (t > last_done) last_done = t;
                if (rc != LCP_OK && rc_all == LCP_OK) rc_all = rc;
                it = out.erase(it);
                progress = true;
            }
        }
        if (!progress) std::this_thread::yield();
    }
    if (wall_s) *wall_s = n > 0 ? last_done - reqs[0].arrival_s : 0.0;
    return rc_all;
}

}  // extern "C"
